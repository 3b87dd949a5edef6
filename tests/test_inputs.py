"""The seeded input generators: deterministic, clean CSR, shapes of the workloads."""
import numpy as np

import oracle as O
import ppr_inputs as gen


def check_clean(rp, ci):
    n = len(rp) - 1
    assert rp[0] == 0 and rp[-1] == len(ci)
    d = np.diff(rp)
    assert d.min() >= 1                                  # no sinks (Sec. 2 assumption)
    assert O.validate(O.Graph(rp, ci)) == 0              # sorted, no dups, no self-loops
    assert ci.min() >= 0 and ci.max() < n


def test_chung_lu_shape_and_determinism():
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    check_clean(rp, ci)
    rp2, ci2 = gen.chung_lu(10_000, 100_000, 2.2, seed=1, threads=1)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    rp3, _ = gen.chung_lu(10_000, 100_000, 2.2, seed=2)
    assert not np.array_equal(rp, rp3)
    d_out = np.diff(rp)
    d_in = np.bincount(ci, minlength=10_000)
    # power-law: heavy tails on both sides
    assert d_out.max() > 50 * d_out.mean() and d_in.max() > 50 * d_in.mean()
    assert 80_000 < len(ci) <= 100_000 + 10_000


def test_rmat_small_shape_and_determinism():
    rp, ci = gen.rmat(14, 16, seed=1)
    check_clean(rp, ci)
    rp2, ci2 = gen.rmat(14, 16, seed=1, threads=3)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    n = 1 << 14
    assert len(rp) == n + 1
    assert 0.6 * 16 * n < len(ci) < 1.1 * 16 * n
    d_in = np.bincount(ci, minlength=n)
    assert d_in.max() > 30 * d_in.mean()


def test_sources_and_subgraph():
    s = gen.sources(10_000, 10, seed=1)
    assert s.dtype == np.int32 and len(s) == 10 and s.min() >= 0 and s.max() < 10_000
    assert np.array_equal(s, gen.sources(10_000, 10, seed=1))
    rp, ci = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
    srp, sci = gen.bfs_subgraph(rp, ci, 0, 200, seed=1)
    assert len(srp) == 201
    check_clean(srp, sci)


def test_benchmark_workload_is_fixed():
    """The 64-source R-MAT scale-20 workload the benchmark and the parity tests
    share: its size after cleaning, a checksum of the CSR and of the sources.
    A change in the generator changes every recorded measurement."""
    import hashlib
    rp, ci = gen.rmat(20, 16, seed=1)
    assert (len(rp) - 1, len(ci)) == (1_048_576, 16_586_703)
    assert hashlib.sha256(rp.tobytes() + ci.tobytes()).hexdigest()[:16] == "6af68c985594cb03"
    s = gen.sources(len(rp) - 1, 64, seed=2)
    assert s[:4].tolist() == [577067, 931816, 260467, 971048] and int(s.sum()) == 36578074
