"""Host logic of bench.py that its JSON line rests on (no GPU): the
algorithmic byte counts of the dominant kernels, the measured peak, and the
rule that an ncu traffic record is used only while the kernel's source is
the one it was captured on."""
import json

import pytest

import bench

N20, M20 = 1_048_576, 16_586_703      # R-MAT scale 20, edge factor 16, seed 1, after cleaning


def test_fp32_pass_bytes():
    # in-CSR 4(n+1) + 4m, degrees 4n, then per node and column: z_e gathered,
    # own old row, z_e written, r_f read (16 B) or, at the ideal-cache minimum, 12 B
    base = 4 * (N20 + 1) + 4 * M20 + 4 * N20
    assert bench.fp32_pass_bytes(N20, M20, 64) == base + 16 * N20 * 64
    assert bench.fp32_pass_bytes_min(N20, M20, 64) == base + 12 * N20 * 64
    assert round(bench.fp32_pass_bytes(N20, M20, 64) / 1e6, 1) == 1148.5
    assert round(bench.fp32_pass_bytes_min(N20, M20, 64) / 1e6) == 880


def test_sweep_bytes():
    # in-CSR, per-node scales (12 B), the Q1.63 tile read and written once
    assert bench.sweep_bytes(N20, M20, 64) == 4 * (N20 + 1) + 4 * M20 + 12 * N20 + 16 * N20 * 64
    assert round(bench.sweep_bytes(N20, M20, 64) / 1e6, 1) == 1156.9


def test_peak_is_the_measured_copy_bandwidth():
    """The measured copy bandwidth when the machine's peaks file is present,
    else the stated fallback, labelled as such."""
    path = bench.os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    peak, kind = bench.peaks()
    if not bench.os.path.exists(path):
        assert (peak, kind) == (6800.0, "fallback")
        return
    with open(path) as f:
        assert peak == float(json.load(f)["hbm_gbs"]) and kind == "measured"


@pytest.mark.parametrize("kernel,workload", [("refine_pass_kernel", "rmat20-k64"), ("walk_kernel", "rmat22-approx")])
def test_traffic_record_follows_the_kernel_source(monkeypatch, kernel, workload):
    fname, sources = bench.TRAFFIC_FILES[kernel]
    with open(bench.os.path.join(bench.ROOT, "profiles", fname)) as f:
        rec = json.load(f)
    if rec["kernel_source_sha"] == bench.kernel_source_sha(sources):
        per = rec.get("per_workload", {})
        want = per[workload]["dram_bytes_per_launch"] if workload in per else rec["dram_bytes_per_launch"]
        assert bench.ncu_traffic(workload, kernel) == float(want)
    else:
        # the kernel changed since the capture: the line reports no traffic
        assert bench.ncu_traffic(workload, kernel) is None
        return
    assert bench.ncu_traffic("rmat22-k1", kernel) is None           # captured on another workload
    monkeypatch.setattr(bench, "kernel_source_sha", lambda sources=(): "0" * 16)
    assert bench.ncu_traffic(workload, kernel) is None              # the kernel changed since the capture


def test_unknown_kernel_has_no_traffic():
    assert bench.ncu_traffic("rmat22-index", "index_query_kernel") is None


def test_hp_roofline_entry():
    """The dominant kernel is the FP32 pass when the query ran any (its bytes
    over its average launch time), else the Q1.63 pass."""
    r = bench.hp_roofline(N20, M20, 64, fp32_ms=33.26, fp32_launches=100, sweep_ms=5.0, sweep_launches=10,
                          workload="none")
    assert r["kernel"] == "refine_pass_kernel<64, float>"
    assert abs(r["achieved"] - bench.fp32_pass_bytes(N20, M20, 64) / 0.3326e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["traffic"] is None                                       # no capture for this workload
    r = bench.hp_roofline(N20, M20, 64, fp32_ms=0.0, fp32_launches=0, sweep_ms=6.0, sweep_launches=10,
                          workload="none")
    assert r["kernel"] == "sweep_kernel<64>"
    assert abs(r["achieved"] - bench.sweep_bytes(N20, M20, 64) / 0.6e-3 / 1e9) < 1e-6


def test_autotuner_calibrates_on_other_sources():
    import ppr_inputs as gen
    n = N20
    timed = set(gen.sources(n, 64, seed=bench.replica_seed(2, 0)).tolist())
    calib = bench.calibration_sources(n, 64, 0)
    assert len(calib) == 128                # two tiles per calibration call at 64 sources
    assert len(bench.calibration_sources(n, 10, 0)) == 10   # below 64, the same bucket needs the same k
    assert len(timed & set(calib.tolist())) <= 4      # independent draws may share a few nodes, not the batch
    assert bench.calibration_sources(n, 64, 1).tolist() != bench.calibration_sources(n, 64, 0).tolist()


def test_serving_admission_halves_then_refuses():
    per_source = lambda k: 100 * k + 50          # workspace bytes of a batch of k
    assert bench.admit_batch(32, 10_000, 0, per_source) == 32
    assert bench.admit_batch(32, 250, 0, per_source) == 2
    assert bench.admit_batch(32, 100, 0, per_source) == 0     # refused: not even one fits
    assert bench.admit_batch(32, 0, 150, per_source) == 1     # the held workspace is reused
    assert bench.admit_batch(3, 349, 0, per_source) == 1      # 3 does not fit, 3 // 2 does


def test_approx_roofline_entry(monkeypatch):
    """Walks: two 32 B sectors per move and per endpoint; index reads: 68 B
    per walk; both per launch (one launch per tile) over the kernel's mean
    event time."""
    monkeypatch.setattr(bench, "ncu_traffic", lambda workload, kernel="sweep_kernel": None)
    st = [{"walks": 1000, "walk_steps": 4000}, {"walks": 3000, "walk_steps": 12000}]
    # two tiles, three steps, 6 ms of walk-kernel time in all: 1 ms per launch
    r = bench.approx_roofline(st, 3, 2, 6.0, 16, False, "rmat22-approx")
    assert r["kernel"] == "walk_kernel<16>"
    assert r["algorithmic_bytes_per_launch"] == 64 * (16000 + 4000) / 2
    assert r["avg_launch_ms"] == pytest.approx(1.0)
    assert r["achieved"] == pytest.approx(64 * 20000 / 2 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.peaks()[0])
    ri = bench.approx_roofline(st, 3, 2, 6.0, 16, True, "rmat22-index")
    assert ri["kernel"] == "index_query_kernel<16>"
    assert ri["algorithmic_bytes_per_launch"] == 68 * 4000 / 2
