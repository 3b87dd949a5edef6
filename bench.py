#!/usr/bin/env python
"""Throughput of high-precision SSPPR queries (l1 <= 1e-8) on one GB300.

Workload (default ``rmat20-k64``): R-MAT scale 20, edge factor 16,
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), duplicates and self-loops removed,
sinks patched; alpha = 0.2, lambda = 1e-8; one step = one batch of 64 uniform
random sources (seed 2) answered by one ``ppr_sssp_query`` call.  Synthetic
data: the graph stands in for the paper's SNAP graphs.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle
(Algorithm 3 run single-threaded, as the paper's C++ did) on the same graph
and sources, one query per step.

Multi-GPU: queries are independent, so N processes (torchrun) each answer
their own batches (replicas, no collective on the data path); the timed
region is bracketed by barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (scale, edge_factor, k per step, k_tile)
    "rmat20-k64": (20, 16, 64, 64),
    "rmat20-k16": (20, 16, 16, 16),
    "rmat20-k8": (20, 16, 8, 8),
    "rmat22-k1": (22, 16, 1, 1),
    "rmat22-k64": (22, 16, 64, 64),
    "rmat22-approx": (22, 16, 256, 16),  # SpeedPPR, eps = 0.5, 256 sources (seed 3) in 16-column tiles
    "rmat22-index": (22, 16, 256, 16),   # SpeedPPR-Index (walks read from the index), same sources
}
APPROX_WORKLOADS = ("rmat22-approx", "rmat22-index")
ALPHA, LAMBDA, EPS = 0.2, 1e-8, 0.5
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy bandwidth is the roofline's peak)
METRIC = "SSPPR queries/s at l1<=1e-8 (HP, plain GPU method)"
METRIC_APPROX = "SSPPR queries/s, eps=0.5 relative error for pi>=1/n (SpeedPPR)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def sweep_bytes(n: int, m: int, kt: int) -> int:
    """Algorithmic DRAM bytes of one sweep launch over a tile of kt sources:
    in-CSR (row_ptr 4(n+1), col_idx 4m), per-node scales (8 + 4 per node) and
    the tile's z vector read once and written once (2 * 8 kt per node)."""
    return 4 * (n + 1) + 4 * m + 12 * n + 16 * n * kt


def fp32_pass_bytes(n: int, m: int, kt: int) -> int:
    """Algorithmic bytes of one (over-relaxed, in-place) FP32 correction pass:
    in-CSR (4(n+1) + 4m), degrees (4n), z_e gathered once, the row's own old
    z_e read once (the relaxation), z_e written once and r_f read once (16 n kt)."""
    return 4 * (n + 1) + 4 * m + 4 * n + 16 * n * kt


def fp32_pass_bytes_min(n: int, m: int, kt: int) -> int:
    """Lower bound of the same pass under an ideal cache: z_e read once in all
    (the own old row coming from the gathered copy), written once, r_f read
    once (12 n kt)."""
    return 4 * (n + 1) + 4 * m + 4 * n + 12 * n * kt


TRAFFIC_FILES = {
    # kernel family: (committed ncu summary, sources the capture was taken on)
    "sweep_kernel": ("sweep_kernel_traffic.json", ("sweep_kernel.cuh", "fixconv.cuh")),
    # the FP32 pass's launch (its L2 window, the order of its work list) is set in hp.cu
    "refine_pass_kernel": ("refine_pass_kernel_traffic.json",
                           ("refine_kernel.cuh", "f32_lanes.cuh", "sweep_kernel.cuh", "fixconv.cuh", "hp.cu")),
    "walk_kernel": ("walk_kernel_traffic.json", ("walk_kernel.cuh",)),
}


def kernel_source_sha(sources=("sweep_kernel.cuh",)) -> str:
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2101_03652_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kernel: str = "sweep_kernel"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    if kernel not in TRAFFIC_FILES:
        return None
    fname, sources = TRAFFIC_FILES[kernel]
    path = os.path.join(ROOT, "profiles", fname)
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("kernel_source_sha") != kernel_source_sha(sources):
            return None
        per = rec.get("per_workload", {})
        if workload in per:
            return float(per[workload]["dram_bytes_per_launch"])
        if workload in rec.get("workloads", []):
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(base: int, rank: int) -> int:
    """Each replica answers its own sources: the source seed is offset by rank
    (queries are independent, so ranks exchange no data)."""
    return base + 1000 * rank


def max_over_ranks(value: float, device) -> float:
    """The job's time is the slowest rank's (max all-reduce of one scalar)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


CALIB_SEED = 12  # sources of the autotuner's calibration batch (never the timed ones)


def make_inputs(workload: str, rank: int):
    import ppr_inputs as gen
    scale, ef, k, kt = WORKLOADS[workload]
    rp, ci = gen.rmat(scale, ef, seed=1)
    seed = 3 if workload in APPROX_WORKLOADS else 2
    src = gen.sources(len(rp) - 1, k, seed=replica_seed(seed, rank))
    return rp, ci, src, kt


def calibration_sources(n: int, k: int, rank: int):
    """The autotuner's calibration batch, drawn with its own seed so that the
    setting is chosen on other sources than the ones timed: k sources, or two
    batches' worth (2k) when k >= 64, where the tuner's k bucket is the same
    and two tiles per call average the batch-to-batch spread of pass counts."""
    import ppr_inputs as gen
    return gen.sources(n, 2 * k if k >= 64 else k, seed=replica_seed(CALIB_SEED, rank))


def hp_roofline(n: int, m: int, kt: int, fp32_ms: float, fp32_launches: int, sweep_ms: float, sweep_launches: int,
                workload: str):
    """Roofline entry of a high-precision workload's dominant kernel: the FP32
    correction pass when the query ran any, else the Q1.63 pass."""
    if fp32_launches > 0:
        avg = fp32_ms / fp32_launches
        per_launch, per_launch_min = fp32_pass_bytes(n, m, kt), fp32_pass_bytes_min(n, m, kt)
        name = f"refine_pass_kernel<{kt}, float>"
    else:
        avg = sweep_ms / max(sweep_launches, 1)
        per_launch = per_launch_min = sweep_bytes(n, m, kt)
        name = f"sweep_kernel<{kt}>"
    achieved = per_launch / (avg / 1e3) / 1e9
    traffic = ncu_traffic(workload, name.split("<")[0])
    peak, peak_kind = peaks()
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / peak, "nominal_peak": NOMINAL_HBM_GBS,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "traffic": traffic,
            "traffic_gbs": None if traffic is None else traffic / (avg / 1e3) / 1e9,
            "algorithmic_bytes_per_launch": per_launch, "algorithmic_bytes_lower_bound": per_launch_min,
            "frac_of_lower_bound": per_launch_min / (avg / 1e3) / 1e9 / peak, "avg_launch_ms": avg}


def hp_side_record(P, label: str, rp, ci, src, steps: int, warmup: int, rank: int, local: int, flush):
    """A second high-precision workload timed like the headline one (autotuned
    on a calibration batch outside the timed region, L2 flushed before every
    step, CUDA events on the stream): queries/s, passes and the dominant
    kernel's roofline entry."""
    import torch
    n, m, k = len(rp) - 1, len(ci), len(src)
    g = P.Graph(rp, ci)
    out = torch.empty((k, n), dtype=torch.float64, device="cuda")
    t_tune = time.perf_counter()
    kt, sw, _ = g.autotune(calibration_sources(n, k, rank), lam=LAMBDA, alpha=ALPHA)
    tuned = {"k_tile": int(kt), "switch_edges": int(sw), "seconds": time.perf_counter() - t_tune,
             "calibration_seed": CALIB_SEED}
    opts = dict(lam=LAMBDA, alpha=ALPHA, k_tile=0, switch_edges=-1)
    for _ in range(warmup):
        flush.zero_()
        g.query(src, P.PPR_HP, out_pi=out, **opts)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev, sweeps, launches = [], [], 0
    fp32_ms = sweep_ms = 0.0
    fp32_launches = sweep_launches = 0
    with ClockSampler(local) as clk:
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = g.query(src, P.PPR_HP, out_pi=out, **opts)
            e1.record(stream)
            ev.append((e0, e1))
            sweeps.append(st[0]["sweeps"])
            launches += st[0]["kernel_launches"]
            fp32_ms += st[0]["ms_fp32"]
            fp32_launches += sum(st[t]["fp32_passes"] for t in range(0, k, kt))
            sweep_ms += st[0]["ms_sweep"]
            sweep_launches += st[0]["sweep_launches"]
        torch.cuda.synchronize()
    assert max(x["final_l1_residual"] for x in st) <= LAMBDA
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    g.close()
    return {"workload": label, "n": n, "m": m, "sources_per_step": k, "steps": steps, "warmup": warmup,
            "k_tile": int(kt), "autotuned": tuned, "ms_per_step": total_ms / steps,
            "queries_per_s": k * steps / (total_ms / 1e3), "sweeps_per_tile": statistics.median(sweeps),
            "launches_per_step": launches / steps,
            "roofline": hp_roofline(n, m, int(kt), fp32_ms, fp32_launches, sweep_ms, sweep_launches, label),
            "clocks": clk.summary()}


def approx_roofline(st, steps: int, n_tiles: int, walk_ms: float, kt: int, indexed: bool, workload: str):
    """Roofline entry of a SpeedPPR step's dominant kernel: the walks (two 32 B
    sectors per move and per endpoint) or, with the index, the index reads
    (per walk one 4 B entry and the two 32 B sectors of its endpoint's count
    and estimate); st are the stats of the last step, walk_ms the kernel's
    event time summed over the timed steps."""
    walks = sum(x["walks"] for x in st)
    if indexed:
        per_launch = 68 * walks / n_tiles
        kernel_name = f"index_query_kernel<{kt}>"
    else:
        per_launch = 64 * (sum(x["walk_steps"] for x in st) + walks) / n_tiles
        kernel_name = f"walk_kernel<{kt}>"
    avg_ms = walk_ms / steps / n_tiles
    achieved = per_launch / (avg_ms / 1e3) / 1e9
    # DRAM bytes per launch from the committed ncu capture (None if the source changed since)
    traffic = ncu_traffic(workload, kernel_name.split("<")[0])
    peak, peak_kind = peaks()
    # the counts are already their minimum: the lower-bound fraction is the same
    return {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "traffic": traffic,
            "traffic_gbs": None if traffic is None else traffic / (avg_ms / 1e3) / 1e9,
            "algorithmic_bytes_per_launch": per_launch, "algorithmic_bytes_lower_bound": per_launch,
            "frac_of_lower_bound": achieved / peak, "avg_launch_ms": avg_ms}


def approx_side_record(P, rp, ci, steps: int, warmup: int, rank: int, flush):
    """SpeedPPR (eps = 0.5) on R-MAT-22 with the workload's 256 sources in
    16-column tiles, once drawing walks and once reading them from the
    SpeedPPR-Index (built outside the timed region): queries/s from CUDA
    events around each step, L2 flushed before every step, and the dominant
    kernel's roofline entry."""
    import torch
    import ppr_inputs as gen
    _, _, k, kt = WORKLOADS["rmat22-approx"]
    n = len(rp) - 1
    src = gen.sources(n, k, seed=replica_seed(3, rank))
    g = P.Graph(rp, ci)
    out = torch.empty((k, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rec = {"graph": f"R-MAT scale 22, edge factor 16", "n": n, "m": len(ci), "eps": EPS, "alpha": ALPHA,
           "sources_per_step": k, "k_tile": kt, "steps": steps, "warmup": warmup}
    for label, indexed in (("walks", False), ("index", True)):
        opts = dict(eps=EPS, alpha=ALPHA, k_tile=kt)
        t_build = None
        if indexed:
            t = time.perf_counter()
            g.build_index(0x1DE5, ALPHA)
            torch.cuda.synchronize()
            t_build = time.perf_counter() - t
            opts["flags"] = P.PPR_FLAG_INDEX
        for _ in range(warmup):
            flush.zero_()
            g.query(src, P.PPR_APPROX, out_pi=out, **opts)
        torch.cuda.synchronize()
        ms, walk_ms, st = [], 0.0, None
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = g.query(src, P.PPR_APPROX, out_pi=out, **opts)[1]
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            walk_ms += st[0]["ms_walk"]
        workload = "rmat22-index" if indexed else "rmat22-approx"
        rec[label] = {"workload": workload, "ms_per_step": sum(ms) / steps,
                      "queries_per_s": k * steps / (sum(ms) / 1e3),
                      "roofline": approx_roofline(st, steps, -(-k // kt), walk_ms, kt, indexed, workload)}
        if t_build is not None:
            rec[label]["index_build_s"] = t_build
    g.close()
    return rec


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    rp, ci, src, _ = make_inputs(args.workload, 0)
    g = O.Graph(rp, ci)
    approx = args.workload in APPROX_WORKLOADS
    times = []
    for i in range(args.warmup + args.steps):
        s = int(src[i % len(src)])
        t = time.perf_counter()
        if approx:
            O.speedppr(g, s, eps=EPS, seed=0x5EED, source_index=i % len(src))
        else:
            O.powerpush(g, s, ALPHA, LAMBDA)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps / total
    alg = "Algorithm 4 (walks drawn per query)" if approx else "Algorithm 3"
    sample = f"{args.steps} sources of the workload, one {alg} query per step, FP64, single thread"
    print(json.dumps({
        "impl": "reference", "metric": METRIC_APPROX if approx else METRIC, "value": value, "unit": "queries/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "graph": f"R-MAT scale {WORKLOADS[args.workload][0]}",
                   "n": len(rp) - 1, "m": len(ci), "alpha": ALPHA,
                   ("eps" if approx else "lambda"): (EPS if approx else LAMBDA), "queries_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    import paper_2101_03652_gb300 as P

    rp, ci, src, kt = make_inputs(args.workload, rank)
    n, m, k = len(rp) - 1, len(ci), len(src)
    g = P.Graph(rp, ci)
    stream = torch.cuda.current_stream()
    out = torch.empty((k, n), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    approx = args.workload in APPROX_WORKLOADS
    indexed = args.workload == "rmat22-index"
    opts = dict(lam=LAMBDA, alpha=ALPHA, k_tile=kt)
    if approx:
        opts = dict(eps=EPS, alpha=ALPHA, k_tile=kt)
    if indexed:
        # the index is built once per graph (preprocessing, outside the timed region)
        g.build_index(0x1DE5, ALPHA)
        opts["flags"] = P.PPR_FLAG_INDEX
    mode = P.PPR_APPROX if approx else P.PPR_HP
    tuned = None
    if not approx and not args.no_autotune:
        # the k-tile and the queue->pass switch come from the library's
        # autotuner, run outside the timed region on a calibration batch of
        # other sources
        t_tune = time.perf_counter()
        kt_t, sw_t, _ = g.autotune(calibration_sources(n, k, rank), lam=LAMBDA, alpha=ALPHA)
        tuned = {"k_tile": int(kt_t), "switch_edges": int(sw_t), "seconds": time.perf_counter() - t_tune,
                 "calibration_seed": CALIB_SEED}
        opts = dict(lam=LAMBDA, alpha=ALPHA, k_tile=0, switch_edges=-1)
        kt = int(kt_t)

    def step(out_buf):
        return g.query(src, mode, out_pi=out_buf, **opts)[1]

    for _ in range(args.warmup):
        flush.zero_()
        step(out)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sweep_ms, sweep_launches, launches, sweeps = 0.0, 0, 0, []
    fp32_ms, fp32_launches = 0.0, 0
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            st = step(out)
            ev[i][1].record(stream)
            sweep_ms += st[0]["ms_sweep"] if not approx else st[0]["ms_walk"]
            sweep_launches += st[0]["sweep_launches"]
            if not approx:
                fp32_ms += st[0]["ms_fp32"]
                fp32_launches += sum(st[t]["fp32_passes"] for t in range(0, k, kt))
            launches += st[0]["kernel_launches"]
            sweeps.append(st[0]["sweeps"])
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), "cuda")

    # end to end: host source ids in, host (pinned) PPR vectors out, copies inside the timed region
    host_out = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 5))
    flush.zero_()
    step(host_out)
    torch.cuda.synchronize()
    e2e_total = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        step(host_out)
        e2e_total += time.perf_counter() - t
    e2e_total = max_over_ranks(e2e_total, "cuda")

    # learned warm start (model trained on the workload's graph, held-out sources)
    warm = None
    if not args.skip_warm and args.workload == "rmat20-k64":
        warm = warm_start_comparison(P, g, n, k, kt, out, flush, rank)

    # the same method on the larger R-MAT graph of the roofline target, and on
    # the small graph where a pass takes microseconds (one GPU only)
    side = {}
    if ws == 1 and not args.skip_side and args.workload == "rmat20-k64":
        import ppr_inputs as gen
        rp22, ci22 = gen.rmat(22, 16, seed=1)
        src22 = gen.sources(len(rp22) - 1, 64, seed=2)
        side["rmat22_k64"] = hp_side_record(P, "rmat22-k64", rp22, ci22, src22, min(args.steps, 5), 2, rank, local,
                                            flush)
        side["speedppr_rmat22"] = approx_side_record(P, rp22, ci22, 2, 1, rank, flush)
        del rp22, ci22
        rpc, cic = gen.chung_lu(10_000, 100_000, 2.2, seed=1)
        srcc = gen.sources(len(rpc) - 1, 10, seed=1)
        side["small_graph"] = hp_side_record(P, "chung-lu-10k-k10", rpc, cic, srcc, max(args.steps, 20),
                                             max(args.warmup, 3), rank, local, flush)

    # sanity of the last answers (the parity tests check them against the oracle)
    pi0 = out[0].double()
    mass = float(pi0.sum().item())
    assert abs(1.0 - mass) <= (1e-4 if approx else LAMBDA * 1.01), f"mass {mass}"

    if rank != 0:
        g.close()
        if ws > 1:
            dist.destroy_process_group()
        return

    value = ws * k * args.steps / (total_ms / 1e3)
    n_tiles = -(-k // kt)  # one walk (or index) launch per tile of kt sources
    if approx:
        roofline = approx_roofline(st, args.steps, n_tiles, sweep_ms, kt, indexed, args.workload)
    else:
        # dominant kernel: the FP32 correction pass (the Q1.63 passes only certify)
        roofline = hp_roofline(n, m, kt, fp32_ms, fp32_launches, sweep_ms, sweep_launches, args.workload)
    cpu = None
    cpu_context = None
    if ws == 1 and not args.skip_cpu:
        import oracle as O
        og = O.Graph(rp, ci)
        t = time.perf_counter()
        done = 0
        while done < 1 or (time.perf_counter() - t < 10 and done < 3):
            if approx:
                O.speedppr(og, int(src[done]), eps=EPS, seed=0x5EED, source_index=done)
            else:
                O.powerpush(og, int(src[done]), ALPHA, LAMBDA)
            done += 1
        dt = time.perf_counter() - t
        alg = "Algorithm 4" if approx else "Algorithm 3"
        if indexed:
            alg = "Algorithm 4 with walks drawn per query (no index)"
        cpu = {"value": done / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} of the workload's sources, {alg} in FP64 on one host core"}
        if not approx:
            # context: the plain power iteration on all host cores (OpenMP)
            from oracle import context as CX
            cg = CX.ContextGraph(rp, ci)
            t = time.perf_counter()
            done_c = 0
            while done_c < 1 or (time.perf_counter() - t < 5 and done_c < 8):
                CX_pi, CX_it = cg.powitr(int(src[done_c]), ALPHA, LAMBDA)
                done_c += 1
            dt_c = time.perf_counter() - t
            cg.close()
            cpu_context = {"value": done_c / dt_c, "unit": "queries/s", "cores": CX.threads(),
                           "kind": "powitr_openmp",
                           "sample": f"{done_c} of the workload's sources, PowItr ({CX_it} iterations) in FP64 "
                                     f"on {CX.threads()} host threads; context, not a baseline"}
    rec = {
        "metric": METRIC_APPROX if approx else METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 push, u32 counts, f64 estimates" if approx else
                 "f32 correction passes, int64 (Q1.63 fixed point) certifying passes, f64 output",
        "data": "synthetic",
        "config": {"workload": args.workload, "graph": f"R-MAT scale {WORKLOADS[args.workload][0]}, "
                   f"edge factor {WORKLOADS[args.workload][1]}, a/b/c/d 0.57/0.19/0.19/0.05",
                   "n": n, "m": m, "alpha": ALPHA, ("eps" if approx else "lambda"): (EPS if approx else LAMBDA),
                   "sources_per_step": k, "k_tile": kt, "autotuned": tuned,
                   "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{ws}"},
        "sweeps_per_tile": statistics.median(sweeps),
        "e2e": {"value": ws * k * e2e_steps / e2e_total, "unit": "queries/s", "h2d_bytes_per_step": 4 * k,
                "d2h_bytes_per_step": 8 * k * n},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_context": cpu_context,
        "warm_start": warm,
        **side,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(rec))
    g.close()
    if ws > 1:
        dist.destroy_process_group()


def warm_start_comparison(P, g, n, k, kt, out, flush, rank, train_n=4096, held_n=1024, epochs=8, passes=8):
    """Train the learned warm start on train_n sources (seed 4) and compare
    queries/s and passes on held_n held-out sources (seed 5) with the plain
    zero start, same batches of k sources, L2 flushed before each batch."""
    import numpy as np
    import torch
    import ppr_inputs as gen
    train = gen.sources(n, train_n, seed=4)
    held = gen.sources(n, held_n, seed=replica_seed(5, rank))
    model = P.Model(g, seed=0x5EED, correction_passes=passes)
    t = time.perf_counter()
    losses = model.train(train, epochs=epochs, lr=2e-3, shuffle_seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    res = {}
    for name, ws in (("plain", None), ("warm", model)):
        ev = []
        sweeps = []
        edges = []
        g.query(held[:k], P.PPR_HP, out_pi=out, lam=LAMBDA, k_tile=kt, warm_start=ws)  # warm-up
        for b in range(0, held_n, k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = g.query(held[b:b + k], P.PPR_HP, out_pi=out, lam=LAMBDA, k_tile=kt, warm_start=ws)
            e1.record()
            ev.append((e0, e1))
            sweeps.append(st[0]["sweeps"])
            # edges touched per query: out-edges scattered by its queue phase
            # plus in-edges gathered by its passes (m per pass)
            edges.extend(x["edges_pushed"] + x["edges_swept"] for x in st)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        res[name] = {"queries_per_s": held_n / (ms / 1e3), "passes_mean": float(np.mean(sweeps)),
                     "edges_touched_per_query": float(np.mean(edges))}
    model.close()
    return {"metric": "queries/s at l1<=1e-8 on held-out sources", "train_sources": train_n,
            "held_out_sources": held_n, "epochs": epochs, "correction_passes": passes,
            "train_seconds_incl_labels": train_s, "final_train_l1": float(losses[-1]),
            "plain": res["plain"], "warm": res["warm"],
            "speedup": res["warm"]["queries_per_s"] / res["plain"]["queries_per_s"],
            "edges_touched_ratio": res["warm"]["edges_touched_per_query"] / res["plain"]["edges_touched_per_query"]}


def admit_batch(k: int, free_bytes: int, held_bytes: int, state_bytes) -> int:
    """Admission of a serving batch: the largest k (halved until it fits)
    whose query workspace, state_bytes(k), fits in free device memory plus the
    workspace the graph already holds (the library reuses it); 0 when not even
    one source fits, and the batch is refused."""
    while k >= 1:
        if state_bytes(k) <= free_bytes + held_bytes:
            return k
        k //= 2
    return 0


def run_serve(args):
    """Serving: requests (one source each) arrive as a Poisson stream; a single
    GPU server takes up to 32 queued requests per batch, admitted against free
    device memory (ppr_query_state_bytes), and answers them with the plain
    zero start or the learned warm start.  Latency = completion - arrival;
    the clock is virtual and advances by each batch's measured GPU time."""
    import collections
    import numpy as np
    import torch
    import ppr_inputs as gen
    import __graft_entry__
    __graft_entry__.build()
    import paper_2101_03652_gb300 as P
    torch.cuda.set_device(0)
    t = time.perf_counter()
    rp, ci = gen.rmat(args.serve_scale, args.serve_ef, seed=1)
    gen_s = time.perf_counter() - t
    n, m = len(rp) - 1, len(ci)
    t = time.perf_counter()
    g = P.Graph(rp, ci)
    load_s = time.perf_counter() - t
    del rp, ci
    kmax = 32
    out = torch.empty((kmax, n), dtype=torch.float64, device="cuda")
    free0 = torch.cuda.mem_get_info()[0]

    def run_batch(srcs, model):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st = g.query(srcs, P.PPR_HP, out_pi=out[:len(srcs)], lam=LAMBDA, warm_start=model)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, st[0]["sweeps"]

    def admit(k):
        return admit_batch(k, torch.cuda.mem_get_info()[0], g.workspace_bytes(), g.state_bytes)

    def peak(model, seed, batches=3):
        srcs = gen.sources(n, kmax * batches, seed=seed)
        run_batch(srcs[:kmax], model)  # warm-up
        tot, sw = 0.0, []
        for b in range(batches):
            d, s = run_batch(srcs[b * kmax:(b + 1) * kmax], model)
            tot += d
            sw.append(s)
        return kmax * batches / tot, float(np.mean(sw))

    plain_qps, plain_passes = peak(None, seed=6)
    t = time.perf_counter()
    model = P.Model(g, seed=0x5EED, correction_passes=8)
    train = gen.sources(n, args.serve_train, seed=7)
    model.train(train, epochs=1, lr=2e-3, shuffle_seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    warm_qps, warm_passes = peak(model, seed=6)

    def simulate(rate, model, seed):
        rng = np.random.default_rng(seed)
        nreq = args.serve_requests
        arrivals = np.cumsum(rng.exponential(1.0 / rate, nreq))
        srcs = gen.sources(n, nreq, seed=seed)
        queue = collections.deque()
        lat = np.zeros(nreq)
        t_free, i, done, refused = 0.0, 0, 0, 0
        while done < nreq:
            while i < nreq and arrivals[i] <= t_free:
                queue.append(i)
                i += 1
            if not queue:
                t_free = arrivals[i]
                continue
            k = admit(min(kmax, len(queue)))
            if k == 0:
                # not even one source fits: the queued requests are refused
                while queue:
                    lat[queue.popleft()] = np.nan
                    refused += 1
                    done += 1
                continue
            batch = [queue.popleft() for _ in range(k)]
            d, _ = run_batch(srcs[batch], model)
            t_free += d
            for j in batch:
                lat[j] = t_free - arrivals[j]
            done += k
        span = t_free - arrivals[0]
        ok = lat[~np.isnan(lat)]
        return {"p50_ms": 1e3 * float(np.percentile(ok, 50)) if len(ok) else None,
                "p99_ms": 1e3 * float(np.percentile(ok, 99)) if len(ok) else None,
                "queries_per_s": len(ok) / span if span > 0 else None, "refused": refused}

    load = []
    for frac in (0.5, 0.8):
        rate = frac * plain_qps
        load.append({"rate_frac_of_plain_peak": frac, "arrival_qps": rate,
                     "plain": simulate(rate, None, seed=8), "warm": simulate(rate, model, seed=8)})
    print(json.dumps({
        "metric": "serving: p50/p99 latency and queries/s at l1<=1e-8, learned warm start vs plain batched",
        "workload": "rmat%d-serve" % args.serve_scale, "data": "synthetic",
        "graph": {"scale": args.serve_scale, "edge_factor": args.serve_ef, "n": n, "m": m},
        "batch": kmax, "requests": args.serve_requests, "train_sources": args.serve_train,
        "setup_s": {"generate": gen_s, "load": load_s, "train_incl_labels": train_s},
        "free_hbm_gb_after_load": free0 / 1e9,
        "peak": {"plain": {"queries_per_s": plain_qps, "passes": plain_passes},
                 "warm": {"queries_per_s": warm_qps, "passes": warm_passes}},
        "load": load}))
    model.close()
    g.close()


def run_eps_sweep(args):
    """Accuracy study of SpeedPPR over eps (the methodology of Sec. 8's
    accuracy experiments on synthetic inputs): for each eps, queries/s with
    walks and with the index, the mean l1 error against certified
    lambda = 1e-8 answers of the same sources, and the share of entries with
    pi >= 1/n whose relative error exceeds eps."""
    import numpy as np
    import torch
    import ppr_inputs as gen
    import __graft_entry__
    __graft_entry__.build()
    import paper_2101_03652_gb300 as P
    rp, ci = gen.rmat(args.sweep_scale, 16, seed=1)
    n, m = len(rp) - 1, len(ci)
    src = gen.sources(n, 16, seed=3)
    g = P.Graph(rp, ci)
    exact, st_hp = g.query(src, P.PPR_HP, lam=LAMBDA, alpha=ALPHA)
    assert max(x["final_l1_residual"] for x in st_hp) <= LAMBDA
    exact = exact.cpu().numpy()
    g.build_index(0x1DE5, ALPHA)
    out = torch.empty((len(src), n), dtype=torch.float64, device="cuda")
    rows = []
    for eps in (0.1, 0.2, 0.3, 0.4, 0.5):
        rec = {"eps": eps}
        for name, flags in (("walks", 0), ("index", P.PPR_FLAG_INDEX)):
            g.query(src, P.PPR_APPROX, out_pi=out, eps=eps, alpha=ALPHA, flags=flags)  # warm-up
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, st = g.query(src, P.PPR_APPROX, out_pi=out, eps=eps, alpha=ALPHA, flags=flags)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            est = out.cpu().numpy()
            big = exact >= 1.0 / n
            rel = np.abs(est - exact)[big] / exact[big]
            rec[name] = {"queries_per_s": len(src) / dt, "walks_per_source": float(np.mean([x["walks"] for x in st])),
                         "mean_l1_error": float(np.abs(est - exact).sum(axis=1).mean()),
                         "max_rel_error_pi_ge_1_over_n": float(rel.max()),
                         "share_rel_error_above_eps": float((rel > eps).mean())}
        rows.append(rec)
    g.close()
    print(json.dumps({"metric": "SpeedPPR accuracy over eps", "unit": "see rows", "data": "synthetic",
                      "config": {"workload": "eps-sweep", "graph": f"R-MAT scale {args.sweep_scale}, edge factor 16",
                                 "n": n, "m": m, "alpha": ALPHA, "sources": len(src), "mu": "1/n",
                                 "reference": "HP answers certified at lambda = 1e-8"},
                      "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat20-k64", choices=sorted(WORKLOADS) + ["serve", "eps-sweep"])
    ap.add_argument("--sweep-scale", type=int, default=20, help="R-MAT scale of the eps-sweep study")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the oracle CPU baseline")
    ap.add_argument("--skip-warm", action="store_true", help="omit the learned warm-start comparison")
    ap.add_argument("--no-autotune", action="store_true", help="use the workload's fixed k-tile and the default switch")
    ap.add_argument("--skip-side", action="store_true",
                    help="omit the R-MAT-22 and small-graph records of the default run")
    ap.add_argument("--serve-scale", type=int, default=25, help="R-MAT scale of the serving workload")
    ap.add_argument("--serve-ef", type=int, default=32)
    ap.add_argument("--serve-train", type=int, default=2048)
    ap.add_argument("--serve-requests", type=int, default=512)
    args = ap.parse_args()
    if args.impl == "reference" and args.workload in ("serve", "eps-sweep"):
        if dist_env()[1] == 0:
            print(json.dumps({"impl": "reference", "workload": args.workload,
                              "unavailable": "a latency / accuracy study of the GPU path; the oracle is timed "
                                             "on the R-MAT query workloads"}))
        return
    if args.workload == "serve":
        run_serve(args)
    elif args.workload == "eps-sweep":
        run_eps_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
