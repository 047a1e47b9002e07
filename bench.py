#!/usr/bin/env python
"""Benchmark of the batched FP64 inclusion-based CCD root finder on GB300.

Default workload (one "step"): 64 simulation instances with log-uniform
query counts summing to 20,000,000 queries (VF:EE 1:1, seed 3, per-instance
scale 10^U(-2,2) and eps, delta = 1e-6, m_I = 1e6, ms = 0), solved by one
ccd_multi_batch call (per-segment eps from bounds, then the four solver
stages) replayed from a CUDA graph, with launch shapes picked by the
project's autotuner.  Inputs are resident in HBM when the timed region
starts; they total 3.84 GB, far more than the 129 MB L2, so no flush is
needed between steps.  The line also carries the plain form (one call per
instance-kind), the 1,000,000-query simulation-shaped workload's rate, the
roofline of the dominant kernel, an end-to-end rate through host buffers and
the CPU oracle on a sample.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (a bounded sample of the same workload per step).
Other modes: ``--workload simulation-mixed | served | line-search |
active-set``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CCD queries/sec FP64, 0 false negatives; p50/p99 batch latency; % FP64 peak"
# The paper's own average times per query (its "Ours" rows, Sec. 5 results
# table) on the CPU it names: context only, a different dataset and machine.
PAPER_CONTEXT = {
    "cpu": "AMD EPYC 7452 at 2.35 GHz, C++ with AVX2, per-query averages (one core implied)",
    "simulation_us_per_query": {"VF": 0.74, "EE": 0.78},
    "handcrafted_us_per_query": {"VF": 1532.54, "EE": 3029.83},
    "note": "the paper's datasets are not available here; the synthetic workloads differ",
}
# FP64 pipe instructions (add, sub, mul or fused multiply-add, one each) of
# the fixed F expression.  A t-quantity evaluation (one t value: 12 positions
# fma(dx, t, x0), then VF 9 / EE 6 differences) is shared by a run of boxes
# with equal t_L.  Per t and coordinate a box has two partials (VF 2 fma
# q - u e1; EE 2 x (fma + difference) p1 - (p3 + v d2)) and four corners
# (fma - v e2 / + u d1); the min and max of the four are the two extreme
# corners, one fma each, so the solvers evaluate 2 of them.  Plus 3 for
# w(B).  (FULL_BOX_OPS: all four corners, as the definition reads.)
T_OPS = {0: 12 + 9, 1: 12 + 6}
BOX_OPS = {0: 2 * 3 * 4 + 3, 1: 2 * 3 * 6 + 3}
FULL_BOX_OPS = {0: 2 * 3 * 6 + 3, 1: 2 * 3 * 8 + 3}
# deep solver with shared partials: one partial per (t value, parameter),
# VF a(t,u) = fma(-u, e1, q) (3), EE c(t,v) = p1 - fma(v, d2, p3) (6); a box
# then needs only its 4 extreme corners (12) and w(B) (3)
A_OPS = {0: 3, 1: 6}
SHARED_BOX_OPS = 12 + 3
# the same check evaluated on its own as the definition reads (no sharing,
# all 8 corners): 2 t-quantities + box
OPS_PER_CHECK = {k: 2 * T_OPS[k] + FULL_BOX_OPS[k] for k in (0, 1)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--n", type=int, default=None,
                    help="simulation-mixed (default 1,000,000) / degenerate-heavy (100,000) / "
                         "line-search queries")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--cpu-sample", type=int, default=400_000)
    ap.add_argument("--ref-sample", type=int, default=40_000)
    ap.add_argument("--max-itr", type=int, default=10**6,
                    help="check limit m_I (smaller values for profiling cases only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pages", type=int, default=None,
                    help="simulation-mixed: frontier pages of the deep tier (smaller workspace, "
                         "e.g. for profiling)")
    ap.add_argument("--workload", default="multi-instance",
                    choices=["simulation-mixed", "degenerate-heavy", "multi-instance", "served",
                             "line-search", "active-set"])
    ap.add_argument("--scale", type=float, default=1.0,
                    help="multi-instance/served: fraction of the full query count")
    ap.add_argument("--duration", type=float, default=30.0, help="served: seconds of arrivals")
    ap.add_argument("--req-scale", type=float, default=1.0,
                    help="served: request sizes are log-uniform in [100, 500k] times this")
    ap.add_argument("--retune", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="multi-instance: the default launch shapes instead of the autotuner's")
    ap.add_argument("--ms-list", default="0,1e-4",
                    help="degenerate-heavy: the minimum separations each step runs")
    ap.add_argument("--tuning", default=None,
                    help="multi-instance: launch shapes as JSON (deep_threads, deep_slots, "
                         "small_blocks_per_sm, small_cap, pool_cap) instead of the autotuner's")
    ap.add_argument("--no-extras", action="store_true",
                    help="multi-instance: skip the plain-form and simulation-mixed comparisons "
                         "that follow the timed region (small profiling cases)")
    ap.add_argument("--nx", type=int, default=512, help="active-set: vertices per sheet side")
    ap.add_argument("--compare-printed-cap", action="store_true",
                    help="line-search: also time d = max(p d_i, delta) (about a minute a step)")
    args = ap.parse_args()
    heavy = args.workload == "degenerate-heavy"
    if args.n is None:
        args.n = 100_000 if heavy else 1_000_000
    if args.seed is None:
        args.seed = 2 if heavy else 1
    return args


def dist_env():
    from paper_2009_13349_gb300 import parallel
    return parallel.env()


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_rank{self.index}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            if self.path:
                try:
                    os.unlink(self.path)
                except OSError:
                    pass
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def recorded_traffic(kernel: str):
    """The committed ncu record of ``kernel``'s DRAM traffic
    (profiles/traffic.json, from a small-case capture of the current
    source), or None if there is none or the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2009_13349_gb300", "csrc", "ccd.cu")
    try:
        rec = json.load(open(path)).get(kernel)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except (OSError, ValueError, AttributeError):
        return None
    if not rec or rec.get("sha256_prefix") != sha:
        return None
    return rec


def stage_traffic(kernel: str, c: dict, stage: int):
    """DRAM bytes per step of a solver stage: the recorded bytes per
    evaluated box of each kind (small-case capture) times this run's boxes,
    from the kernels' counters.  None without a record of the current
    source."""
    rec = recorded_traffic(kernel)
    if not rec or stage not in (1, 2, 3):
        return None
    ev, ee = {1: ("evals_pool", "evals_pool_ee"), 2: ("evals_small", "evals_small_ee"),
              3: ("evals_deep", "evals_deep_ee")}[stage]
    bpb = rec["bytes_per_box"]
    return bpb["0"] * (c[ev] - c[ee]) + bpb["1"] * c[ee]


STAGES = ["root_kernel", "pool_kernel (pooled small frontiers)",
          "solve_kernel<32> (one-warp frontier)", "solve_kernel<128> (deep)"]


def stage_ops(c: dict, stage: int, n_by_kind: dict) -> tuple[float, float]:
    """(executed FP64 instructions, the same work evaluated check by check as
    the definition reads) of one solver stage, from the kernels' own
    counters; the *_ee counters split mixed-kind batches exactly."""
    if stage == 0:
        ops = sum(n * OPS_PER_CHECK[k] for k, n in n_by_kind.items())
        return ops, ops
    if stage == 1:
        # boxes from shared partials: SHARED_BOX_OPS each plus the partials;
        # the rest (iterations with more distinct partials than the table
        # holds) evaluate their corners directly
        ee, tee = c["evals_pool_ee"], c["tq_pool_ee"]
        sh, shee, aee = c["evals_pool_shared"], c["evals_pool_shared_ee"], c["a_tasks_pool_ee"]
        ops = ((c["evals_pool"] - ee - (sh - shee)) * BOX_OPS[0] + (ee - shee) * BOX_OPS[1]
               + sh * SHARED_BOX_OPS + (c["a_tasks_pool"] - aee) * A_OPS[0] + aee * A_OPS[1]
               + (c["tq_pool"] - tee) * T_OPS[0] + tee * T_OPS[1])
        return ops, c["checks_pool"] * max(OPS_PER_CHECK.values())
    if stage == 2:
        tee, eee = c["tq_small_ee"], c["evals_small_ee"]
        ops = ((c["tq_small"] - tee) * T_OPS[0] + tee * T_OPS[1]
               + (c["evals_small"] - eee) * BOX_OPS[0] + eee * BOX_OPS[1])
        return ops, c["checks_small"] * max(OPS_PER_CHECK.values())
    tee, aee = c["tq_deep_ee"], c["a_tasks_deep_ee"]
    shared, shee, evee = c["evals_shared_deep"], c["evals_shared_deep_ee"], c["evals_deep_ee"]
    ops = ((c["tq_deep"] - tee) * T_OPS[0] + tee * T_OPS[1] + (c["a_tasks_deep"] - aee) * A_OPS[0]
           + aee * A_OPS[1] + shared * SHARED_BOX_OPS
           + (c["evals_deep"] - evee - (shared - shee)) * BOX_OPS[0] + (evee - shee) * BOX_OPS[1])
    return ops, c["checks_deep"] * max(OPS_PER_CHECK.values())


def fp64_peak(ccd, sms):
    """FP64 pipe rate measured in this run (fma.rn.f64 chains on every SM)."""
    peak = 0.0
    for _ in range(3):
        ms, ops = ccd.fp64_peak_probe(sms * 8, 8192)
        peak = max(peak, ops / (ms * 1e-3))
    return peak


def make_workload(n, seed):
    from paper_2009_13349_gb300 import workloads as W
    return W.simulation_mixed(n=n, seed=seed)


def make_jobs(args, seed):
    """The calls of one step: (batch, ms) pairs.  simulation-mixed: both kinds
    at ms = 0; degenerate-heavy: both kinds at ms = 0 and at ms = 1e-4."""
    from paper_2009_13349_gb300 import workloads as W
    if args.workload == "degenerate-heavy":
        wl = W.degenerate_heavy(n=args.n, seed=seed)
        ms_list = [float(x) for x in args.ms_list.split(",")]
        return wl, [(b, ms) for ms in ms_list for b in wl.batches]
    wl = make_workload(args.n, seed)
    return wl, [(b, 0.0) for b in wl.batches]


def job_label(b, ms):
    return ("VF" if b.kind == 0 else "EE") + ("" if ms == 0 else f" ms={ms:g}")


def cpu_baseline(batches, sample: int, seed: int = 123, max_itr: int = 10**6, ms=None):
    """Oracle on a bounded random sample of the batches (sizes proportional),
    each batch with its own scene eps (and minimum separation ms[i]), all
    host cores."""
    import oracle
    rng = np.random.default_rng(seed)
    cores = os.cpu_count() or 1
    total = sum(b.n for b in batches)
    ms = ms or [0.0] * len(batches)
    picks = []
    for b, m in zip(batches, ms):
        k = min(b.n, max(1, int(round(sample * b.n / total))))
        picks.append((b, m, np.sort(rng.choice(b.n, k, replace=False))))
    total_q, total_s = 0, 0.0
    for b, m, idx in picks:
        err = oracle.err_from_bounds(b.kind, b.verts, ms_nonzero=m > 0)   # whole-instance eps
        t0 = time.perf_counter()
        oracle.ccd_batch(b.kind, b.verts[idx], err, ms=m, delta=1e-6, max_itr=max_itr,
                         nthreads=cores)
        total_s += time.perf_counter() - t0
        total_q += idx.size
    return total_q / total_s, cores, total_s, total_q


def workload_config(args):
    """The simulation-mixed (or degenerate-heavy) workload's config keys."""
    if args.workload == "degenerate-heavy":
        return {"workload": f"degenerate-heavy {args.n} queries per GPU (VF:EE 1:1; coplanar, "
                            f"collinear, parallel-edge, vertex-on-vertex and grazing-tangent "
                            f"motions on a 2^-20 grid), seed {args.seed}, each step at ms = "
                            + " and at ms = ".join(args.ms_list.split(",")),
                "delta": 1e-6, "max_itr": args.max_itr,
                "ms": [float(x) for x in args.ms_list.split(",")]}
    return {"workload": f"simulation-mixed {args.n} queries per GPU (VF:EE 1:1), seed {args.seed}",
            "delta": 1e-6, "max_itr": args.max_itr, "ms": 0.0}


def multi_config(n_total, scale, max_itr=10**6):
    """The multi-instance workload's config keys, the same for both arms."""
    return {"workload": f"multi-instance: 64 simulation instances, {n_total} queries per GPU "
                        f"(log-uniform 1k-2M each, VF:EE 1:1, per-instance scale 10^U(-2,2) "
                        f"and eps), seed 3" + ("" if scale == 1.0 else f", scale {scale}"),
            "delta": 1e-6, "max_itr": max_itr, "ms": 0.0}


def multi_workload(scale, rank=0):
    from paper_2009_13349_gb300 import parallel
    from paper_2009_13349_gb300 import workloads as W
    return W.multi_instance(count=64, total=int(20_000_000 * scale),
                            seed=parallel.rank_seed(3, rank))


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores, every step a
    bounded random sample of the multi-instance workload (each instance with
    its own eps)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = multi_workload(args.scale)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    errs = [oracle.err_from_bounds(b.kind, b.verts) for b in wl.batches]
    sizes = np.array([b.n for b in wl.batches], dtype=np.float64)

    def step():
        # args.ref_sample queries drawn over the whole workload, then solved
        # instance by instance
        owner = rng.choice(len(wl.batches), args.ref_sample, p=sizes / sizes.sum())
        q, s = 0, 0.0
        for j in np.unique(owner):
            b = wl.batches[j]
            k = int(np.sum(owner == j))
            idx = rng.choice(b.n, min(k, b.n), replace=False)
            t0 = time.perf_counter()
            oracle.ccd_batch(b.kind, b.verts[idx], errs[j], delta=1e-6, max_itr=10**6,
                             nthreads=cores)
            s += time.perf_counter() - t0
            q += idx.size
        return q, s

    for _ in range(args.warmup):
        step()
    qs, ss, lat = 0, 0.0, []
    for _ in range(args.steps):
        q, s = step()
        qs += q
        ss += s
        lat.append(s * 1e3)
    value = qs / ss
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ss / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**multi_config(wl.n, args.scale), "sample_per_step": args.ref_sample},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.ref_sample} random queries of the workload per step"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
    }
    print(json.dumps(out))


def measure_simulation_mixed(args, dev, steps, warmup, seed, stage_detail=True):
    """The 1,000,000-query simulation-shaped workload: scene eps, then
    ccd_vf_batch and ccd_ee_batch, each kind on its own stream.  Returns the
    timing, stage and roofline figures and the buffers for the caller."""
    import torch
    from paper_2009_13349_gb300 import ccd
    wl, jobs = make_jobs(args, seed)
    batches = [b for b, _ in jobs]
    verts = [ccd.to_soa(b.verts, dev) for b in batches]
    ws = [ccd.workspace(b.n, args.max_itr, dev, pages=args.pages) for b in batches]
    res = [ccd.Result(torch.empty(b.n, dtype=torch.uint8, device=dev),
                      torch.empty(b.n, dtype=torch.float64, device=dev),
                      torch.empty(b.n, dtype=torch.float64, device=dev),
                      torch.empty(b.n, dtype=torch.int64, device=dev)) for b in batches]
    stream = torch.cuda.current_stream(dev)
    # the VF and EE batches of a step run on their own streams, so that each
    # fills the SMs the other's stages leave idle at their ends
    side = [torch.cuda.Stream(dev) for _ in batches]

    def step(stage_sets=None):
        for j, (b, ms) in enumerate(jobs):
            side[j].wait_stream(stream)
            with torch.cuda.stream(side[j]):
                if stage_sets is not None:
                    ccd.set_stage_events(stage_sets[j])
                err = ccd.err_from_bounds(b.kind, verts[j], ms_nonzero=ms > 0, stream=side[j])
                ccd.batch(b.kind, verts[j], err, ms=ms, delta=1e-6, max_itr=args.max_itr,
                          ws=ws[j], out=res[j], stream=side[j])
        ccd.set_stage_events(None)
        for sj in side:
            stream.wait_stream(sj)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)

    def new_event():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    stage_sets = [[[new_event() for _ in range(5)] for _ in batches] for _ in range(steps)]
    marks = [new_event() for _ in range(steps + 1)]
    torch.cuda.synchronize(dev)
    return {"wl": wl, "jobs": jobs, "batches": batches, "verts": verts, "ws": ws, "res": res,
            "side": side, "stream": stream, "step": step, "stage_sets": stage_sets,
            "marks": marks}


def simulation_mixed_figures(args, S, steps, peak):
    """Stage times (per kind, and per stage the union of the kinds'
    intervals), counters, truth checks and the roofline of a timed run."""
    from paper_2009_13349_gb300 import ccd
    batches, marks, stage_sets = S["batches"], S["marks"], S["stage_sets"]
    stage_ms = np.zeros((len(batches), 4))
    span_ms = np.zeros(4)
    for s in range(steps):
        for k in range(4):
            for j in range(len(batches)):
                ev = stage_sets[s][j]
                stage_ms[j, k] += ev[k].elapsed_time(ev[k + 1]) / steps
            t0 = min(marks[s].elapsed_time(stage_sets[s][j][k]) for j in range(len(batches)))
            t1 = max(marks[s].elapsed_time(stage_sets[s][j][k + 1]) for j in range(len(batches)))
            span_ms[k] += (t1 - t0) / steps
    counters = [ccd.workspace_counters(w) for w in S["ws"]]
    fn, toi_bad, checks = 0, 0, []
    for j, b in enumerate(batches):
        col = S["res"][j].collides.cpu().numpy()
        toi = S["res"][j].toi.cpu().numpy()
        hit = b.truth == 1
        fn += int(np.sum(col[hit] == 0))
        toi_bad += int(np.sum(toi[hit] > b.t_star[hit]))
        checks.append(S["res"][j].checks.cpu().numpy())
    checks = np.concatenate(checks)
    top = int(np.argmax(stage_ms.sum(axis=0)))
    ops, naive = 0.0, 0.0
    for j, b in enumerate(batches):
        o, nv = stage_ops(counters[j], top, {b.kind: b.n})
        ops += o
        naive += nv
    achieved = ops / (span_ms[top] * 1e-3)
    return {"stage_ms": stage_ms, "span_ms": span_ms, "counters": counters, "fn": fn,
            "toi_bad": toi_bad, "checks": checks, "top": top, "achieved": achieved,
            "naive": naive / (span_ms[top] * 1e-3), "peak": peak}


def run_native(args):
    """--workload simulation-mixed: the 1,000,000-query simulation-shaped
    workload on its own (its line of the earlier benchmark)."""
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2009_13349_gb300 import ccd, parallel
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp64_peak(ccd, sms)
    S = measure_simulation_mixed(args, dev, args.steps, args.warmup,
                                 parallel.rank_seed(args.seed, rank))
    batches, jobs = S["batches"], S["jobs"]
    in_bytes = 192 * sum(b.n for b in batches)
    # inputs that fit in L2 are evicted before every step by writing a
    # buffer twice its size; each step is then timed on its own
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if in_bytes <= 129e6 else None
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    clocks.start()
    for s in range(args.steps):
        if flush is not None:
            flush.fill_(s & 0xFF)
        S["marks"][s].record(S["stream"])
        S["step"](S["stage_sets"][s])
        ends[s].record(S["stream"])
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    marks = S["marks"]
    step_ms = [marks[s].elapsed_time(ends[s]) for s in range(args.steps)]
    total_ms = parallel.max_over_ranks(float(sum(step_ms)), device=dev)
    F = simulation_mixed_figures(args, S, args.steps, peak)
    top = F["top"]
    traffic = None
    if top == 3:
        traffic = sum(stage_traffic("solve_kernel<128> " + args.workload, c, 3) or 0
                      for c in F["counters"]) or None
    total_queries = sum(b.n for b in batches) * world
    out = {
        "metric": METRIC, "value": parallel.job_throughput(sum(b.n for b in batches), world,
                                                           total_ms / args.steps),
        "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {**workload_config(args),
                   "l2": (f"inputs {in_bytes / 1e6:.0f} MB per step "
                          + ("> 129 MB L2; no flush" if flush is None
                             else "< 129 MB L2: a 256 MB buffer written before each step, "
                                  "steps timed one by one")),
                   "streams": "the VF and EE batches of a step on two CUDA streams",
                   "parallelism": f"{world} GPU(s), queries sharded, no collective"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "roofline": {"bound": "alu", "kernel": STAGES[top], "achieved": F["achieved"] / 1e9,
                     "peak": peak / 1e9, "unit": "G FP64 ops/s", "frac": F["achieved"] / peak,
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per step of the stage (all its launches)",
                     "peak_source": "FP64 fma.rn.f64 issue rate measured in this run "
                                    "(one FP64 pipe op = one add, mul or fma)",
                     "work": "executed FP64 add/sub/mul/fma instructions from the kernel's counters",
                     "duration": "per step, the union of the VF and EE launches' intervals "
                                 "(two streams)",
                     "naive_equivalent_gops": F["naive"] / 1e9},
        "stage_ms_per_step": {job_label(b, ms): {STAGES[k]: float(F["stage_ms"][j, k])
                                                 for k in range(4)}
                              for j, (b, ms) in enumerate(jobs)},
        "stage_union_ms_per_step": {STAGES[k]: float(F["span_ms"][k]) for k in range(4)},
        "counters": {job_label(b, ms): F["counters"][j] for j, (b, ms) in enumerate(jobs)},
        "checks": {"mean": float(F["checks"].mean()),
                   "p99": float(np.percentile(F["checks"], 99)), "max": int(F["checks"].max()),
                   "early_termination_pct": float(100.0 * np.mean(F["checks"] >= args.max_itr))},
        "false_negatives": F["fn"], "toi_after_truth": F["toi_bad"],
        "gpu_launches": args.steps * len(batches) * 8,
        "paper_context": PAPER_CONTEXT,
        "clocks": clk,
    }
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(b.verts.T)).pin_memory() for b in batches]
        out_host = [(torch.empty(b.n, dtype=torch.uint8).pin_memory(),
                     torch.empty(b.n, dtype=torch.float64).pin_memory(),
                     torch.empty(b.n, dtype=torch.float64).pin_memory()) for b in batches]
        dres = [ccd.Result(r.collides, r.toi, r.out_tol, None) for r in S["res"]]

        def e2e_step():
            for j, (b, ms) in enumerate(jobs):
                with torch.cuda.stream(S["side"][j]):
                    S["verts"][j].copy_(host[j], non_blocking=True)
                    err = ccd.err_from_bounds(b.kind, S["verts"][j], ms_nonzero=ms > 0,
                                              stream=S["side"][j])
                    ccd.batch(b.kind, S["verts"][j], err, ms=ms, delta=1e-6,
                              max_itr=args.max_itr, ws=S["ws"][j], out=dres[j],
                              stream=S["side"][j])
                    out_host[j][0].copy_(dres[j].collides, non_blocking=True)
                    out_host[j][1].copy_(dres[j].toi, non_blocking=True)
                    out_host[j][2].copy_(dres[j].out_tol, non_blocking=True)
            torch.cuda.synchronize(dev)

        e2e_step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        el = (time.perf_counter() - t0) / args.steps
        out["e2e"] = {"value": total_queries / el, "unit": "queries/s",
                      "h2d_bytes_per_step": sum(h.numel() * 8 for h in host),
                      "d2h_bytes_per_step": sum(b.n * (1 + 8 + 8) for b in batches),
                      "ms_per_step": el * 1e3}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        # degenerate-heavy queries average about 0.1 core-second in the oracle
        sample = args.cpu_sample if args.workload != "degenerate-heavy" else min(args.cpu_sample,
                                                                                 3000)
        qps, cores, secs, nq = cpu_baseline(batches, sample, max_itr=args.max_itr,
                                            ms=[ms for _, ms in jobs])
        out["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"{nq} random queries of the workload ({secs:.1f} s)"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def _gpu_name(torch, dev):
    return torch.cuda.get_device_properties(dev).name


# our kernel launches per ccd_multi_batch call with its per-segment eps:
# 3 (eps from bounds) + validation, level 0, pooled VF, pooled EE, one-warp,
# order-by-level, deep
MULTI_LAUNCHES = 10


def run_multi_instance(args):
    """The headline: 64 simulation instances (log-uniform sizes, 20M queries,
    VF:EE 1:1, per-instance scale and eps) in one ccd_multi_batch call
    replayed from a CUDA graph, autotuned launch shapes.  Extra keys: the
    plain form (one call per instance-kind), the simulation-shaped 1M
    workload, the roofline, e2e through host buffers, the oracle on a
    sample."""
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2009_13349_gb300 import autotune, ccd, parallel
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = fp64_peak(ccd, sms)

    wl = multi_workload(args.scale, rank)
    counts = [b.n for b in wl.batches]
    kinds = [b.kind for b in wl.batches]
    n = sum(counts)
    verts = torch.empty((24, n), dtype=torch.float64, device=dev)
    parts, off = [], 0
    for b in wl.batches:
        t = ccd.to_soa(b.verts, dev)
        verts[:, off:off + b.n].copy_(t)
        parts.append(t)
        off += b.n
    seg = ccd.make_segments(counts, kinds, 0.0, 1e-6, args.max_itr)
    sd = ccd.segments_to_device(seg, dev)
    s = torch.cuda.Stream(dev)

    # autotune on a sample: the first instances up to ~2M queries
    k, acc = 0, 0
    while k < len(counts) and acc < 2_000_000:
        acc += counts[k]
        k += 1
    sv = verts[:, :acc].contiguous()
    ssd = ccd.segments_to_device(seg[:k], dev)
    ccd.segments_err_from_bounds(sv, ssd)

    def measure(t):
        wst = ccd.multi_workspace(acc, args.max_itr, t, dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ccd.multi_batch(sv, ssd, args.max_itr, ws=wst, tuning=t, with_checks=False)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    if args.tuning:
        tuning, timings = json.loads(args.tuning), None
    elif args.no_tune:
        tuning, timings = None, None
    else:
        tuning, timings = autotune.get_or_tune(_gpu_name(torch, dev), "multi-instance", measure,
                                               autotune.candidates(sms), reps=1,
                                               retune=args.retune)
    del sv, ssd
    torch.cuda.empty_cache()

    out = ccd.Result(torch.empty(n, dtype=torch.uint8, device=dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.int64, device=dev))
    ws = ccd.multi_workspace(n, args.max_itr, tuning, dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for e in ev:
        e.record(s)                       # creates the handles the library records into
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        ccd.segments_err_from_bounds(verts, sd, stream=s)
        ccd.multi_batch(verts, sd, args.max_itr, ws=ws, out=out, tuning=tuning, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    ccd.set_stage_events(ev)              # recorded by the graph at every replay
    with torch.cuda.graph(g, stream=s):
        ccd.segments_err_from_bounds(verts, sd, stream=s)
        ccd.multi_batch(verts, sd, args.max_itr, ws=ws, out=out, tuning=tuning, stream=s)
    ccd.set_stage_events(None)
    for _ in range(args.warmup):
        with torch.cuda.stream(s):
            g.replay()
    torch.cuda.synchronize(dev)

    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    stage_ms = np.zeros((args.steps, 4))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    clocks.start()
    graph_events = True
    marks[0].record(s)
    for i in range(args.steps):
        with torch.cuda.stream(s):
            g.replay()
        marks[i + 1].record(s)
        s.synchronize()                   # the stage events are reused by every replay
        if graph_events:
            try:
                stage_ms[i] = [ev[j].elapsed_time(ev[j + 1]) for j in range(4)]
            except RuntimeError:
                graph_events = False
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if not graph_events:
        # the graph's event nodes could not be timed: time the stages of the
        # same call launched directly, right after the timed region
        ccd.set_stage_events(ev)
        for i in range(args.steps):
            with torch.cuda.stream(s):
                ccd.segments_err_from_bounds(verts, sd, stream=s)
                ccd.multi_batch(verts, sd, args.max_itr, ws=ws, out=out, tuning=tuning, stream=s)
            s.synchronize()
            stage_ms[i] = [ev[j].elapsed_time(ev[j + 1]) for j in range(4)]
        ccd.set_stage_events(None)
    if world > 1:
        dist.barrier()
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    total_ms = parallel.max_over_ranks(marks[0].elapsed_time(marks[-1]), device=dev)
    bm = total_ms / args.steps
    counters = ccd.workspace_counters(ws, stream=s)
    batched = (out.collides.cpu().numpy(), out.toi.cpu().numpy(), out.out_tol.cpu().numpy())
    checks = out.checks.cpu().numpy()

    # roofline of the dominant stage (all stages are one launch per call
    # except the pooled stage, one per kind, back to back)
    mean_stage = stage_ms.mean(axis=0)
    top = int(np.argmax(mean_stage))
    n_by_kind = {0: sum(c for c, k in zip(counts, kinds) if k == 0),
                 1: sum(c for c, k in zip(counts, kinds) if k == 1)}
    ops, naive = stage_ops(counters, top, n_by_kind)
    achieved = ops / (mean_stage[top] * 1e-3)
    dt = (tuning or {}).get("deep_threads") or 256
    kname = (f"solve_kernel_seg<{dt}> (deep)" if top == 3 else
             STAGES[top].replace("solve_kernel<32>", "solve_kernel_seg<32>")
             .replace("root_kernel", "root_kernel_seg"))
    traffic = stage_traffic({1: "pool_kernel multi-instance",
                             3: f"solve_kernel_seg<{dt}> multi-instance"}.get(top, ""), counters, top)

    fn, toi_bad, off = 0, 0, 0
    for b in wl.batches:
        sl = slice(off, off + b.n)
        hit = b.truth == 1
        fn += int(np.sum(batched[0][sl][hit] == 0))
        toi_bad += int(np.sum(batched[1][sl][hit] > b.t_star[hit]))
        off += b.n

    res = {
        "metric": METRIC, "value": parallel.job_throughput(n, world, bm), "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": bm,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {**multi_config(n, args.scale, args.max_itr),
                   "form": "one ccd_multi_batch call (eps per segment + 4 solver stages) "
                           "replayed from a CUDA graph",
                   "tuning": tuning,
                   "l2": f"inputs {192 * n / 1e9:.2f} GB per step > 129 MB L2; no flush",
                   "parallelism": f"{world} GPU(s), each its own instance set, no collective"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved / 1e9,
                     "peak": peak / 1e9, "unit": "G FP64 ops/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per step of the stage (all its launches)",
                     "peak_source": "FP64 fma.rn.f64 issue rate measured in this run "
                                    "(one FP64 pipe op = one add, mul or fma)",
                     "work": "executed FP64 add/sub/mul/fma instructions from the kernel's "
                             "counters (per kind)",
                     "duration": ("mean CUDA-event time of the stage over the timed replays "
                                  "(events recorded by the graph)" if graph_events else
                                  "mean CUDA-event time of the stage over as many direct "
                                  "launches of the same call right after the timed region"),
                     "naive_equivalent_gops": naive / (mean_stage[top] * 1e-3) / 1e9},
        "stage_ms_per_step": {STAGES[j]: float(mean_stage[j]) for j in range(4)},
        "counters": counters,
        "checks": {"mean": float(checks.mean()), "p99": float(np.percentile(checks, 99)),
                   "max": int(checks.max()),
                   "early_termination_pct": float(100.0 * np.mean(checks >= args.max_itr))},
        "false_negatives": fn, "toi_after_truth": toi_bad,
        "gpu_launches": args.steps * MULTI_LAUNCHES,
        "paper_context": PAPER_CONTEXT,
        "clocks": clk,
        "autotune": None if timings is None else [[t, s_] for t, s_ in timings],
    }

    if not args.no_e2e:
        # host buffers in, results out, as a stream of steps: every step
        # copies its inputs from pinned host memory to the device and its
        # results back, around the graph.  Two buffer sets (a second graph on
        # the second set) let step i+1's upload and step i-1's download run on
        # copy streams while step i computes.
        host = torch.empty((24, n), dtype=torch.float64).pin_memory()
        host.copy_(verts.cpu())
        out_host = [(torch.empty(n, dtype=torch.uint8).pin_memory(),
                     torch.empty(n, dtype=torch.float64).pin_memory(),
                     torch.empty(n, dtype=torch.float64).pin_memory()) for _ in range(2)]
        verts_b = torch.empty_like(verts)
        out_b = ccd.Result(torch.empty_like(out.collides), torch.empty_like(out.toi),
                           torch.empty_like(out.out_tol), torch.empty_like(out.checks))
        g_b = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_b, stream=s):
            ccd.segments_err_from_bounds(verts_b, sd, stream=s)
            ccd.multi_batch(verts_b, sd, args.max_itr, ws=ws, out=out_b, tuning=tuning, stream=s)
        sets = [(verts, out, g), (verts_b, out_b, g_b)]
        up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        # (the graph g records the stage events `ev` at every replay: they
        # must live as long as g, so these take other names)
        xev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("up", "comp", "dl")}
        for b in range(2):                  # handles exist before the first wait
            for k in xev:
                xev[k][b].record(s)

        def e2e_steps(k):
            for i in range(k):
                b = i % 2
                vb, ob, gb = sets[b]
                up.wait_event(xev["comp"][b])         # step i-2 has read its inputs
                with torch.cuda.stream(up):
                    vb.copy_(host, non_blocking=True)
                xev["up"][b].record(up)
                s.wait_event(xev["up"][b])
                s.wait_event(xev["dl"][b])            # step i-2's results are read out
                with torch.cuda.stream(s):
                    gb.replay()
                xev["comp"][b].record(s)
                down.wait_event(xev["comp"][b])
                with torch.cuda.stream(down):
                    out_host[b][0].copy_(ob.collides, non_blocking=True)
                    out_host[b][1].copy_(ob.toi, non_blocking=True)
                    out_host[b][2].copy_(ob.out_tol, non_blocking=True)
                xev["dl"][b].record(down)
            torch.cuda.synchronize(dev)

        e2e_steps(2)
        k_e2e = max(2, min(args.steps, 6))
        t0 = time.perf_counter()
        e2e_steps(k_e2e)
        el = (time.perf_counter() - t0) / k_e2e
        for b in range(2):
            assert np.array_equal(out_host[b][1].numpy(), batched[1])
            assert np.array_equal(out_host[b][0].numpy(), batched[0])
        res["e2e"] = {"value": n * world / el, "unit": "queries/s",
                      "h2d_bytes_per_step": host.numel() * 8, "d2h_bytes_per_step": n * 17,
                      "ms_per_step": el * 1e3, "steps": k_e2e,
                      "api": "ccd_segments_err_from_bounds + ccd_multi_batch (graph)",
                      "overlap": "step i+1's upload and step i-1's download on copy streams "
                                 "during step i's graph (two buffer sets)"}
        del host, out_host, verts_b, out_b, g_b

    if args.no_extras:
        if rank == 0:
            print(json.dumps(res))
        if world > 1:
            dist.destroy_process_group()
        return

    # the plain form: one eps + batch call per instance-kind, in sequence
    wsp = ccd.workspace(max(counts), args.max_itr, dev)
    plain_out = [None] * len(parts)

    def plain_step():
        for j, (t, kind) in enumerate(zip(parts, kinds)):
            e = ccd.err_from_bounds(kind, t)
            plain_out[j] = ccd.batch(kind, t, e, delta=1e-6, max_itr=args.max_itr, ws=wsp,
                                     out=plain_out[j], with_checks=False)

    plain_step()
    torch.cuda.synchronize()
    k_plain = 2
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(k_plain + 1)]
    pev[0].record()
    for i in range(k_plain):
        plain_step()
        pev[i + 1].record()
    torch.cuda.synchronize()
    plain_ms = [pev[i].elapsed_time(pev[i + 1]) for i in range(k_plain)]
    same, off = True, 0
    for j, c in enumerate(counts):
        r = plain_out[j]
        same &= bool(np.array_equal(r.collides.cpu().numpy(), batched[0][off:off + c]))
        same &= bool(np.array_equal(r.toi.cpu().numpy(), batched[1][off:off + c]))
        same &= bool(np.array_equal(r.out_tol.cpu().numpy(), batched[2][off:off + c]))
        off += c
    pm = float(np.mean(plain_ms))
    res["plain"] = {"value": n / (pm * 1e-3), "ms_per_step": pm, "steps": k_plain,
                    "form": f"one eps + batch call per instance-kind ({len(counts)} calls)",
                    "identical_outputs": same}
    res["speedup_vs_plain"] = pm / bm
    del wsp, plain_out, parts
    del ws, out
    torch.cuda.empty_cache()

    # the simulation-shaped 1M workload (the earlier headline), a few steps
    k_sim = 5
    S = measure_simulation_mixed(args, dev, k_sim, 2, parallel.rank_seed(args.seed, rank))
    S["marks"][0].record(S["stream"])
    for i in range(k_sim):
        S["step"](S["stage_sets"][i])
        S["marks"][i + 1].record(S["stream"])
    torch.cuda.synchronize(dev)
    F = simulation_mixed_figures(args, S, k_sim, peak)
    sim_ms = S["marks"][0].elapsed_time(S["marks"][-1]) / k_sim
    res["simulation_mixed_1m"] = {
        "value": S["wl"].n / (sim_ms * 1e-3), "ms_per_step": sim_ms, "steps": k_sim,
        "workload": workload_config(args)["workload"],
        "dominant_kernel": STAGES[F["top"]], "dominant_frac_of_peak": F["achieved"] / peak,
        "dominant_ms": float(F["span_ms"][F["top"]]),
        "false_negatives": F["fn"], "toi_after_truth": F["toi_bad"]}
    del S
    torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        qps, cores, secs, nq = cpu_baseline(wl.batches, args.cpu_sample)
        res["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"{nq} random queries of the workload, spread over the "
                                         f"instances by size ({secs:.1f} s)"}
    if rank == 0:
        print(json.dumps(res))
    if world > 1:
        dist.destroy_process_group()


def run_served(args):
    """The served workload: 16 clients with Poisson arrivals; request sizes
    log-uniform in [100, 500k] x --req-scale (uniform unit-cube generator),
    delta in {1e-4, 1e-6}, ms in {0, 1e-4}, m_I = 1e6.  The C server
    (ccd_batch_*: device-resident request queue, admission within a 40 GB
    arena, 4 lanes, time-sliced deep rounds, a frontier-page pool shared by
    the lanes) against one call per request (ccd_vf_batch / ccd_ee_batch
    with eps from the request's bounds, each after the previous one), at
    offered loads 0.7 and 1.2 of the capacity measured on the same mix."""
    import torch
    from paper_2009_13349_gb300 import ccd
    from paper_2009_13349_gb300 import workloads as W
    from paper_2009_13349_gb300.serve import (Request, Server, latency_stats, run_stream,
                                              serial_baseline)
    dev = torch.device("cuda", 0)
    lo = max(1, int(round(100 * args.req_scale)))
    hi = max(lo + 1, int(round(500_000 * args.req_scale)))
    pool_n = max(4 * hi, 100_000)
    pools = {k: W.unit_cube(k, pool_n, seed=40 + k).verts for k in (0, 1)}
    rng = np.random.default_rng(4)
    budget = 40 << 30
    ws_one = ccd.workspace(hi, 10**6, dev)

    def draw(i, t):
        size = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        kind = int(rng.integers(0, 2))
        a = int(rng.integers(0, pool_n - size))
        return Request(i, kind, pools[kind][a:a + size], delta=float(rng.choice([1e-4, 1e-6])),
                       ms=float(rng.choice([0.0, 1e-4])), max_itr=10**6, arrival=t)

    def run_one(r):
        """One call for one request: upload, eps, batch, results to the host."""
        v = ccd.to_soa(r.aos, dev)
        e = ccd.err_from_bounds(r.kind, v, ms_nonzero=r.ms > 0)
        o = ccd.batch(r.kind, v, e, ms=r.ms, delta=r.delta, max_itr=r.max_itr, ws=ws_one,
                      with_checks=False)
        r.collides, r.toi, r.out_tol = (o.collides.cpu().numpy(), o.toi.cpu().numpy(),
                                        o.out_tol.cpu().numpy())

    # capacity on the request mix: 24 requests solved one after another
    mix = [draw(i, 0.0) for i in range(24)]
    run_one(mix[0])
    t0 = time.perf_counter()
    for r in mix:
        run_one(r)
    cap = sum(r.n for r in mix) / (time.perf_counter() - t0)
    mean_size = (hi - lo) / np.log(hi / lo)
    results = {}
    for load in (0.7, 1.2):
        rate = load * cap / mean_size / 16.0
        spec = []
        for c in range(16):
            t = 0.0
            while True:
                t += rng.exponential(1.0 / rate)
                if t > args.duration:
                    break
                spec.append(t)
        spec.sort()
        state = rng.bit_generator.state
        reqs_a = [draw(i, t) for i, t in enumerate(spec)]
        rng.bit_generator.state = state
        reqs_b = [draw(i, t) for i, t in enumerate(spec)]
        srv = Server(budget=budget, lanes=4, max_batch=max(hi, 1 << 20))
        run_stream(srv, reqs_a)
        st = srv.stats()
        srv.close()
        serial_baseline(run_one, reqs_b)
        same = all(np.array_equal(a.collides, b.collides) and np.array_equal(a.toi, b.toi)
                   and np.array_equal(a.out_tol, b.out_tol) for a, b in zip(reqs_a, reqs_b))
        results[str(load)] = {"served": latency_stats(reqs_a),
                              "one_call_per_request": latency_stats(reqs_b),
                              "identical": bool(same), "requests": len(spec),
                              "server": st}
    hi_load = results["1.2"]
    print(json.dumps({
        "metric": METRIC, "value": hi_load["served"]["queries_per_s"], "unit": "queries/s",
        "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"served: 16 Poisson clients, sizes log-uniform {lo}..{hi} "
                               "(unit-cube generator), delta {1e-4,1e-6}, ms {0,1e-4}, m_I 1e6, "
                               "40 GB arena, 4 lanes",
                   "duration_s": args.duration, "capacity_queries_per_s": cap},
        "loads": results}))


def run_line_search(args):
    """One line-search step (Algorithm 4's CCD part) over a candidate set of
    args.n pairs: distance, p validation, MSCCD passes, reduction.  Also the
    printed cap d = max(p d_i, delta), and the oracle's step on the same set
    (all host cores) for a check and a CPU rate."""
    import torch
    import oracle
    from oracle.linesearch import line_search_ccd
    from paper_2009_13349_gb300 import ccd, workloads as W
    dev = torch.device("cuda", 0)
    wl = W.line_search_scene(n=args.n, seed=args.seed if args.seed != 1 else 5)
    vf, ee = wl.batches[0].verts, wl.batches[1].verts
    verts = ccd.to_soa(np.concatenate([vf, ee]), dev)
    ws = ccd.line_search_workspace(len(vf) + len(ee), 10**6, dev)
    stream = torch.cuda.current_stream(dev)

    def timed(cap, steps, warmup):
        out = None
        for _ in range(warmup):
            ccd.line_search(verts, len(vf), len(ee), p=0.5, delta=1e-6, cap=cap, ws=ws)
        ms = []
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            out = ccd.line_search(verts, len(vf), len(ee), p=0.5, delta=1e-6, cap=cap, ws=ws)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b))
        return out, ms

    clocks = Clocks(0)
    clocks.start()
    res, ms = timed("min", args.steps, args.warmup)
    clk = clocks.stop()
    res_max, ms_max = (timed("max", 1, 0) if args.compare_printed_cap else (None, None))
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    o = line_search_ccd(vf, ee, p=0.5, delta=1e-6, nthreads=cores)
    cpu_s = time.perf_counter() - t0
    keys = ("alpha", "p", "d", "d_i", "eps_i", "delta_i", "passes", "validated")
    n = len(vf) + len(ee)
    step_ms = float(np.median(ms))
    print(json.dumps({
        "metric": "line-search step (Algorithm 4 CCD part): candidates/s", "value": n / (step_ms * 1e-3),
        "unit": "candidates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"line-search scene {n} candidates (VF:EE 1:1), seed 5",
                   "p": 0.5, "delta": 1e-6, "rho": 1e-9, "max_itr": 10**6, "cap": "min"},
        "step": {k: res[k] for k in keys},
        "printed_cap_max": ({"ms_per_step": float(np.median(ms_max)),
                             "step": {k: res_max[k] for k in keys}}
                            if res_max is not None else None),
        "identical_to_oracle": all(res[k] == o[k] for k in keys),
        "cpu_baseline": {"value": n / cpu_s, "unit": "candidates/s", "cores": cores,
                         "kind": "oracle", "sample": "the whole candidate set, one step"},
        "clocks": clk}))


def run_active_set(args):
    """Algorithm 3 on a two-sheet cloth scene: scene eps, broad phase, CCD of
    every candidate, compaction.  Reports candidate pairs per second of the
    whole step and the stage split; the oracle's step on a small scene of the
    same recipe gives the CPU rate."""
    import torch
    from oracle import activeset as A
    from paper_2009_13349_gb300 import ccd, workloads as W
    dev = torch.device("cuda", 0)
    nx = args.nx
    m = W.cloth_scene(nx=nx, seed=6)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    x0, x1, f, e = t(m.x0, torch.float64), t(m.x1, torch.float64), t(m.faces, torch.int32), \
        t(m.edges, torch.int32)
    stream = torch.cuda.current_stream(dev)

    def ev():
        x = torch.cuda.Event(enable_timing=True)
        x.record(stream)
        return x

    out = None
    for _ in range(args.warmup):
        out = ccd.construct_active_set(x0, x1, f, e)
    total, bp, act = [], [], []
    clocks = Clocks(0)
    clocks.start()
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        a = ev()
        margin = float(ccd.scene_eps(x0, x1).max())
        vf, ee = ccd.broad_phase(x0, x1, f, e, margin)
        b = ev()
        out = ccd.active_set(x0, x1, f, e, vf, ee)
        c = ev()
        torch.cuda.synchronize(dev)
        total.append(a.elapsed_time(c))
        bp.append(a.elapsed_time(b))
        act.append(b.elapsed_time(c))
    clk = clocks.stop()
    n_cand = vf.shape[0] + ee.shape[0]
    ms = float(np.median(total))
    small = W.cloth_scene(nx=24, seed=6)
    t0 = time.perf_counter()
    o = A.construct_active_set(small.x0, small.x1, small.faces, small.edges,
                               nthreads=os.cpu_count() or 1)
    cpu_s = time.perf_counter() - t0
    cpu_cand = len(o["candidates"][0]) + len(o["candidates"][1])
    kind = out["kind"].cpu().numpy()
    print(json.dumps({
        "metric": "active-set construction (Algorithm 3): candidate pairs/s", "value": n_cand / (ms * 1e-3),
        "unit": "candidates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"two-sheet cloth {nx}x{nx} per sheet, seed 6",
                   "vertices": int(len(m.x0)), "faces": int(len(m.faces)), "edges": int(len(m.edges)),
                   "delta": 1e-6, "max_itr": 10**6, "margin": "largest scene eps"},
        "stage_ms": {"eps_and_broad_phase": float(np.median(bp)), "ccd_and_compaction": float(np.median(act))},
        "candidates": {"vf": int(vf.shape[0]), "ee": int(ee.shape[0])},
        "active": {"vf": int((kind == 0).sum()), "ee": int((kind == 1).sum())},
        "cpu_baseline": {"value": cpu_cand / cpu_s, "unit": "candidates/s", "cores": os.cpu_count(),
                         "kind": "oracle (brute-force broad phase + CCD)",
                         "sample": "the same recipe at 24x24 per sheet, one step"},
        "clocks": clk}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "multi-instance":
        run_multi_instance(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "line-search":
        run_line_search(args)
    elif args.workload == "active-set":
        run_active_set(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
