#!/usr/bin/env python
"""Benchmark of the batched FP64 inclusion-based CCD root finder on GB300.

Workload (one "step"): the simulation-shaped mixed workload of 1,000,000
queries (500,000 vertex-face + 500,000 edge-edge, seed 1): scene eps from
bounds, then ccd_vf_batch and ccd_ee_batch, delta = 1e-6, m_I = 1e6, ms = 0.
Inputs are resident in HBM when the timed region starts; they total 192 MB,
more than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (bounded sample per step).
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
# FP64 add/sub/mul of the fixed F expression.  A t-quantity evaluation (one t
# value: 12 positions x0 + dx t = 24 ops, then VF 9 / EE 6 differences) is
# shared by a run of boxes with equal t_L; a box evaluation from two
# t-quantity sets costs 2 t x 3 coords x (VF 10 / EE 12) + 3 (w(B)).
T_OPS = {0: 24 + 9, 1: 24 + 6}
BOX_OPS = {0: 2 * 3 * 10 + 3, 1: 2 * 3 * 12 + 3}
# the same check evaluated on its own (no sharing): 2 t-quantities + box
OPS_PER_CHECK = {k: 2 * T_OPS[k] + BOX_OPS[k] for k in (0, 1)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=20_000)
    ap.add_argument("--ref-sample", type=int, default=4_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--deep-slots", type=int, default=None,
                    help="cap the deep-solver slots (smaller workspace, e.g. for profiling)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n, seed):
    from paper_2009_13349_gb300 import workloads as W
    return W.simulation_mixed(n=n, seed=seed)


def cpu_baseline(wl, sample: int, seed: int = 123):
    """Oracle on a bounded random sample of the workload, all host cores."""
    import oracle
    rng = np.random.default_rng(seed)
    cores = os.cpu_count() or 1
    total_q, total_s = 0, 0.0
    for b in wl.batches:
        k = max(1, int(round(sample * b.n / wl.n)))
        idx = rng.choice(b.n, k, replace=False)
        err = oracle.err_from_bounds(b.kind, b.verts)      # scene eps of the full batch
        t0 = time.perf_counter()
        oracle.ccd_batch(b.kind, b.verts[idx], err, delta=1e-6, max_itr=10**6, nthreads=cores)
        total_s += time.perf_counter() - t0
        total_q += k
    return total_q / total_s, cores, total_s, total_q


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = make_workload(args.n, args.seed)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(7)
    errs = {b.kind: oracle.err_from_bounds(b.kind, b.verts) for b in wl.batches}

    def step():
        q, s = 0, 0.0
        for b in wl.batches:
            k = max(1, int(round(args.ref_sample * b.n / wl.n)))
            idx = rng.choice(b.n, k, replace=False)
            t0 = time.perf_counter()
            oracle.ccd_batch(b.kind, b.verts[idx], errs[b.kind], delta=1e-6, max_itr=10**6,
                             nthreads=cores)
            s += time.perf_counter() - t0
            q += k
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
        "config": {"workload": f"simulation-mixed {args.n} queries (VF:EE 1:1), seed {args.seed}",
                   "delta": 1e-6, "max_itr": 10**6, "ms": 0.0,
                   "sample_per_step": args.ref_sample},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.ref_sample} random queries of the workload per step"},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
    }
    print(json.dumps(out))


def run_native(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2009_13349_gb300 import ccd

    wl = make_workload(args.n, args.seed + rank)   # each rank its own batch (weak scaling)
    batches = wl.batches
    verts = [ccd.to_soa(b.verts, dev) for b in batches]
    host = [torch.from_numpy(np.ascontiguousarray(b.verts.T)).pin_memory() for b in batches]
    ws = [ccd.workspace(b.n, 10**6, dev, deep_slots=args.deep_slots) for b in batches]
    res = [ccd.Result(torch.empty(b.n, dtype=torch.uint8, device=dev),
                      torch.empty(b.n, dtype=torch.float64, device=dev),
                      torch.empty(b.n, dtype=torch.float64, device=dev),
                      torch.empty(b.n, dtype=torch.int64, device=dev)) for b in batches]
    stream = torch.cuda.current_stream(dev)

    def step(stage_sets=None):
        for j, b in enumerate(batches):
            if stage_sets is not None:
                ccd.set_stage_events(stage_sets[j])
            err = ccd.err_from_bounds(b.kind, verts[j])
            ccd.batch(b.kind, verts[j], err, delta=1e-6, max_itr=10**6, ws=ws[j], out=res[j])
        ccd.set_stage_events(None)

    # FP64 pipe peak, measured in this run (fma.rn.f64 chains, all SMs)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = 0.0
    for _ in range(3):
        ms, ops = ccd.fp64_peak_probe(sms * 8, 8192)
        peak = max(peak, ops / (ms * 1e-3))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    def new_event():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    stage_sets = [[[new_event() for _ in range(4)] for _ in batches] for _ in range(args.steps)]
    marks = [new_event() for _ in range(args.steps + 1)]
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = Clocks(local)
    clocks.start()
    marks[0].record(stream)
    for s in range(args.steps):
        step(stage_sets[s])
        marks[s + 1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    step_ms = [marks[s].elapsed_time(marks[s + 1]) for s in range(args.steps)]
    total_ms = marks[0].elapsed_time(marks[-1])
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    stage_ms = np.zeros((len(batches), 3))
    for s in range(args.steps):
        for j in range(len(batches)):
            ev = stage_sets[s][j]
            for k in range(3):
                stage_ms[j, k] += ev[k].elapsed_time(ev[k + 1]) / args.steps
    counters = [ccd.workspace_counters(w) for w in ws]

    # correctness of the timed outputs against the constructed truths
    fn, toi_bad, checks = 0, 0, []
    for j, b in enumerate(batches):
        col = res[j].collides.cpu().numpy()
        toi = res[j].toi.cpu().numpy()
        hit = b.truth == 1
        fn += int(np.sum(col[hit] == 0))
        toi_bad += int(np.sum(toi[hit] > b.t_star[hit]))
        checks.append(res[j].checks.cpu().numpy())
    checks = np.concatenate(checks)

    # roofline of the dominant kernel
    names = ["root_kernel", "solve_kernel<32> (small frontier)", "solve_kernel<512> (deep)"]
    per_kernel = stage_ms.sum(axis=0)
    top = int(np.argmax(per_kernel))
    # executed FP64 arithmetic, from the kernel's own counters
    if top == 0:
        alg_ops = sum(b.n * OPS_PER_CHECK[b.kind] for b in batches)
        naive = alg_ops
    else:
        sfx = "small" if top == 1 else "deep"
        alg_ops = sum(counters[j]["tq_" + sfx] * T_OPS[b.kind] +
                      counters[j]["evals_" + sfx] * BOX_OPS[b.kind] for j, b in enumerate(batches))
        naive = sum(counters[j]["checks_" + sfx] * OPS_PER_CHECK[b.kind]
                    for j, b in enumerate(batches))
    achieved = alg_ops / (per_kernel[top] * 1e-3)
    total_queries = sum(b.n for b in batches) * world
    value = total_queries / (total_ms / args.steps * 1e-3)

    out = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"simulation-mixed {args.n} queries per GPU (VF:EE 1:1), seed {args.seed}",
                   "delta": 1e-6, "max_itr": 10**6, "ms": 0.0,
                   "l2": "inputs 192 MB per step > 129 MB L2; no flush",
                   "parallelism": f"{world} GPU(s), queries sharded, no collective"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "roofline": {"bound": "alu", "kernel": names[top], "achieved": achieved / 1e9,
                     "peak": peak / 1e9, "unit": "GFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": "FP64 fma.rn.f64 issue rate measured in this run "
                                    "(one FP64 pipe op = one add or mul; -fmad=false)",
                     "work": "executed FP64 add/sub/mul from the kernel's counters",
                     "naive_equivalent_gflops": naive / (per_kernel[top] * 1e-3) / 1e9},
        "stage_ms_per_step": {names[k]: float(per_kernel[k]) for k in range(3)},
        "counters": {("VF" if b.kind == 0 else "EE"): counters[j] for j, b in enumerate(batches)},
        "checks": {"mean": float(checks.mean()), "p50": float(np.percentile(checks, 50)),
                   "p99": float(np.percentile(checks, 99)), "max": int(checks.max()),
                   "early_termination_pct": float(100.0 * np.mean(checks >= 10**6))},
        "false_negatives": fn, "toi_after_truth": toi_bad,
        "gpu_launches": args.steps * len(batches) * 6,
        "clocks": clk,
    }

    if not args.no_e2e:
        h2d = sum(h.numel() * 8 for h in host)
        d2h = sum(b.n * (1 + 8 + 8) for b in batches)
        out_host = [(torch.empty(b.n, dtype=torch.uint8).pin_memory(),
                     torch.empty(b.n, dtype=torch.float64).pin_memory(),
                     torch.empty(b.n, dtype=torch.float64).pin_memory()) for b in batches]
        dres = [ccd.Result(r.collides, r.toi, r.out_tol, None) for r in res]

        def e2e_step():
            for j, b in enumerate(batches):
                verts[j].copy_(host[j], non_blocking=True)
                err = ccd.err_from_bounds(b.kind, verts[j])
                ccd.batch(b.kind, verts[j], err, delta=1e-6, max_itr=10**6, ws=ws[j],
                          out=dres[j])
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
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": el * 1e3}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        qps, cores, secs, nq = cpu_baseline(wl, args.cpu_sample)
        out["cpu_baseline"] = {"value": qps, "unit": "queries/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"{nq} random queries of the workload ({secs:.1f} s)"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
