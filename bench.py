#!/usr/bin/env python
"""Benchmark: setup + solve seconds to a 1e-8 relative residual on one GB300.

Workload (one step): the 64x64x16 extruded ice-sheet operator (N = 65,536,
vertical:horizontal ratio 1e6, log-normal horizontal coefficient sigma 1 seed
1, Neumann top, frictionless shelf on half the domain), column-preserving
partition into 1024 leaves of 2x2 lines, 8 levels, eps = 1e-2:
partition + symbolic analysis + numeric factorization (Algorithm 1) + PCG with
the hierarchical preconditioner (Algorithm 2) to ||b - A x|| / ||b|| <= 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``value`` = device time per step with A and b resident in HBM (CUDA events on
the solver's stream, max over ranks); ``e2e`` = the same step through hs_solve
on host buffers (host<->device copies inside the timed region).  With N > 1
every rank solves its own replica (the path does not shard: replicas only).
``--impl reference`` times the CPU oracle (plain C, FP64, one core) on the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "setup+solve s to 1e-8 rel. residual, mixed/batched vs plain FP64, one GB300"
WORKLOAD = "aniso-ice-64x64x16 (N=65536), 1024 leaves x 64 DOF, depth 8, eps 1e-2, PCG rtol 1e-8"
NOMINAL_FP64_TFLOPS = 1.25
# DRAM read + write bytes per k_factor_phase launch of this workload's mixed step: mean of the
# first three level-0 phase launches in an ncu capture of the current kernel
FACTOR_TRAFFIC_BYTES = 71.9e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tol", type=float, default=1e-2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=256,
                    help="problems of the batched workload timed beside the main step (0: skip)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-rank leg (512x512x20 workload)")
    ap.add_argument("--verbose", action="store_true")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, device):
    """The largest `value` over all ranks of the process group (the step
    time of the slowest replica)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 8:
                    continue
                try:
                    sm.append(float(f[0]))
                    smax.append(float(f[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_step(prob, tol, depth, leaf_lines):
    """One oracle step: partition + factor + PCG (plain C, FP64, one thread)."""
    import oracle
    t0 = time.perf_counter()
    perm, lp = oracle.partition(prob, leaf_lines)
    f = oracle.Factor(prob, perm, lp, depth, tol)
    x, it, rr, rc = f.pcg(rtol=1e-8)
    dt = time.perf_counter() - t0
    assert rc == 0 and rr <= 1e-8
    return dt, it


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1811_11248_gb300 import inputs
    import oracle
    oracle.build()
    prob = inputs.anisotropic_64x64x16()
    for _ in range(args.warmup):
        cpu_oracle_step(prob, args.tol, 8, 4)
    ts = [cpu_oracle_step(prob, args.tol, 8, 4)[0] for _ in range(args.steps)]
    v = float(np.mean(ts))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": "the whole workload: oracle partition + factor + PCG, one thread"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_leg(args, stream, dev, barrier, flush_l2):
    """The batched workload: setup + per-problem PCG of `args.batched`
    independent problems (grids 16x16x4 .. 48x48x12, ratio 1e3 .. 1e6) in one
    handle; problems/s = problems / device seconds (A, b resident in HBM)."""
    import torch
    from paper_1811_11248_gb300 import hsolve, inputs
    cnt = args.batched
    pp, A = inputs.batched_workload(cnt)
    with torch.cuda.stream(stream):
        rp = torch.from_numpy(A.rowptr).to(dev)
        ci = torch.from_numpy(A.col).to(dev)
        va = torch.from_numpy(A.val).to(dev)
        b = torch.from_numpy(A.b).to(dev)
        x = torch.empty(A.n, dtype=torch.float64, device=dev)
    coords = np.ascontiguousarray(A.coords)
    stream.synchronize()
    out = {"problems": cnt, "dofs": int(A.n), "workload": "batched anisotropic ice-sheet problems, seeds 0-%d" % (cnt - 1)}
    for name, prec in (("fp64", hsolve.HS_PREC_FP64), ("mixed", hsolve.HS_PREC_MIXED)):
        opt = hsolve.hs_default_options(tol=1e-2, rtol=1e-8, mem=hsolve.HS_MEM_DEVICE, stream=stream.cuda_stream,
                                        coords=coords, precision=prec)
        ts, its, res = [], 0, 0.0
        for k in range(1 + max(1, args.steps // 2)):
            flush_l2()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = hsolve.hs_setup_batched(pp, A.n, rp, ci, va, opt=opt)
            info, rc, it, rel = h.hs_krylov_batched(b, x)
            e1.record(stream)
            e1.synchronize()
            h.close()
            if k > 0:  # the first pass is a warm-up
                ts.append(e0.elapsed_time(e1) / 1e3)
            its, res = max(its, int(it.max())), max(res, float(rel.max()))
        t = float(np.mean(ts))
        out[name] = {"s": t, "problems_per_s": cnt / t, "iters_max": its, "rel_resid_max": res}
    out["problems_per_s"] = out["mixed"]["problems_per_s"]
    return out


def learned_leg(args, stream, dev, barrier, flush_l2):
    """Rank predictor trained on the GPU with the library's kernels on ranks
    recorded from the 16x16x8, 64x64x16 and batched workloads (problems
    0-63), then the 512x512x20 workload (N = 5,242,880, ratio 1e6, sigma 1.5)
    set up and solved by full RRQR in FP64, by the mixed form, and by the
    mixed form with the predictor (rank-0 speculation)."""
    import torch
    from paper_1811_11248_gb300 import hsolve, inputs, rank_model
    t0 = time.perf_counter()
    f1, r1, s1 = rank_model.collect(inputs.anisotropic_16x16x8(), depth=4, stream=stream.cuda_stream)
    f2, r2, s2 = rank_model.collect(inputs.anisotropic_64x64x16(), depth=8, stream=stream.cuda_stream)
    f3, r3, s3 = rank_model.collect_batched([inputs.batched_problem(k) for k in range(64)], stream=stream.cuda_stream)
    X, R, S = np.concatenate([f1, f2, f3]), np.concatenate([r1, r2, r3]), np.concatenate([s1, s2, s3])
    model, losses = rank_model.fit(X, R, S, epochs=40)
    t_train = time.perf_counter() - t0
    prob = inputs.anisotropic_512x512x20()
    with torch.cuda.stream(stream):
        rp = torch.from_numpy(prob.rowptr).to(dev)
        ci = torch.from_numpy(prob.col).to(dev)
        va = torch.from_numpy(prob.val).to(dev)
        b = torch.from_numpy(prob.b).to(dev)
        x = torch.empty(prob.n, dtype=torch.float64, device=dev)
    coords = np.ascontiguousarray(prob.coords)
    stream.synchronize()
    out = {"workload": "aniso-ice-512x512x20 (N=5242880), ratio 1e6, sigma 1.5, eps 1e-2, PCG rtol 1e-8",
           "training": {"samples": int(len(R)), "steps": int(len(losses)), "loss_first": float(losses[:10].mean()),
                        "loss_last": float(losses[-50:].mean()), "collect_and_train_s": t_train}}
    packed = model.packed()
    for name, prec, mv in (("fp64_rrqr", hsolve.HS_PREC_FP64, None), ("mixed", hsolve.HS_PREC_MIXED, None),
                           ("learned", hsolve.HS_PREC_MIXED, packed)):
        ts = []
        for k in range(3 if name == "fp64_rrqr" else 2):
            # pass 0 warms up, pass 1 is timed, pass 2 records the ranks
            opt = hsolve.hs_default_options(tol=1e-2, rtol=1e-8, mem=hsolve.HS_MEM_DEVICE, stream=stream.cuda_stream,
                                            coords=coords, precision=prec, rank_model=mv, record_ranks=int(k == 2))
            flush_l2()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = hsolve.hs_setup(prob.n, rp, ci, va, opt=opt)
            info, rc = h.hs_krylov(b, x)
            e1.record(stream)
            e1.synchronize()
            if k == 1:
                ts.append(e0.elapsed_time(e1) / 1e3)
            if k == 2:
                f5, r5, s5 = h.rank_samples()
            h.close()
        out[name] = {"s": float(np.mean(ts)), "iters": int(info.iters), "rel_resid": float(info.rel_resid)}
    out["predictor_on_512x512x20"] = rank_model.accuracy(model, f5, r5, s5)
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1811_11248_gb300 import build as libbuild
    from paper_1811_11248_gb300 import hsolve, inputs
    libbuild.build()
    hsolve.lib()

    prob = inputs.anisotropic_64x64x16()
    n = prob.n
    stream = torch.cuda.Stream(dev)
    # inputs resident in HBM (value) and in pinned host memory (e2e)
    with torch.cuda.stream(stream):
        rp = torch.from_numpy(prob.rowptr).to(dev)
        ci = torch.from_numpy(prob.col).to(dev)
        va = torch.from_numpy(prob.val).to(dev)
        b = torch.from_numpy(prob.b).to(dev)
        x = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(320 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    h_rp = torch.from_numpy(prob.rowptr).pin_memory()
    h_ci = torch.from_numpy(prob.col).pin_memory()
    h_va = torch.from_numpy(prob.val).pin_memory()
    h_b = torch.from_numpy(prob.b).pin_memory()
    h_x = torch.zeros(n, dtype=torch.float64).pin_memory()
    coords = np.ascontiguousarray(prob.coords)
    stream.synchronize()

    def opt(mem, profile=0, prec=None):
        prec = hsolve.HS_PREC_MIXED if prec is None else prec
        return hsolve.hs_default_options(tol=args.tol, depth=8, leaf_lines=4, rtol=1e-8, mem=mem,
                                         profile=profile, stream=stream.cuda_stream, coords=coords,
                                         precision=prec)

    def step(profile=0, prec=None):
        """partition + setup + PCG, device-resident A and b."""
        h = hsolve.hs_setup(n, rp, ci, va, opt=opt(hsolve.HS_MEM_DEVICE, profile, prec))
        info, rc = h.hs_krylov(b, x)
        return h, info

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.add_(1.0)

    def barrier():
        stream.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def nvtx(name=None):
        """NVTX range around a timed loop (a profiler can filter on it)."""
        try:
            if name:
                torch.cuda.nvtx.range_push(name)
            else:
                torch.cuda.nvtx.range_pop()
        except Exception:
            pass

    def timed(prec):
        times, iters, resid, launches = [], [], [], 0
        nvtx("timed_fp64" if prec == hsolve.HS_PREC_FP64 else "timed_mixed")
        for _ in range(args.steps):
            flush_l2()
            barrier()
            l0 = hsolve.hs_launch_count()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h, info = step(prec=prec)
            e1.record(stream)
            e1.synchronize()
            launches += hsolve.hs_launch_count() - l0
            barrier()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(info.iters)
            resid.append(info.rel_resid)
            h.close()
        nvtx()
        return float(np.mean(times)), int(np.max(iters)), float(np.max(resid)), launches // max(args.steps, 1)

    for prec in (hsolve.HS_PREC_FP64, hsolve.HS_PREC_MIXED):
        for _ in range(max(3, args.warmup)):
            h, info = step(prec=prec)
            h.close()

    clocks = ClockSampler(local)
    clocks.start()
    t64, it64, res64, _ = timed(hsolve.HS_PREC_FP64)
    t_step, it_mx, res_mx, launches = timed(hsolve.HS_PREC_MIXED)
    clk = clocks.stop()
    if world > 1:
        t_step = max_over_ranks(t_step, dev)

    # e2e: hs_solve on host buffers (H2D of A and b, D2H of x inside)
    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        flush_l2()
        barrier()
        t0 = time.perf_counter()
        info_e, rc = hsolve.hs_solve(n, h_rp, h_ci, h_va, h_b, h_x, opt=opt(hsolve.HS_MEM_HOST))  # mixed form
        e2e_times.append(time.perf_counter() - t0)
        assert rc == 0 and info_e.rel_resid <= 1e-8
    xe = h_x.numpy()
    true_res = float(np.linalg.norm(prob.b - prob.matvec(xe)) / np.linalg.norm(prob.b))
    assert true_res <= 1e-8, true_res
    h2d = prob.rowptr.nbytes + prob.col.nbytes + prob.val.nbytes + prob.b.nbytes
    d2h = 8 * n

    # per-kernel-class device times (profiled replicas of one step of each form)
    flush_l2()
    barrier()
    hp, infop = step(profile=1, prec=hsolve.HS_PREC_FP64)
    stats = hp.kernel_stats()
    hp.close()
    flush_l2()
    barrier()
    hp, infop = step(profile=1)
    stats_mx = hp.kernel_stats()
    hp.close()
    fp64_peak = hsolve.hs_measure_fp64_peak(stream.cuda_stream)
    fac = stats_mx["factor"]
    achieved = fac["flops"] / (fac["ms"] * 1e-3) / 1e12 if fac["ms"] > 0 else 0.0
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak if fp64_peak > 0 else None, "traffic": FACTOR_TRAFFIC_BYTES,
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "kernel": "k_factor_phase (FP64 Cholesky + scaling, FP32 CPQR in the mixed form)",
            "peak_kind": f"measured FP64 FMA probe (nominal {NOMINAL_FP64_TFLOPS} TFLOP/s)",
            "avg_launch_ms": fac["ms"] / max(fac["launches"], 1),
            "flops_per_launch": fac["flops"] / max(fac["launches"], 1)}

    line = {"metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "precision": "mixed: FP64 Cholesky/scaling/Krylov residual, FP32 compression (CPQR), Schur products and "
                                    "stored factor",
                       "l2": "flushed (320 MB write) before each step", "replicas": world},
            "iters": it_mx, "rel_resid": res_mx,
            "plain_fp64": {"value": t64, "unit": "s", "iters": it64, "rel_resid": res64,
                           "kernel_ms": {k: round(v["ms"], 4) for k, v in stats.items()}},
            "e2e": {"value": float(np.mean(e2e_times)), "unit": "s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roof, "clocks": clk,
            "kernel_ms": {k: round(v["ms"], 4) for k, v in stats_mx.items()}}
    if args.batched > 0:
        line["batched"] = batched_leg(args, stream, dev, barrier, flush_l2)
    if not args.no_learned:
        line["learned"] = learned_leg(args, stream, dev, barrier, flush_l2)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, it = cpu_oracle_step(prob, args.tol, 8, 4)
        line["cpu_baseline"] = {"value": dt, "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": "one full step of the workload (partition + factor + PCG), one thread",
                                "iters": it}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
