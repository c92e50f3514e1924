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
``--impl reference`` times the CPU oracle (plain C, FP64, all host cores) on
the same workload.

Besides the headline step the line carries, each on its own workload:
  plain_fp64     the same step in FP64 throughout;
  tol_1e-4       the 64x64x16 workload at eps = 1e-4, FP64 and mixed;
  vector         the 256x256x10 two-component thin-shell operator
                 (N = 1,310,720), GMRES(50) with FP64 restarts, FP64, mixed
                 and mixed with BF16 Schur products;
  batched        256 independent problems in one handle, problems/s;
  learned        the 512x512x20 workload (N = 5,242,880): full RRQR in FP64,
                 the mixed form, the mixed form with the trained rank
                 predictor (median and spread of several timed samples);
  dc_vs_nodc     PCG iterations and time with and without deferred
                 compression on 16..128 squared x 9 grids at eps 1e-1..1e-4;
  paper_settings the 64x64x16 workload with GMRES(200) to 1e-12 (Sec. 5);
  n_sweep        time per DOF, iterations and mean rank per level over grid
                 sizes (Thm. 1);
  roofline_kernels  each kernel class against its own bound.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "setup+solve s to 1e-8 rel. residual, mixed/batched vs plain FP64, one GB300"
WORKLOAD = "aniso-ice-64x64x16 (N=65536), 1024 leaves x 64 DOF, depth 8, eps 1e-2, PCG rtol 1e-8"
NOMINAL_FP64_TFLOPS = 1.25
# DRAM read + write bytes per k_factor_phase launch of this workload's mixed
# step (mean of the first three level-0 phase launches), from the ncu capture
# summarised in the file below; the kernel is unchanged since that capture
FACTOR_TRAFFIC_BYTES = 72.2e6
FACTOR_TRAFFIC_SOURCE = "profiles/k_factor_phase_aniso-64x64x16_mixed.md"
LEGS = ("tol_1e-4", "vector", "batched", "learned", "dc_vs_nodc", "paper_settings", "n_sweep")


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
    ap.add_argument("--legs", default=",".join(LEGS),
                    help="comma-separated extra legs to run (empty: the headline step only)")
    ap.add_argument("--oracle-large", action="store_true",
                    help="also time the oracle's factorization + PCG of the 512x512x20 workload once (minutes)")
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
    """nvidia-smi clocks and throttle reasons sampled during the timed region
    (into a temporary file that is removed afterwards)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="hs_clocks_", suffix=".csv")
        os.close(fd)
        self.gpu = gpu_index

    def start(self):
        try:
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
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_step(prob, tol, depth, leaf_lines, threads=1):
    """One oracle step: partition + factor + PCG (plain C, FP64; the clusters
    of a phase on `threads` host threads, the result independent of it)."""
    import oracle
    t0 = time.perf_counter()
    perm, lp = oracle.partition(prob, leaf_lines)
    f = oracle.Factor(prob, perm, lp, depth, tol, threads=threads)
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
    cores = host_cores()
    for _ in range(args.warmup):
        cpu_oracle_step(prob, args.tol, 8, 4, threads=cores)
    ts = [cpu_oracle_step(prob, args.tol, 8, 4, threads=cores)[0] for _ in range(args.steps)]
    v = float(np.mean(ts))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": f"the whole workload: oracle partition + factor + PCG, {cores} threads"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Ctx:
    """Stream, L2 flush and barrier shared by the legs."""

    def __init__(self, dev, world):
        import torch
        self.torch = torch
        self.dev = dev
        self.world = world
        self.stream = torch.cuda.Stream(dev)
        self.flush = torch.empty(320 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def flush_l2(self):
        with self.torch.cuda.stream(self.stream):
            self.flush.add_(1.0)

    def barrier(self):
        self.stream.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        self.torch.cuda.synchronize(self.dev)

    def to_dev(self, prob):
        with self.torch.cuda.stream(self.stream):
            d = dict(rp=self.torch.from_numpy(prob.rowptr).to(self.dev), ci=self.torch.from_numpy(prob.col).to(self.dev),
                     va=self.torch.from_numpy(prob.val).to(self.dev), b=self.torch.from_numpy(prob.b).to(self.dev),
                     x=self.torch.empty(prob.n, dtype=self.torch.float64, device=self.dev))
        self.stream.synchronize()
        return d

    def timed_solve(self, prob, d, samples, warm=1, must_converge=True, **kw):
        """Setup + Krylov of `prob` from device-resident A, b: `samples`
        timed runs after `warm` warm-ups; -> (times s, info, true relative
        residual, stats of the last run if profile was asked).  With
        must_converge=False a Krylov solve that stops at maxit is kept."""
        from paper_1811_11248_gb300 import hsolve
        coords = np.ascontiguousarray(prob.coords)
        ts, info, stats = [], None, None
        for k in range(samples + warm):
            opt = hsolve.hs_default_options(mem=hsolve.HS_MEM_DEVICE, stream=self.stream.cuda_stream, coords=coords,
                                            **kw)
            self.flush_l2()
            self.barrier()
            e0 = self.torch.cuda.Event(enable_timing=True)
            e1 = self.torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            h = hsolve.hs_setup(prob.n, d["rp"], d["ci"], d["va"], opt=opt)
            info, rc = h.hs_krylov(d["b"], d["x"], check=False)
            e1.record(self.stream)
            e1.synchronize()
            if k >= warm:
                ts.append(e0.elapsed_time(e1) / 1e3)
            if kw.get("profile"):
                stats = h.kernel_stats()
            h.close()
            if rc != 0 and (must_converge or rc != hsolve.HS_ERR_NOCONV):
                raise RuntimeError(f"solve failed: {hsolve.lib().hs_status_str(rc).decode()}")
        xe = d["x"].cpu().numpy()
        true = float(np.linalg.norm(prob.b - prob.matvec(xe)) / np.linalg.norm(prob.b))
        return ts, info, true, stats


def summary(ts, info, true):
    return {"s": float(np.mean(ts)), "samples": len(ts), "iters": int(info.iters),
            "true_rel_resid": true}


def leg_tol_1e4(ctx):
    """The 64x64x16 workload at eps = 1e-4 (FP64 and mixed)."""
    from paper_1811_11248_gb300 import hsolve, inputs
    prob = inputs.anisotropic_64x64x16()
    d = ctx.to_dev(prob)
    out = {"workload": "aniso-ice-64x64x16, eps 1e-4, PCG rtol 1e-8"}
    for name, prec in (("fp64", hsolve.HS_PREC_FP64), ("mixed", hsolve.HS_PREC_MIXED)):
        # median of 5 (single samples of this leg vary by several ms)
        ts, info, true, _ = ctx.timed_solve(prob, d, 5, tol=1e-4, depth=8, rtol=1e-8, precision=prec)
        out[name] = dict(summary(ts, info, true), median_s=float(np.median(ts)), min_s=float(np.min(ts)),
                         max_s=float(np.max(ts)))
    return out


def leg_vector(ctx):
    """The 256x256x10 two-component thin-shell operator (N = 1,310,720),
    GMRES(50) with FP64 true-residual restarts to 1e-8 (FP64 and mixed)."""
    from paper_1811_11248_gb300 import hsolve, inputs
    prob = inputs.thin_shell_vector()
    d = ctx.to_dev(prob)
    out = {"workload": "vector-256x256x10x2 (N=1310720), ratio 1e6, coupling 0.5, eps 1e-2, GMRES(50)+IR rtol 1e-8"}
    for name, prec, prod in (("fp64", hsolve.HS_PREC_FP64, hsolve.HS_PRODUCTS_TF32X3),
                             ("mixed", hsolve.HS_PREC_MIXED, hsolve.HS_PRODUCTS_TF32X3),
                             ("mixed_bf16", hsolve.HS_PREC_MIXED, hsolve.HS_PRODUCTS_BF16)):
        ts, info, true, _ = ctx.timed_solve(prob, d, 2, tol=1e-2, rtol=1e-8, precision=prec, schur_products=prod,
                                            krylov=hsolve.HS_KRYLOV_GMRES, restart=50)
        out[name] = summary(ts, info, true)
    del d
    return out


def leg_batched(ctx, count, steps):
    """The batched workload: setup + per-problem PCG of `count` independent
    problems (grids 16x16x4 .. 48x48x12, ratio 1e3 .. 1e6) in one handle;
    problems/s = problems / device seconds (A, b resident in HBM)."""
    torch = ctx.torch
    from paper_1811_11248_gb300 import hsolve, inputs
    pp, A = inputs.batched_workload(count)
    d = ctx.to_dev(A)
    coords = np.ascontiguousarray(A.coords)
    out = {"problems": count, "dofs": int(A.n), "workload": "batched anisotropic ice-sheet problems, seeds 0-%d" % (count - 1)}
    for name, prec in (("fp64", hsolve.HS_PREC_FP64), ("mixed", hsolve.HS_PREC_MIXED)):
        opt = hsolve.hs_default_options(tol=1e-2, rtol=1e-8, mem=hsolve.HS_MEM_DEVICE, stream=ctx.stream.cuda_stream,
                                        coords=coords, precision=prec)
        ts, its, res = [], 0, 0.0
        for k in range(1 + max(3, steps // 2)):
            ctx.flush_l2()
            ctx.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            h = hsolve.hs_setup_batched(pp, A.n, d["rp"], d["ci"], d["va"], opt=opt)
            info, rc, it, rel = h.hs_krylov_batched(d["b"], d["x"])
            e1.record(ctx.stream)
            e1.synchronize()
            h.close()
            if k > 0:  # the first pass is a warm-up
                ts.append(e0.elapsed_time(e1) / 1e3)
            its, res = max(its, int(it.max())), max(res, float(rel.max()))
        t = float(np.mean(ts))
        out[name] = {"s": t, "samples": len(ts), "problems_per_s": count / t, "iters_max": its, "rel_resid_max": res}
    out["problems_per_s"] = out["mixed"]["problems_per_s"]
    return out


def leg_learned(ctx, samples=5):
    """Rank predictor trained on the GPU with the library's kernels on ranks
    recorded from the 16x16x8, 64x64x16 and batched workloads (problems
    0-63), then the 512x512x20 workload (N = 5,242,880, ratio 1e6, sigma
    1.5) set up and solved by full RRQR in FP64, by the mixed form, and by
    the mixed form with the predictor; `samples` timed runs of each form
    after a warm-up (median, min, max), plus one profiled run of the mixed
    form for the HBM roofline of its solve phase and SpMV."""
    from paper_1811_11248_gb300 import hsolve, inputs, rank_model
    st = ctx.stream.cuda_stream
    t0 = time.perf_counter()
    f1, r1, s1 = rank_model.collect(inputs.anisotropic_16x16x8(), depth=4, stream=st)
    f2, r2, s2 = rank_model.collect(inputs.anisotropic_64x64x16(), depth=8, stream=st)
    f3, r3, s3 = rank_model.collect_batched([inputs.batched_problem(k) for k in range(64)], stream=st)
    X, R, S = np.concatenate([f1, f2, f3]), np.concatenate([r1, r2, r3]), np.concatenate([s1, s2, s3])
    model, losses = rank_model.fit(X, R, S, epochs=40)
    t_train = time.perf_counter() - t0
    prob = inputs.anisotropic_512x512x20()
    d = ctx.to_dev(prob)
    out = {"workload": "aniso-ice-512x512x20 (N=5242880), ratio 1e6, sigma 1.5, eps 1e-2, PCG rtol 1e-8",
           "training": {"samples": int(len(R)), "steps": int(len(losses)), "loss_first": float(losses[:10].mean()),
                        "loss_last": float(losses[-50:].mean()), "collect_and_train_s": t_train}}
    packed = model.packed()
    for name, prec, mv in (("fp64_rrqr", hsolve.HS_PREC_FP64, None), ("mixed", hsolve.HS_PREC_MIXED, None),
                           ("learned", hsolve.HS_PREC_MIXED, packed)):
        ts, info, true, _ = ctx.timed_solve(prob, d, samples, tol=1e-2, rtol=1e-8, precision=prec, rank_model=mv)
        out[name] = {"median_s": float(np.median(ts)), "min_s": float(np.min(ts)), "max_s": float(np.max(ts)),
                     "samples": len(ts), "iters": int(info.iters), "true_rel_resid": true}
    out["learned_gain"] = 1.0 - out["learned"]["median_s"] / out["mixed"]["median_s"]
    # ranks on the workload (predictor accuracy) and the profiled mixed run
    opt = hsolve.hs_default_options(tol=1e-2, rtol=1e-8, mem=hsolve.HS_MEM_DEVICE, stream=st,
                                    coords=np.ascontiguousarray(prob.coords), precision=hsolve.HS_PREC_FP64,
                                    record_ranks=1)
    h = hsolve.hs_setup(prob.n, d["rp"], d["ci"], d["va"], opt=opt)
    f5, r5, s5 = h.rank_samples()
    h.close()
    out["predictor_on_512x512x20"] = rank_model.accuracy(model, f5, r5, s5)
    _, _, _, stats = ctx.timed_solve(prob, d, 1, tol=1e-2, rtol=1e-8, precision=hsolve.HS_PREC_MIXED, profile=1)
    del d
    return out, stats


def leg_dc_vs_nodc(ctx):
    """PCG iterations and setup + solve time with deferred compression and
    without it (options.no_dc), FP64, on 16, 32, 64, 128 squared x 9 grids
    (ratio 1e6, sigma 1, Neumann top, shelf), eps 1e-1 .. 1e-4 (Tables 5-6)."""
    from paper_1811_11248_gb300 import hsolve, inputs
    out = {"workload": "aniso-ice nx x nx x 9, ratio 1e6, sigma 1 seed 1, PCG rtol 1e-8, FP64", "rows": []}
    for nx in (16, 32, 64, 128):
        prob = inputs.grid_operator(nx, nx, 9, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
        d = ctx.to_dev(prob)
        row = {"nx": nx, "n": int(prob.n)}
        for nodc in (0, 1):
            key = "nodc" if nodc else "dc"
            row[key] = {}
            for eps in (1e-1, 1e-2, 1e-3, 1e-4):
                ts, info, true, _ = ctx.timed_solve(prob, d, 1, tol=eps, rtol=1e-8, precision=hsolve.HS_PREC_FP64,
                                                    no_dc=nodc)
                row[key][f"{eps:g}"] = {"iters": int(info.iters), "s": float(ts[0]), "true_rel_resid": true}
        out["rows"].append(row)
    return out


def rounding_floor(prob, x):
    """u || |A| |x| || / ||b||: the smallest relative residual an FP64
    evaluation of b - A x can resolve at x."""
    rows = np.repeat(np.arange(prob.n), np.diff(prob.rowptr))
    ax = np.zeros(prob.n)
    np.add.at(ax, rows, np.abs(prob.val) * np.abs(x[prob.col]))
    return float(np.finfo(float).eps * np.linalg.norm(ax) / np.linalg.norm(prob.b))


def leg_paper_settings(ctx):
    """Sec. 5's solver settings: right-preconditioned GMRES(200), stopping at
    1e-12, at most 1000 iterations (FP64 and mixed), on the 64x64x16 grid at
    vertical:horizontal ratio 1e3, where 1e-12 lies above the FP64 rounding
    floor of the residual; and on the ratio-1e6 workload, whose floor
    (about 5e-10) 1e-12 lies below, the residual it stagnates at."""
    from paper_1811_11248_gb300 import hsolve, inputs
    out = {}
    for ratio in (1e3, 1e6):
        prob = inputs.grid_operator(64, 64, 16, ratio=ratio, sigma=1.0, seed=1, bc="ice", shelf=0.5)
        d = ctx.to_dev(prob)
        key = f"ratio_{ratio:g}"
        out[key] = {"workload": f"aniso-ice-64x64x16 ratio {ratio:g}, eps 1e-2, GMRES(200) rtol 1e-12 maxit 1000"}
        for name, prec in (("fp64", hsolve.HS_PREC_FP64), ("mixed", hsolve.HS_PREC_MIXED)):
            ts, info, true, _ = ctx.timed_solve(prob, d, 1, warm=1 if ratio < 1e6 else 0,
                                                must_converge=ratio < 1e6, tol=1e-2, depth=8, rtol=1e-12,
                                                maxit=1000, precision=prec, krylov=hsolve.HS_KRYLOV_GMRES,
                                                restart=200)
            out[key][name] = summary(ts, info, true)
            out[key][name]["rounding_floor"] = rounding_floor(prob, d["x"].cpu().numpy())
        del d
    return out


def leg_n_sweep(ctx):
    """Thm. 1 (factor cost O(N r^2), solve O(N r)): the mixed form on
    32..256 squared x 16 grids (ratio 1e6, sigma 1, eps 1e-2): setup + solve
    time per DOF, iterations, and the mean rank of the clusters eliminated
    at each level."""
    from paper_1811_11248_gb300 import hsolve, inputs
    out = {"workload": "aniso-ice nx x nx x 16, ratio 1e6, sigma 1 seed 1, eps 1e-2, mixed, PCG rtol 1e-8", "rows": []}
    for nx in (32, 64, 128, 256):
        prob = inputs.grid_operator(nx, nx, 16, ratio=1e6, sigma=1.0, seed=1, bc="ice", shelf=0.5)
        d = ctx.to_dev(prob)
        ts, info, true, _ = ctx.timed_solve(prob, d, 2, tol=1e-2, rtol=1e-8, precision=hsolve.HS_PREC_MIXED)
        opt = hsolve.hs_default_options(tol=1e-2, mem=hsolve.HS_MEM_DEVICE, stream=ctx.stream.cuda_stream,
                                        coords=np.ascontiguousarray(prob.coords), precision=hsolve.HS_PREC_MIXED)
        h = hsolve.hs_setup(prob.n, d["rp"], d["ci"], d["va"], opt=opt)
        ranks = []
        for l in range(h.num_levels()):
            s0, fi, ph = h.level_info(l)
            done = ph >= 0
            ranks.append(float(fi[done].mean()) if done.any() else 0.0)
        h.close()
        t = float(np.mean(ts))
        out["rows"].append({"nx": nx, "n": int(prob.n), "s": t, "us_per_dof": 1e6 * t / prob.n,
                            "iters": int(info.iters), "true_rel_resid": true,
                            "mean_rank_per_level": [round(x, 3) for x in ranks[:6]]})
        del d
    return out


def kernel_roofline(stats, p64, p32, hbm):
    """Each kernel class against its own bound: the factor and Schur kernels
    by their FP64 and FP32 algorithmic flops (roofline time F64 / P64 +
    F32 / P32), the solve phase and the SpMV by their algorithmic bytes
    against the HBM copy bandwidth.  frac = roofline time / measured time."""
    out = {}
    names = {"factor": "k_factor_phase", "factor_fused": "k_factor_level_fused", "schur": "k_schur_phase"}
    for cls, kern in names.items():
        st = stats[cls]
        if st["ms"] <= 0:
            continue
        t_roof = st["flops"] / (p64 * 1e12) + st["flops32"] / (p32 * 1e12)
        out[kern] = {"bound": "alu", "ms": round(st["ms"], 4), "launches": st["launches"],
                     "fp64_flops": st["flops"], "fp32_flops": st["flops32"],
                     "roofline_ms": round(1e3 * t_roof, 4), "frac": t_roof / (st["ms"] * 1e-3)}
    for cls, kern in (("apply", "solve phase (k_ap_*, k_dense_gemv, k_permute)"), ("spmv", "k_spmv")):
        st = stats[cls]
        if st["ms"] <= 0:
            continue
        gbs = st["bytes"] / (st["ms"] * 1e-3) / 1e9
        out[kern] = {"bound": "hbm", "ms": round(st["ms"], 4), "launches": st["launches"], "bytes": st["bytes"],
                     "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
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
    legs = [x for x in args.legs.split(",") if x]
    if args.no_learned and "learned" in legs:
        legs.remove("learned")
    if args.batched <= 0 and "batched" in legs:
        legs.remove("batched")

    ctx = Ctx(dev, world)
    stream = ctx.stream
    prob = inputs.anisotropic_64x64x16()
    n = prob.n
    d = ctx.to_dev(prob)
    rp, ci, va, b, x = d["rp"], d["ci"], d["va"], d["b"], d["x"]
    # inputs in pinned host memory (e2e)
    h_rp = torch.from_numpy(prob.rowptr).pin_memory()
    h_ci = torch.from_numpy(prob.col).pin_memory()
    h_va = torch.from_numpy(prob.val).pin_memory()
    h_b = torch.from_numpy(prob.b).pin_memory()
    h_x = torch.zeros(n, dtype=torch.float64).pin_memory()
    coords = np.ascontiguousarray(prob.coords)

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
            ctx.flush_l2()
            ctx.barrier()
            l0 = hsolve.hs_launch_count()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h, info = step(prec=prec)
            e1.record(stream)
            e1.synchronize()
            launches += hsolve.hs_launch_count() - l0
            ctx.barrier()
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
        ctx.flush_l2()
        ctx.barrier()
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
    ctx.flush_l2()
    ctx.barrier()
    hp, infop = step(profile=1, prec=hsolve.HS_PREC_FP64)
    stats = hp.kernel_stats()
    hp.close()
    ctx.flush_l2()
    ctx.barrier()
    hp, infop = step(profile=1)
    stats_mx = hp.kernel_stats()
    hp.close()
    fp64_peak = hsolve.hs_measure_fp64_peak(stream.cuda_stream)
    fp32_peak = hsolve.hs_measure_fp32_peak(stream.cuda_stream)
    hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
    fac = stats_mx["factor"]
    # the level-0 factor kernel of the mixed step: FP64 Cholesky + scaling and
    # FP32 compression, as FP64-equivalent flops (the FP32 part weighted by
    # the measured FP64 / FP32 peak ratio) over its CUDA-event time
    eq_flops = fac["flops"] + fac["flops32"] * fp64_peak / fp32_peak
    achieved = eq_flops / (fac["ms"] * 1e-3) / 1e12 if fac["ms"] > 0 else 0.0
    roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak if fp64_peak > 0 else None, "traffic": FACTOR_TRAFFIC_BYTES,
            "traffic_unit": "bytes per launch (ncu dram read + write)", "traffic_source": FACTOR_TRAFFIC_SOURCE,
            "kernel": "k_factor_phase (level 0: FP64 Cholesky + scaling, FP32 CPQR in the mixed form)",
            "peak_kind": f"measured FP64 FMA probe of this GPU (nominal {NOMINAL_FP64_TFLOPS} TFLOP/s); "
                         f"FP32 work weighted by the measured FP32 probe ({fp32_peak:.1f} TFLOP/s)",
            "avg_launch_ms": fac["ms"] / max(fac["launches"], 1),
            "fp64_flops_per_launch": fac["flops"] / max(fac["launches"], 1),
            "fp32_flops_per_launch": fac["flops32"] / max(fac["launches"], 1)}
    ksum = sum(v["ms"] for v in stats_mx.values())

    line = {"metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "precision": "mixed: FP64 Cholesky/scaling/Krylov residual, FP32 compression (CPQR) and stored "
                                    "factor, Schur products on the tensor cores (TF32 x3 split, FP32 accumulate)",
                       "l2": "flushed (320 MB write) before each step", "replicas": world},
            "iters": it_mx, "rel_resid": res_mx,
            "plain_fp64": {"value": t64, "unit": "s", "iters": it64, "rel_resid": res64,
                           "kernel_ms": {k: round(v["ms"], 4) for k, v in stats.items()}},
            "e2e": {"value": float(np.mean(e2e_times)), "unit": "s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roof, "clocks": clk,
            "kernel_ms": {k: round(v["ms"], 4) for k, v in stats_mx.items()},
            "kernel_ms_sum": round(ksum, 4),
            "peaks": {"fp64_tflops": fp64_peak, "fp32_tflops": fp32_peak, "hbm_gbs": hbm,
                      "kind": "FMA probes measured in this run; HBM from MEASURED_PEAKS.json"},
            "roofline_kernels": {"aniso-ice-64x64x16 mixed": kernel_roofline(stats_mx, fp64_peak, fp32_peak, hbm),
                                 "aniso-ice-64x64x16 fp64": kernel_roofline(stats, fp64_peak, fp32_peak, hbm)}}
    del d
    for leg in legs:
        t0 = time.perf_counter()
        if leg == "tol_1e-4":
            line[leg] = leg_tol_1e4(ctx)
        elif leg == "vector":
            line[leg] = leg_vector(ctx)
        elif leg == "batched":
            line[leg] = leg_batched(ctx, args.batched, args.steps)
        elif leg == "learned":
            line[leg], st5 = leg_learned(ctx)
            line["roofline_kernels"]["aniso-ice-512x512x20 mixed"] = kernel_roofline(st5, fp64_peak, fp32_peak, hbm)
        elif leg == "dc_vs_nodc":
            line[leg] = leg_dc_vs_nodc(ctx)
        elif leg == "paper_settings":
            line[leg] = leg_paper_settings(ctx)
        elif leg == "n_sweep":
            line[leg] = leg_n_sweep(ctx)
        if args.verbose:
            print(f"leg {leg}: {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        dt1, it = cpu_oracle_step(prob, args.tol, 8, 4, threads=1)
        dtn, _ = cpu_oracle_step(prob, args.tol, 8, 4, threads=cores)
        line["cpu_baseline"] = {"value": dtn, "unit": "s", "cores": cores, "kind": "oracle",
                                "sample": f"one full step of the workload (partition + factor + PCG), {cores} threads "
                                          "(the clusters of a phase in parallel)",
                                "one_thread_s": dt1, "iters": it}
        if args.oracle_large:
            import oracle
            p5 = inputs.anisotropic_512x512x20()
            t0 = time.perf_counter()
            perm, lp = oracle.partition(p5, 4)
            f5 = oracle.Factor(p5, perm, lp, oracle.default_depth(len(lp) - 1), 1e-2, threads=cores)
            t1 = time.perf_counter()
            _, it5, rr5, rc5 = f5.pcg(rtol=1e-8)
            line["cpu_baseline"]["aniso-ice-512x512x20"] = {"partition_factor_s": t1 - t0,
                                                             "pcg_s": time.perf_counter() - t1, "iters": it5,
                                                             "cores": cores}
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
