"""Benchmark: KKT refactor + solve throughput and latency on GB300.

One step = one interior-point iteration's linear-algebra work on a fresh
K_k: equilibrate, scatter, refactor, solve, residual and FGMRES refinement to
a backward error <= tol (Alg. 1 loop body). Default workload: the 25,000-bus
grid shaped like the paper's Northeast system (FP64), mu from 1e-1 to 1e-9.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload northeast25k|eastern70k|grid200] [--precision fp64|fp32]

Prints one JSON line (rank 0). Under torchrun every rank runs its own
independent scenario sequence (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from kktgen import WORKLOADS, KKTPattern, make_grid, mu_schedule  # noqa: E402

METRIC = "KKT refactor+solves/s & p99 latency at rel. residual ≤1e-10 vs plain FP64"
UNIT = "refactor+solves/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="northeast25k", choices=sorted(WORKLOADS) + ["batch", "serving"])
    ap.add_argument("--sessions", type=int, default=256, help="serving: number of sessions")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: total request rate (1/s)")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: HBM budget")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the mixed-precision comparison run")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--max-pivots", type=int, default=None, help="pivots per supernode (library default if unset)")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernels one by one instead of CUDA graphs")
    ap.add_argument("--assemble", action="store_true",
                    help="each step also evaluates the model on the GPU (K values from the iterate)")
    ap.add_argument("--precond", default="lu", choices=["lu", "jacobi"],
                    help="refinement preconditioner: exact triangular solves or Jacobi sweeps")
    ap.add_argument("--sweeps", type=int, default=4, help="Jacobi sweeps per triangular factor")
    ap.add_argument("--slack-range", type=float, nargs=2, default=None, metavar=("LO", "HI"),
                    help="keep the inequality slacks' term -(1/sigma_s), 1/sigma_s log-uniform on [LO, HI], "
                         "on the flow-limit rows (single-system workloads; off: the literal -dc)")
    ap.add_argument("--tree-min-fronts", type=int, default=None,
                    help="levels with fewer fronts run in the persistent tree kernels (library default if unset)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(base, rank):
    """Every rank solves its own scenario sequence (replicas, weak scaling)."""
    return base + 1000 * rank


def reduce_max(x, device=None):
    """Max over the ranks of a host float: one all-reduce, the only
    collective of the bench (timing, not data path)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, steps, max_total_ms):
    """Whole-job throughput: the steps of every rank over the slowest rank's time."""
    return world * steps / (max_total_ms / 1000.0)


def workload(name, seed):
    w = WORKLOADS[name]
    grid = make_grid(seed, w["n_bus"], w["n_branch"], w["n_gen"])
    pat = KKTPattern(grid)
    mus = mu_schedule(w["mu0"], w["mu1"], w["steps"])
    return w, pat, mus


# Distinct inputs the timed steps cycle through (every step reads its inputs
# from HBM: L2 is flushed before each timed step), so a timed region long
# enough for the clock record (hundreds of steps) needs neither hours of input
# generation nor gigabytes of inputs.
POOL_STEPS = 24


def pool_size(args):
    return args.warmup + min(args.steps, POOL_STEPS)


def at(args, i):
    """Input index of step i: the warm-up steps, then the timed steps cycling the pool."""
    n = pool_size(args)
    return i if i < n else args.warmup + (i - args.warmup) % (n - args.warmup)


def inputs(pat, mus, seed, count, slack_range=None):
    """Values and right-hand sides for `count` IPM steps (schedule cycled);
    slack_range: keep the inequality slacks' term in the (2,2) block."""
    vals, rhs = [], []
    for i in range(count):
        k = i % len(mus)
        vals.append(pat.values(pat.point(seed, k, mus[k], slack_range=slack_range)))
        rhs.append(pat.rhs(seed, k))
    return vals, rhs


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- algorithmic bytes

def algorithmic_bytes(plan, n, nnz, wbytes):
    """Minimal traffic of each phase, from the factor sizes (per refactor / solve)."""
    nlu = plan["nnz_lu"]
    return {
        "refactor": nnz * (8 + 4) + nlu * (wbytes + 4) + n * 8,
        "solve": nlu * (wbytes + 4) + 4 * n * wbytes,
        "spmv": nnz * (8 + 4) + 3 * n * 8,
    }


# DRAM bytes (read + write) of the dominant kernel per unit of the roofline
# (for tree_factor_kernel: its launches of one refactorization) from one ncu
# capture of the same command (profiles/), keyed by (kernel, workload,
# precision, tree levels); an entry is removed whenever the kernel changes.
MEASURED_TRAFFIC = {
    ("tree_factor_kernel", "northeast25k", "fp64", 58): 24890368 + 10752,
}

PHASE_OF = {
    "front_warp_kernel": "refactor", "front_leaf_kernel": "refactor", "front_cta_kernel": "refactor",
    "front_panel_kernel": "refactor",
    "schur_tile_kernel": "refactor", "ruiz_kernel": "refactor", "scale_kernel": "refactor",
    "solve_fwd_kernel": "solve", "solve_bwd_kernel": "solve", "solve_pre_kernel": "solve",
    "solve_post_kernel": "solve", "spmv_resid_kernel": "spmv", "tree_factor_kernel": "refactor",
    "tree_fwd_kernel": "solve", "tree_bwd_kernel": "solve", "jacobi_kernels": "solve",
}


# ----------------------------------------------------------------- reference arm

def cpu_run(pat, vals, rhs, tol, budget_s, max_steps):
    """The oracle as it stands, single thread: analysis untimed, then per step
    Ruiz + LU with frozen pivots + FGMRES to tol, until the budget is used.
    Returns the step times, the backward errors and the solutions (inputs
    0, 1, ... in order)."""
    import oracle as O
    an = O.analyze(pat.rowptr, pat.colidx, vals[0])
    times, oms, xs = [], [], []
    t_all = time.perf_counter()
    for i in range(min(max_steps, len(vals))):
        t0 = time.perf_counter()
        lu, d, _ = O.refactor(pat.rowptr, pat.colidx, vals[i], an)
        x, it, om = O.fgmres(pat.rowptr, pat.colidx, vals[i], lu, d, rhs[i], 30, 10, tol)
        times.append(time.perf_counter() - t0)
        oms.append(om)
        xs.append(x)
        if time.perf_counter() - t_all > budget_s and len(times) >= 2:
            break
    return times, oms, xs


def error_vs_oracle(x_oracle, results):
    """Error of each GPU result against the oracle's FP64 solution of the same
    system K_k x = b_k: |x - x_oracle|_inf / |x_oracle|_inf per input, for each
    precision in `results` (name -> list of solutions, inputs 0, 1, ... in
    order). Both sides stop at the same backward error, so the difference is
    bounded by the condition number of K_k times that tolerance, not by it."""
    out = {"inputs": len(x_oracle), "norm": "max|x - x_oracle| / max|x_oracle|"}
    for name, xs in results.items():
        if xs is None:
            continue
        errs = []
        for a, o in zip(xs, x_oracle):
            den = float(np.max(np.abs(o)))
            errs.append(float(np.max(np.abs(np.asarray(a) - o))) / (den if den > 0 else 1.0))
        out[name] = {"max": max(errs), "median": float(np.median(errs)), "per_result": errs}
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        raise SystemExit("--impl reference times the oracle on a single-system workload")
    w, pat, mus = workload(args.workload, args.seed)
    n_in = args.warmup + args.steps
    vals_p, rhs_p = inputs(pat, mus, args.seed, pool_size(args), args.slack_range)
    vals = [vals_p[at(args, i)] for i in range(n_in)]
    rhs = [rhs_p[at(args, i)] for i in range(n_in)]
    times, oms, _ = cpu_run(pat, vals, rhs, args.tol, 1e9, n_in)
    t = times[args.warmup:] if len(times) > args.warmup else times
    ms = 1000.0 * sum(t) / len(t)
    value = 1000.0 / ms
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": len(t), "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64", "tol": args.tol,
                   "slack_range": args.slack_range},
        "p50_ms": 1000 * float(np.percentile(t, 50)), "p99_ms": 1000 * float(np.percentile(t, 99)),
        "omega_max": float(max(oms)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d full steps of %s (oracle analysis untimed)" % (len(t), args.workload)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ native arm

def run_native(args):
    import torch
    import paper_2302_08656_gb300 as K

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    seed = rank_seed(args.seed, rank)       # independent scenario per rank
    w, pat, mus = workload(args.workload, seed)
    n_in = pool_size(args)
    vals_h, rhs_h = inputs(pat, mus, seed, n_in, args.slack_range)
    vals = [torch.from_numpy(v).to(dev) for v in vals_h]
    rhs = [torch.from_numpy(b).to(dev) for b in rhs_h]
    xs = [torch.empty_like(b) for b in rhs]
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(4 * l2, 512 << 20), dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed_run(solver, tag):
        stream = torch.cuda.current_stream()
        for i in range(args.warmup):
            solver.refactor_refine(vals[i], rhs[i], out=xs[i], tol=args.tol, raise_on_noconv=False)
        l0 = solver.info().launches
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        oms, iters = [], []
        barrier()
        for t in range(args.steps):
            i = at(args, args.warmup + t)
            flush.zero_()
            ev0[t].record(stream)
            _, info = solver.refactor_refine(vals[i], rhs[i], out=xs[i], tol=args.tol, raise_on_noconv=False)
            ev1[t].record(stream)
            oms.append(info.backward_err)
            iters.append(info.iters)
        barrier()
        launches = solver.info().launches - l0
        ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        return ms, oms, iters, launches

    lib_opts = {"graphs": not args.no_graphs}
    if args.max_pivots:
        lib_opts["max_pivots"] = args.max_pivots
    if args.tree_min_fronts is not None:
        lib_opts["tree_min_fronts"] = args.tree_min_fronts
    if args.precond != "lu":
        lib_opts["precond"] = args.precond
        lib_opts["jacobi_sweeps"] = args.sweeps
    s64 = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=args.precision, **lib_opts)
    plan = s64.plan()
    sampler = ClockSampler(dev.index)
    sampler.start()
    ms, oms, iters, launches = timed_run(s64, args.precision)
    clocks = sampler.stop()
    main_name = "fp64" if args.precision == "fp64" else "fp32_ir"
    results = {main_name: [x.cpu().numpy() for x in xs]}     # one result per pool input, after the timed region
    total_ms = sum(ms)
    if world > 1:
        total_ms = reduce_max(total_ms, device=dev)
    value = aggregate_rate(world, args.steps, total_ms)

    # mixed precision on the same matrices (the graded comparison: FP32 LU + FP64 FGMRES vs plain FP64)
    other = None
    if not args.no_fp32:
        oprec = "fp32" if args.precision == "fp64" else "fp64"
        s32 = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=oprec, **lib_opts)
        ms32, oms32, it32, _ = timed_run(s32, oprec)
        results["fp32_ir" if oprec == "fp32" else "fp64"] = [x.cpu().numpy() for x in xs]
        other = {"precision": "fp32_ir" if oprec == "fp32" else "fp64", "value": 1000.0 * len(ms32) / sum(ms32),
                 "p50_ms": float(np.percentile(ms32, 50)), "p99_ms": float(np.percentile(ms32, 99)),
                 "omega_max": float(max(oms32)), "fgmres_iters_mean": float(np.mean(it32))}
        s32.close()

    # end to end through the C ABI with host buffers (copies inside the timed call)
    hv = [torch.from_numpy(v).pin_memory() for v in vals_h]
    hb = [torch.from_numpy(b).pin_memory() for b in rhs_h]
    hx = torch.empty(pat.n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    barrier()
    for t in range(args.steps):
        i = at(args, args.warmup + t)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64.step_host(hv[i].numpy(), hb[i].numpy(), tol=args.tol, out=hx.numpy(), raise_on_noconv=False)
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    barrier()
    e2e = {"value": 1000.0 * len(e2e_ms) / sum(e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(8 * (pat.nnz + pat.n)), "d2h_bytes_per_step": int(8 * pat.n),
           "p99_ms": float(np.percentile(e2e_ms, 99))}

    # per-kernel timing pass (profiling mode, separate from the timed run)
    s64.set_profiling(True)
    s64.kernel_stats()
    nprof = min(3, args.steps)
    for t in range(nprof):
        i = at(args, args.warmup + t)
        s64.refactor_refine(vals[i], rhs[i], out=xs[i], tol=args.tol, raise_on_noconv=False)
    stats = s64.kernel_stats()
    s64.set_profiling(False)
    wbytes = 8 if args.precision == "fp64" else 4
    ab = algorithmic_bytes(plan, pat.n, pat.nnz, wbytes)
    phase_ms = {}
    for name, (cnt, kms) in stats.items():
        ph = PHASE_OF.get(name)
        if ph:
            phase_ms[ph] = phase_ms.get(ph, 0.0) + kms
    dom = max(stats.items(), key=lambda kv: kv[1][1])[0] if stats else None
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    roofline = None
    if dom:
        ph = PHASE_OF.get(dom, "refactor")
        if dom == "tree_factor_kernel":
            # the kernel's own algorithmic bytes (original entries, panels,
            # contribution blocks) per refactorization; the tree part runs as
            # one or two launches of it (wide levels, then the narrow top)
            n_units = nprof
            bytes_unit = plan["tree_bytes"]
            kms = stats[dom][1] / max(1, n_units)
        else:
            n_units = nprof if ph == "refactor" else stats.get(
                "solve_post_kernel" if ph == "solve" else "spmv_resid_kernel", (0, 0.0))[0]
            bytes_unit = ab[ph]
            kms = phase_ms[ph] / max(1, n_units)
        achieved = bytes_unit / (kms / 1000.0) / 1e9
        key = (dom, args.workload, args.precision, plan["tree_levels"])
        traffic = MEASURED_TRAFFIC.get(key)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": traffic, "kernel": dom, "peak_source": peak_src,
                    "algorithmic_bytes_per_unit": bytes_unit, "units_profiled": n_units,
                    "ms_per_unit": kms, "launches_per_unit": stats[dom][0] / max(1, n_units),
                    "refactor_phase": {"algorithmic_bytes": ab["refactor"], "ms": phase_ms.get("refactor", 0.0) / nprof,
                                       "achieved_gbs": ab["refactor"] / (phase_ms.get("refactor", 1e-9) / nprof / 1000.0) / 1e9}}

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        times, coms, xo = cpu_run(pat, vals_h, rhs_h, args.tol, args.cpu_seconds, n_in)
        cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d of the %s steps (oracle analysis untimed), single thread"
                         % (len(times), args.workload),
               "omega_max": float(max(coms))}
        try:
            accuracy = error_vs_oracle(xo, results)
        except Exception as e:                     # reported in the line, never fatal to it
            accuracy = {"error": repr(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "buses": w["n_bus"], "branches": w["n_branch"],
                       "generators": w["n_gen"], "n": pat.n, "nnz": pat.nnz, "precision": args.precision,
                       "tol": args.tol, "mu": [w["mu0"], w["mu1"]], "slack_range": args.slack_range,
                       "l2": "flushed between timed steps (%d MB write)" % (flush.numel() >> 20),
                       "fronts": plan["n_fronts"], "levels": plan["n_levels"], "nnz_lu": plan["nnz_lu"],
                       "tree_levels": plan["tree_levels"], "tree_units": plan["tree_units"]},
            "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
            "omega_max": float(max(oms)), "fgmres_iters_mean": float(np.mean(iters)),
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": int(launches), "kernel_ms_per_step": {k: v[1] / nprof for k, v in stats.items()},
            "library_options": lib_opts, "converged_steps": int(sum(1 for o in oms if o <= args.tol)),
            "comparison": other, "error_vs_oracle": accuracy,
        }
        print(json.dumps(line), flush=True)
    s64.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ batched (many instances)

def run_batch(args):
    """64 instances of one 2,000-bus pattern and 16 of one 10,000-bus pattern,
    values and right-hand sides from a different seed per instance; FP32
    factors + FP64 refinement; the two batches refactor concurrently; the
    schedule of each is chosen by the autotuner."""
    import torch
    import paper_2302_08656_gb300 as K
    from paper_2302_08656_gb300 import autotune

    dev = torch.device("cuda", 0)
    groups = [("batch2k", 64), ("batch10k", 16)]
    n_in = pool_size(args)
    prec = "fp32" if args.precision == "fp64" else args.precision   # this configuration runs FP32 LU
    ctxs, vals, rhs, outs, omegas, tune_info = [], [], [], [], [], {}
    for name, count in groups:
        w = WORKLOADS[name]
        pat = KKTPattern(make_grid(args.seed, w["n_bus"], w["n_branch"], w["n_gen"]))
        mus = mu_schedule(w["mu0"], w["mu1"], w["steps"])
        v_steps, b_steps = [], []
        for t in range(n_in):
            k = t % len(mus)
            v_steps.append(torch.from_numpy(np.concatenate(
                [pat.values(pat.point(args.seed * 1000 + i, k, mus[k])) for i in range(count)])).to(dev))
            b_steps.append(torch.from_numpy(np.concatenate(
                [pat.rhs(args.seed * 1000 + i, k) for i in range(count)])).to(dev))
        best, times = autotune.tune(pat.rowptr, pat.colidx, pat.n_primal, v_steps[0], b_steps[0],
                                    precision=prec, count=count)
        tune_info[name] = {"count": count, "n": pat.n, "nnz": pat.nnz, "chosen": best, "ms_by_max_pivots": times}
        s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=count, precision=prec, **best)
        ctxs.append(s)
        vals.append(v_steps)
        rhs.append(b_steps)
        outs.append(torch.empty_like(b_steps[0]))
        omegas.append(torch.empty(count, dtype=torch.float64).pin_memory())
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(t):
        t = at(args, t)
        K.refactor_batched(ctxs, [vals[g][t] for g in range(len(ctxs))])
        for g, s in enumerate(ctxs):
            s.solve_checked(rhs[g][t], outs[g], omegas[g])
        torch.cuda.synchronize()
        worst, iters = 0.0, 0
        for g, s in enumerate(ctxs):
            om = omegas[g].numpy()
            if np.any(~(om <= args.tol)):
                _, infos = s.refine(rhs[g][t], out=outs[g], tol=args.tol, raise_on_noconv=False)
                om = np.array([i.backward_err for i in infos])
                iters += sum(i.iters for i in infos)
            worst = max(worst, float(np.max(om)))
        return worst, iters

    for t in range(args.warmup):
        step(t)
    l0 = sum(s.info().launches for s in ctxs)
    ms, oms, its = [], [], []
    sampler = ClockSampler(0)
    sampler.start()
    for t in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        om, it = step(args.warmup + t)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        oms.append(om)
        its.append(it)
    clocks = sampler.stop()
    launches = sum(s.info().launches for s in ctxs) - l0
    per_step = sum(c for _, c in groups)
    line = {
        "metric": METRIC, "value": per_step * len(ms) / (sum(ms) / 1000.0), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batch", "groups": tune_info, "precision": prec, "tol": args.tol,
                   "l2": "flushed between timed steps (512 MB write)",
                   "note": "one step = one refactor + solve (+ refinement if needed) of all 80 instances"},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "omega_max": float(max(oms)), "fgmres_iters_total": int(sum(its)), "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for s in ctxs:
        s.close()


# ------------------------------------------------------------------- serving

def run_serving(args):
    """Sessions with grid sizes log-uniform over 500..25,000 buses, 30..80 IPM
    iterations each, Poisson arrivals at `rate` requests/s in total; FP32 factors
    + FP64 refinement to tol; HBM budget for admission. Each session cycles two
    pre-generated value sets (to bound input generation time)."""
    import torch
    from paper_2302_08656_gb300.serve import (GpuBackend, Server, SessionSpec, estimate_bytes,
                                              log_uniform_sizes, poisson_arrivals)

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(args.seed)
    sizes = log_uniform_sizes(rng, args.sessions, 500, 25_000)
    iters = rng.integers(30, 81, size=args.sessions)
    arrivals = poisson_arrivals(rng, args.rate, list(iters))
    sessions = []
    t0 = time.perf_counter()
    for sid, B in enumerate(sizes):
        grid = make_grid(args.seed * 7919 + sid, B, int(round(1.28 * B)), max(1, int(round(0.2 * B))))
        pat = KKTPattern(grid)
        vs = [torch.from_numpy(pat.values(pat.point(sid, k, 10.0 ** -(1 + 4 * k)))).to(dev) for k in range(2)]
        bs = [torch.from_numpy(pat.rhs(sid, k)).to(dev) for k in range(2)]
        sessions.append(SessionSpec(sid, pat.rowptr, pat.colidx, pat.n_primal, arrivals[sid],
                                    (lambda v, b: (lambda k: (v[k % 2], b[k % 2])))(vs, bs),
                                    est_bytes=estimate_bytes(pat.nnz)))
    gen_s = time.perf_counter() - t0
    backend = GpuBackend(precision="fp32", tol=args.tol, streams=16)
    server = Server(backend, budget_bytes=int(args.budget_gb * (1 << 30)), max_inflight=16, analysis_workers=12)
    sampler = ClockSampler(0)
    sampler.start()
    rep = server.run(sessions)
    clocks = sampler.stop()
    line = {
        "metric": METRIC, "value": rep.solves_per_s, "unit": UNIT, "n_gpus": 1, "steps": rep.completed,
        "warmup": 0, "ms_per_step": 1000.0 * rep.wall_s / max(1, rep.completed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving", "sessions": args.sessions, "buses": [500, 25000], "iterations": [30, 80],
                   "rate_per_s": args.rate, "budget_gb": args.budget_gb, "precision": "fp32", "tol": args.tol,
                   "input_generation_s": gen_s},
        "p50_ms": rep.percentile(50), "p99_ms": rep.percentile(99),
        "p50_ms_steady": rep.percentile(50, steady=True), "p99_ms_steady": rep.percentile(99, steady=True),
        "omega_max": float(max(rep.omegas)), "refined": rep.refined, "max_sessions_resident": rep.max_sessions,
        "max_device_bytes": rep.max_bytes, "admission_waits": rep.admission_waits, "wall_s": rep.wall_s,
        "failed": [[sid, k, err] for sid, k, err in rep.failed],
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ IPM step with GPU model evaluation

def run_ipm(args):
    """One step = GPU model evaluation of K_k from the iterate (V, theta,
    lambda, Sigma) + refactor + solve + refinement; e2e copies the iterate
    (not the nnz values of K) to the device and the solution back."""
    import torch
    import paper_2302_08656_gb300 as K

    dev = torch.device("cuda", 0)
    w = WORKLOADS[args.workload]
    grid = make_grid(args.seed, w["n_bus"], w["n_branch"], w["n_gen"])
    pat = KKTPattern(grid)
    mus = mu_schedule(w["mu0"], w["mu1"], w["steps"])
    n_in = pool_size(args)
    pts = [pat.point(args.seed, i % len(mus), mus[i % len(mus)]) for i in range(n_in)]
    rhs_h = [pat.rhs(args.seed, i % len(mus)) for i in range(n_in)]
    it_h = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (p.V, p.theta, p.lam, p.sigma)]
            for p in pts]
    b_h = [torch.from_numpy(b).pin_memory() for b in rhs_h]
    it_d = [[a.to(dev) for a in it] for it in it_h]
    b_d = [b.to(dev) for b in b_h]
    model = K.KKTModel.from_grid(grid)
    opts = {"precision": args.precision}
    if args.tree_min_fronts is not None:
        opts["tree_min_fronts"] = args.tree_min_fronts
    s = K.KKTSolver(model.rowptr, model.colidx, model.n_primal, **opts)
    vals = torch.empty(model.nnz, dtype=torch.float64, device=dev)
    x = torch.empty(pat.n, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    pt0 = pts[0]

    def step(i, V, th, lam, sig, b):
        model.assemble(V, th, lam, sig, pt0.delta_w, pt0.delta_c, out=vals)
        _, info = s.refactor_refine(vals, b, out=x, tol=args.tol, raise_on_noconv=False)
        return info

    for i in range(args.warmup):
        step(i, *it_d[i], b_d[i])
    ms, oms = [], []
    sampler = ClockSampler(0)
    sampler.start()
    for t in range(args.steps):
        i = at(args, args.warmup + t)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = step(i, *it_d[i], b_d[i])
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        oms.append(info.backward_err)
    clocks = sampler.stop()
    xh = torch.empty(pat.n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for t in range(args.steps):
        i = at(args, args.warmup + t)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dv = [a.to(dev, non_blocking=True) for a in it_h[i]]
        db = b_h[i].to(dev, non_blocking=True)
        step(i, *dv, db)
        xh.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    h2d = int(sum(a.numel() * 8 for a in it_h[0]) + b_h[0].numel() * 8)
    line = {
        "metric": METRIC, "value": 1000.0 * len(ms) / sum(ms), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "assemble": True, "n": pat.n, "nnz": pat.nnz,
                   "precision": args.precision, "tol": args.tol, "l2": "flushed between timed steps (512 MB write)",
                   "note": "one step = GPU model evaluation + refactor + solve + refinement"},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "omega_max": float(max(oms)),
        "e2e": {"value": 1000.0 * len(e2e_ms) / sum(e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(8 * pat.n), "p99_ms": float(np.percentile(e2e_ms, 99))},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    s.close()
    model.close()


def main():
    args = parse()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.assemble:
        run_ipm(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
