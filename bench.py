"""Benchmark: KKT refactor + solve throughput and latency on GB300.

One step = one interior-point iteration's linear-algebra work on a fresh
K_k: equilibrate, scatter, refactor, solve, residual and FGMRES refinement to
a backward error <= tol (Alg. 1 loop body). Default workload: the
70,000-bus grid shaped like the paper's Eastern system, mu from 1e-1 to 1e-9,
numeric LU and triangular solves in FP32 with the residual and FGMRES in FP64
(the value), against the plain FP64 path on the same matrices (fp64_arm).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                    [--workload eastern70k|northeast25k|grid200|batch|serving]
                    [--precision fp32|fp64]

Prints one JSON line (rank 0). Under torchrun every rank runs its own
independent scenario sequence (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import gc
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
PREC_NAME = {"fp64": "fp64", "fp32": "fp32_ir"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="eastern70k", choices=sorted(WORKLOADS) + ["batch", "serving"])
    ap.add_argument("--sessions", type=int, default=256, help="serving: number of sessions")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: total request rate (1/s)")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: HBM budget")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32"],
                    help="factor precision of the main arm (fp32: FP32 LU + FP64 refinement)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", "--no-compare", dest="no_compare", action="store_true",
                    help="skip the other-precision arm on the same matrices")
    ap.add_argument("--no-determined", action="store_true", help="skip the determined-x record")
    ap.add_argument("--det-tol", type=float, default=1e-14,
                    help="determined-x record: refinement tolerance of both precisions")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU-baseline sample")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="--impl reference: budget of its timed steps (at least 3 are timed)")
    ap.add_argument("--max-pivots", type=int, default=None, help="pivots per supernode (library default if unset)")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernels one by one instead of CUDA graphs")
    ap.add_argument("--assemble", action="store_true",
                    help="each step also evaluates the model on the GPU (K values from the iterate)")
    ap.add_argument("--ipm-loop", action="store_true",
                    help="each step is a whole interior-point solve (kkt_ipm_solve) of the workload's grid with "
                         "seeded loads and limits, from the flat start")
    ap.add_argument("--precond", default="lu", choices=["lu", "jacobi", "block"],
                    help="refinement preconditioner: exact triangular solves, Jacobi sweeps, or block-Jacobi sweeps "
                         "(each front's pivots solved exactly inside the sweep)")
    ap.add_argument("--sweeps", type=int, default=4, help="Jacobi sweeps per triangular factor")
    ap.add_argument("--slack-range", type=float, nargs=2, default=None, metavar=("LO", "HI"),
                    help="keep the inequality slacks' term -(1/sigma_s), 1/sigma_s log-uniform on [LO, HI], "
                         "on the flow-limit rows (single-system workloads; off: the literal -dc)")
    ap.add_argument("--group", action="store_true",
                    help="batch: the value refactors the two patterns as one group (the tops of both assembly "
                         "trees in one launch) instead of on forked streams")
    ap.add_argument("--saddle", action="store_true",
                    help="each step is the saddle-point specialised solve (kkt_hykkt_solve) of the workload's "
                         "systems with the slacks' term kept (--slack-range, default 1e-2 1e2), timed beside the "
                         "direct refactor + refine of the same systems")
    ap.add_argument("--gamma", type=float, default=1e8, help="saddle: the augmentation gamma")
    ap.add_argument("--cg-tol", type=float, default=1e-12, help="saddle: relative residual of the reduced system")
    ap.add_argument("--cg-max", type=int, default=500, help="saddle: conjugate-gradient iteration limit")
    ap.add_argument("--oracle-gamma", type=float, default=1e4,
                    help="saddle: gamma of the oracle's timed solves (its LU of H_g is not equilibrated and loses "
                         "accuracy at large gamma)")
    ap.add_argument("--tree-min-fronts", type=int, default=None,
                    help="levels with fewer fronts run in the persistent tree kernels (library default if unset)")
    return ap.parse_args(argv)


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
# generation nor gigabytes of inputs. The timed inputs are spread evenly over
# the whole mu schedule; the warm-up inputs come from another seed.
POOL_STEPS = 24
WARM_SEED = 7777


def pool_size(args):
    return args.warmup + min(args.steps, POOL_STEPS)


def at(args, i):
    """Input index of step i: the warm-up steps, then the timed steps cycling the pool."""
    n = pool_size(args)
    return i if i < n else args.warmup + (i - args.warmup) % (n - args.warmup)


def spread(count, n_sched):
    """`count` schedule indices spread evenly over 0 .. n_sched - 1 (both ends included)."""
    if count <= 1:
        return [0] * count
    return [int(round(t * (n_sched - 1) / (count - 1))) for t in range(count)]


def pool_plan(args, n_sched, seed):
    """(seed, schedule step) of every pool input: warm-up inputs first."""
    warm = [(seed + WARM_SEED, k) for k in spread(args.warmup, n_sched)]
    timed = [(seed, k) for k in spread(min(args.steps, POOL_STEPS), n_sched)]
    return warm + timed


def inputs(pat, mus, plan, slack_range=None):
    """Values and right-hand sides of the inputs (seed, k) of `plan`;
    slack_range: keep the inequality slacks' term in the (2,2) block."""
    vals, rhs = [], []
    for sd, k in plan:
        vals.append(pat.values(pat.point(sd, k, mus[k], slack_range=slack_range)))
        rhs.append(pat.rhs(sd, k))
    return vals, rhs


def rel_resid2(pat, vals, rhs, xs):
    """||b - K x||_2 / ||b||_2 of each result, on the host (scipy product)."""
    out = []
    for v, b, x in zip(vals, rhs, xs):
        r = b - pat.to_scipy(v) @ x
        out.append(float(np.linalg.norm(r) / np.linalg.norm(b)))
    return out


def summary(values):
    return {"max": float(max(values)), "median": float(np.median(values)), "per_result": [float(v) for v in values]}


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
    """Minimal traffic of each phase per refactor / solve / residual, from the
    factor sizes: refactor = nnz(K) (value + scatter index) + nnz(L+U) (factor
    value written + pattern index read) + the scaling vector; solve =
    nnz(L+U) (value + index) + four vectors; residual = nnz(K) (value + index)
    + three vectors."""
    nlu = plan["nnz_lu"]
    return {
        "refactor": nnz * (8 + 4) + nlu * (wbytes + 4) + n * 8,
        "solve": nlu * (wbytes + 4) + 4 * n * wbytes,
        "spmv": nnz * (8 + 4) + 3 * n * 8,
    }


def tree_factor_bytes(plan, wbytes):
    """The refactorization bytes above restricted to the fronts of the tree
    part (what tree_factor_kernel factors): its entries of K, its structural
    entries of L + U and its pivots' scaling factors."""
    return plan["tree_nnz_k"] * (8 + 4) + plan["tree_nnz_lu"] * (wbytes + 4) + plan["tree_pivots"] * 8


# DRAM bytes (read + write) of the dominant kernel per unit of the roofline
# (for tree_factor_kernel: its launches of one refactorization) from one ncu
# capture of the same command (profiles/), keyed by (kernel, workload,
# precision, tree levels); an entry is removed whenever the kernel changes.
MEASURED_TRAFFIC = {
    ("tree_factor_kernel", "eastern70k", "fp32", 73): 41074944,
}

PHASE_OF = {
    "front_warp_kernel": "refactor", "front_leaf_kernel": "refactor", "front_cta_kernel": "refactor",
    "front_panel_kernel": "refactor",
    "schur_tile_kernel": "refactor", "ruiz_kernel": "refactor", "scale_kernel": "refactor",
    "solve_fwd_kernel": "solve", "solve_bwd_kernel": "solve", "solve_pre_kernel": "solve",
    "solve_post_kernel": "solve", "spmv_resid_kernel": "spmv", "tree_factor_kernel": "refactor",
    "tree_fwd_kernel": "solve", "tree_bwd_kernel": "solve", "jacobi_kernels": "solve",
}


def roofline_of(stats, nprof, plan, ab, wbytes, workload_name, precision):
    """Roofline of the dominant kernel of a profiling pass over `nprof` steps."""
    if not stats:
        return None
    phase_ms = {}
    for name, (cnt, kms) in stats.items():
        ph = PHASE_OF.get(name)
        if ph:
            phase_ms[ph] = phase_ms.get(ph, 0.0) + kms
    dom = max(stats.items(), key=lambda kv: kv[1][1])[0]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    ph = PHASE_OF.get(dom, "refactor")
    if dom == "tree_factor_kernel":
        # its launches (one or two: wide levels, then the narrow top) per refactorization
        n_units = nprof
        bytes_unit = tree_factor_bytes(plan, wbytes)
        kms = stats[dom][1] / max(1, n_units)
        per_unit = "refactorization of the tree part (one or two launches)"
    else:
        n_units = nprof if ph == "refactor" else stats.get(
            "solve_post_kernel" if ph == "solve" else "spmv_resid_kernel", (0, 0.0))[0]
        bytes_unit = ab[ph]
        kms = phase_ms[ph] / max(1, n_units)
        per_unit = "%s phase" % ph
    achieved = bytes_unit / (kms / 1000.0) / 1e9
    key = (dom, workload_name, precision, plan["tree_levels"])
    traffic = MEASURED_TRAFFIC.get(key)
    ref_ms = phase_ms.get("refactor", 0.0) / nprof
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": dom, "peak_source": peak_src, "per_unit": per_unit,
            "algorithmic_bytes_per_unit": bytes_unit, "units_profiled": n_units, "ms_per_unit": kms,
            "launches_per_unit": stats[dom][0] / max(1, n_units),
            "multifrontal_traffic_model_bytes": plan["tree_bytes"] if dom == "tree_factor_kernel" else None,
            "refactor_phase": {"algorithmic_bytes": ab["refactor"], "ms": ref_ms,
                               "achieved_gbs": ab["refactor"] / (max(ref_ms, 1e-9) / 1000.0) / 1e9}}


# ----------------------------------------------------------------- reference arm

def cpu_run(pat, vals, rhs, tol, budget_s, max_steps, an=None):
    """The oracle as it stands, single thread: analysis untimed (or given),
    then per step Ruiz + LU with frozen pivots + FGMRES to tol, until the
    budget is used. Returns the step times, the backward errors and the
    solutions (inputs 0, 1, ... in order)."""
    import oracle as O
    if an is None:
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
    """The oracle, as it stands, on the host cores: the same workload, inputs,
    tolerance and metric as the native arm. Its timed steps cycle the same
    input pool and stop once --ref-seconds are used (at least 3 steps), so
    that the run stays within minutes."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        raise SystemExit("--impl reference times the oracle on a single-system workload")
    import oracle as O
    w, pat, mus = workload(args.workload, args.seed)
    plan = pool_plan(args, len(mus), args.seed)
    vals_p, rhs_p = inputs(pat, mus, plan, args.slack_range)
    an = O.analyze(pat.rowptr, pat.colidx, vals_p[0])
    for i in range(args.warmup):
        cpu_run(pat, [vals_p[i]], [rhs_p[i]], args.tol, 1e9, 1, an)
    t, oms = [], []
    t_all = time.perf_counter()
    for step in range(args.steps):
        i = at(args, args.warmup + step)
        ts, om, _ = cpu_run(pat, [vals_p[i]], [rhs_p[i]], args.tol, 1e9, 1, an)
        t += ts
        oms += om
        if time.perf_counter() - t_all > args.ref_seconds and len(t) >= 3:
            break
    ms = 1000.0 * sum(t) / len(t)
    value = 1000.0 / ms
    sample = ("%d of the %d requested steps of %s (one refactor + solve + FGMRES each, the input pool cycled "
              "over the mu schedule; timed steps end once %.0f s are used), oracle analysis untimed"
              % (len(t), args.steps, args.workload, args.ref_seconds))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": len(t), "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64", "tol": args.tol,
                   "slack_range": args.slack_range},
        "p50_ms": 1000 * float(np.percentile(t, 50)), "p99_ms": 1000 * float(np.percentile(t, 99)),
        "omega_max": float(max(oms)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    plan_in = pool_plan(args, len(mus), seed)
    n_in = len(plan_in)
    vals_h, rhs_h = inputs(pat, mus, plan_in, args.slack_range)
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

    def timed_run(solver, vals_, rhs_, xs_, tol, steps):
        """W warm-up steps, then `steps` timed steps cycling the pool; per-step
        CUDA events on the launching stream, L2 flushed before each step."""
        stream = torch.cuda.current_stream()
        for i in range(args.warmup):
            solver.refactor_refine(vals_[i], rhs_[i], out=xs_[i], tol=tol, raise_on_noconv=False)
        l0 = solver.info().launches
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        oms, iters = [], []
        barrier()
        gc.disable()                      # no collector pause inside the timed steps
        for t in range(steps):
            i = args.warmup + (t % (len(vals_) - args.warmup))
            flush.zero_()
            ev0[t].record(stream)
            _, info = solver.refactor_refine(vals_[i], rhs_[i], out=xs_[i], tol=tol, raise_on_noconv=False)
            ev1[t].record(stream)
            oms.append(info.backward_err)
            iters.append(info.iters)
        gc.enable()
        barrier()
        launches = solver.info().launches - l0
        ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        return ms, oms, iters, launches

    def arm_record(prec, ms, oms, iters, tol):
        return {"precision": PREC_NAME[prec], "value": 1000.0 * len(ms) / sum(ms), "ms_per_step": sum(ms) / len(ms),
                "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                "omega_max": float(max(oms)), "converged_steps": int(sum(1 for o in oms if o <= tol)),
                "fgmres_iters_mean": float(np.mean(iters)), "fgmres_iters_max": int(max(iters))}

    lib_opts = {"graphs": not args.no_graphs}
    if args.max_pivots:
        lib_opts["max_pivots"] = args.max_pivots
    if args.tree_min_fronts is not None:
        lib_opts["tree_min_fronts"] = args.tree_min_fronts
    if args.precond != "lu":
        lib_opts["precond"] = args.precond
        lib_opts["jacobi_sweeps"] = args.sweeps
    other_prec = "fp64" if args.precision == "fp32" else "fp32"
    main = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=args.precision, **lib_opts)
    plan = main.plan()
    sampler = ClockSampler(dev.index)
    sampler.start()
    ms, oms, iters, launches = timed_run(main, vals, rhs, xs, args.tol, args.steps)
    clocks = sampler.stop()
    results = {PREC_NAME[args.precision]: [x.cpu().numpy() for x in xs[args.warmup:]]}   # one per timed input
    total_ms = sum(ms)
    if world > 1:
        total_ms = reduce_max(total_ms, device=dev)
    value = aggregate_rate(world, args.steps, total_ms)
    main_rec = arm_record(args.precision, ms, oms, iters, args.tol)

    # the other precision on the same matrices (the graded comparison: FP32 LU + FP64 FGMRES vs plain FP64)
    other = None
    if not args.no_compare:
        so = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=other_prec, **lib_opts)
        mso, omso, ito, _ = timed_run(so, vals, rhs, xs, args.tol, args.steps)
        results[PREC_NAME[other_prec]] = [x.cpu().numpy() for x in xs[args.warmup:]]
        other = arm_record(other_prec, mso, omso, ito, args.tol)
        so.close()

    # end to end through the C ABI with host buffers (copies inside the timed call)
    hv = [torch.from_numpy(v).pin_memory() for v in vals_h]
    hb = [torch.from_numpy(b).pin_memory() for b in rhs_h]
    hx = torch.empty(pat.n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    # the host-buffer path's own warm-up: at least 50 calls (~0.1 s), so that
    # the host side runs at its working clock when the timed calls start
    for t in range(max(args.warmup, 50)):
        i = at(args, t)
        main.step_host(hv[i].numpy(), hb[i].numpy(), tol=args.tol, out=hx.numpy(), raise_on_noconv=False)
    barrier()
    gc.disable()
    for t in range(args.steps):
        i = at(args, args.warmup + t)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        main.step_host(hv[i].numpy(), hb[i].numpy(), tol=args.tol, out=hx.numpy(), raise_on_noconv=False)
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    gc.enable()
    barrier()
    p50 = float(np.percentile(e2e_ms, 50))
    slow = [t for t, v in enumerate(e2e_ms) if v > 1.5 * p50]
    e2e = {"value": 1000.0 * len(e2e_ms) / sum(e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(8 * (pat.nnz + pat.n)), "d2h_bytes_per_step": int(8 * pat.n),
           "p50_ms": p50, "p99_ms": float(np.percentile(e2e_ms, 99)),
           "slow_steps": {"count": len(slow), "threshold_ms": 1.5 * p50, "first": slow[:20],
                          "mean_ms": float(np.mean([e2e_ms[t] for t in slow])) if slow else None}}

    # per-kernel timing pass (profiling mode, separate from the timed run)
    main.set_profiling(True)
    main.kernel_stats()
    nprof = min(3, args.steps)
    for t in range(nprof):
        i = at(args, args.warmup + t)
        main.refactor_refine(vals[i], rhs[i], out=xs[i], tol=args.tol, raise_on_noconv=False)
    stats = main.kernel_stats()
    main.set_profiling(False)
    wbytes = 8 if args.precision == "fp64" else 4
    ab = algorithmic_bytes(plan, pat.n, pat.nnz, wbytes)
    roofline = roofline_of(stats, nprof, plan, ab, wbytes, args.workload, args.precision)

    # systems that determine x (the slacks' term kept in the (2,2) block):
    # both precisions refined to a tolerance at which FP32 factors reach the
    # oracle's x; what that costs in iterations and rate
    det = None
    det_h = None
    if not args.no_determined and args.slack_range is None and args.precond == "lu":
        sr = (1e-2, 1e2)
        dplan = [(seed, k) for k in spread(args.warmup + 8, len(mus))]
        dv_h, db_h = inputs(pat, mus, dplan, sr)
        det_h = (dv_h[args.warmup:], db_h[args.warmup:])
        dv = [torch.from_numpy(v).to(dev) for v in dv_h]
        db = [torch.from_numpy(b).to(dev) for b in db_h]
        dx = [torch.empty_like(b) for b in db]
        dsteps = min(args.steps, 8)
        det = {"slack_range": list(sr), "tol": args.det_tol, "inputs": len(dv) - args.warmup, "steps": dsteps}
        res_det = {}
        for prec, sol in ((args.precision, main), (other_prec, None)):
            if prec != args.precision and args.no_compare:
                continue
            s = sol or K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=prec, **lib_opts)
            dms, doms, dits, _ = timed_run(s, dv, db, dx, args.det_tol, dsteps)
            det[PREC_NAME[prec]] = arm_record(prec, dms, doms, dits, args.det_tol)
            res_det[PREC_NAME[prec]] = [x.cpu().numpy() for x in dx[args.warmup:]]
            if sol is None:
                s.close()
        det_res = res_det
    else:
        det_res = None

    cpu = None
    accuracy = None
    resid2 = None
    if rank == 0:
        tv, tb = vals_h[args.warmup:], rhs_h[args.warmup:]
        resid2 = {name: summary(rel_resid2(pat, tv, tb, r)) for name, r in results.items()}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        an = O.analyze(pat.rowptr, pat.colidx, vals_h[args.warmup])
        times, coms, xo = cpu_run(pat, vals_h[args.warmup:], rhs_h[args.warmup:], args.tol, args.cpu_seconds,
                                  n_in, an)
        cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d of the %d timed inputs of %s (spread over the mu schedule; oracle analysis untimed), "
                         "single thread" % (len(times), n_in - args.warmup, args.workload),
               "omega_max": float(max(coms))}
        try:
            accuracy = error_vs_oracle(xo, results)
        except Exception as e:                     # reported in the line, never fatal to it
            accuracy = {"error": repr(e)}
        if det is not None:
            try:
                nd = 2
                _, dom_, xdo = cpu_run(pat, det_h[0][:nd], det_h[1][:nd], 1e-15, 1e9, nd, an)
                det["oracle_omega"] = [float(o) for o in dom_]
                det["error_vs_oracle"] = error_vs_oracle(xdo, det_res)
            except Exception as e:
                det["error_vs_oracle"] = {"error": repr(e)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "buses": w["n_bus"], "branches": w["n_branch"],
                       "generators": w["n_gen"], "n": pat.n, "nnz": pat.nnz, "precision": PREC_NAME[args.precision],
                       "tol": args.tol, "mu": [w["mu0"], w["mu1"]], "slack_range": args.slack_range,
                       "inputs": "%d timed inputs spread over the %d-step mu schedule (steps %s), cycled; "
                                 "%d warm-up inputs" % (n_in - args.warmup, len(mus),
                                                        [k for _, k in plan_in[args.warmup:]], args.warmup),
                       "l2": "flushed between timed steps (%d MB write)" % (flush.numel() >> 20),
                       "fronts": plan["n_fronts"], "levels": plan["n_levels"], "nnz_lu": plan["nnz_lu"],
                       "tree_levels": plan["tree_levels"], "tree_units": plan["tree_units"]},
            "p50_ms": main_rec["p50_ms"], "p99_ms": main_rec["p99_ms"],
            "omega_max": main_rec["omega_max"], "fgmres_iters_mean": main_rec["fgmres_iters_mean"],
            "converged_steps": main_rec["converged_steps"],
            "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": int(launches), "kernel_ms_per_step": {k: v[1] / nprof for k, v in stats.items()},
            "library_options": lib_opts,
            "fp64_arm" if other_prec == "fp64" else "fp32_arm": other,
            "rel_resid2": resid2, "error_vs_oracle": accuracy, "determined_x": det,
        }
        if other is not None:
            a32, a64 = (main_rec, other) if args.precision == "fp32" else (other, main_rec)
            line["fp32_vs_fp64"] = {"solves_per_s_ratio": a32["value"] / a64["value"],
                                    "p50_ratio": a32["p50_ms"] / a64["p50_ms"],
                                    "p99_ratio": a32["p99_ms"] / a64["p99_ms"]}
        print(json.dumps(line), flush=True)
    main.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ oracle on every host core

def _oracle_worker(task):
    """One host core: the oracle as it stands on systems of one kind until its
    time budget is used (analysis untimed). task = (n_bus, n_branch, n_gen,
    grid seed, [(point seed, mu)], budget_s); returns (solves, seconds)."""
    import oracle as O
    n_bus, n_branch, n_gen, gseed, points, budget = task
    pat = KKTPattern(make_grid(gseed, n_bus, n_branch, n_gen))
    an = None
    done, busy = 0, 0.0
    for psd, mu in points:
        v = pat.values(pat.point(psd, 0, mu))
        b = pat.rhs(psd, 0)
        if an is None:
            an = O.analyze(pat.rowptr, pat.colidx, v)
        t0 = time.perf_counter()
        lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an)
        O.fgmres(pat.rowptr, pat.colidx, v, lu, d, b, 30, 10, 1e-10)
        busy += time.perf_counter() - t0
        done += 1
        if busy > budget and done >= 1:
            break
    return done, busy


def oracle_pool(tasks):
    """Run the oracle tasks on every host core, one process per core, started
    with spawn (never forked from a process that has used the GPU)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(cores, len(tasks))) as pool:
        out = pool.map(_oracle_worker, tasks)
    return out, cores


# ------------------------------------------------------------ batched (many instances)

def run_batch(args):
    """64 instances of one 2,000-bus pattern and 16 of one 10,000-bus pattern,
    values and right-hand sides from a different seed per instance; the two
    batches refactor concurrently, each one launch per level for all its
    instances; the schedule of each is chosen by the autotuner. The value is
    FP32 factors + FP64 refinement; fp64_arm repeats the same steps with FP64
    factors."""
    import torch
    import paper_2302_08656_gb300 as K
    from paper_2302_08656_gb300 import autotune

    dev = torch.device("cuda", 0)
    groups = [("batch2k", 64), ("batch10k", 16)]
    n_in = pool_size(args)
    pats, vals, rhs, mus_of = [], [], [], []
    for name, count in groups:
        w = WORKLOADS[name]
        pat = KKTPattern(make_grid(args.seed, w["n_bus"], w["n_branch"], w["n_gen"]))
        mus = mu_schedule(w["mu0"], w["mu1"], w["steps"])
        ks = spread(n_in, len(mus))
        v_steps, b_steps = [], []
        for k in ks:
            v_steps.append(torch.from_numpy(np.concatenate(
                [pat.values(pat.point(args.seed * 1000 + i, k, mus[k])) for i in range(count)])).to(dev))
            b_steps.append(torch.from_numpy(np.concatenate(
                [pat.rhs(args.seed * 1000 + i, k) for i in range(count)])).to(dev))
        pats.append(pat)
        vals.append(v_steps)
        rhs.append(b_steps)
        mus_of.append(mus)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def arm(prec, use_group):
        ctxs, outs, omegas, tune_info = [], [], [], {}
        for (name, count), pat, v_steps, b_steps in zip(groups, pats, vals, rhs):
            best, times = autotune.tune(pat.rowptr, pat.colidx, pat.n_primal, v_steps[0], b_steps[0],
                                        precision=prec, count=count)
            tune_info[name] = {"count": count, "n": pat.n, "nnz": pat.nnz, "chosen": best, "ms_by_schedule": times}
            ctxs.append(K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=count, precision=prec, **best))
            outs.append(torch.empty_like(b_steps[0]))
            omegas.append(torch.empty(count, dtype=torch.float64).pin_memory())
        group = K.KKTGroup(ctxs) if use_group else None

        def step(t):
            t = at(args, t)
            if group is not None:
                group.refactor([vals[g][t] for g in range(len(ctxs))])
            else:
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
        # profiling pass: per-kernel time of every context, for the roofline
        stats_all = {}
        for s in ctxs:
            s.set_profiling(True)
            s.kernel_stats()
        nprof = min(3, args.steps)
        for t in range(nprof):
            step(args.warmup + t)
        plans = [s.plan() for s in ctxs]
        per_ctx = []
        for s in ctxs:
            st = s.kernel_stats()
            per_ctx.append(st)
            s.set_profiling(False)
            for k, (c, kms) in st.items():
                a = stats_all.setdefault(k, [0, 0.0])
                a[0] += c
                a[1] += kms
        if group is not None:
            group.close()
        for s in ctxs:
            s.close()
        per_step = sum(c for _, c in groups)
        rec = {"precision": PREC_NAME[prec], "value": per_step * len(ms) / (sum(ms) / 1000.0),
               "ms_per_step": float(np.mean(ms)), "p50_ms": float(np.percentile(ms, 50)),
               "p99_ms": float(np.percentile(ms, 99)), "omega_max": float(max(oms)),
               "fgmres_iters_total": int(sum(its)), "gpu_launches": int(launches),
               "launches_per_step": launches / max(1, args.steps), "clocks": clocks, "groups": tune_info,
               "refactorization": "forked streams" if group is None else
               "one group: level parts on forked streams, the tops of both trees in one launch"}
        return rec, stats_all, per_ctx, plans, nprof

    main_prec = "fp32" if args.precision == "fp64" else args.precision   # this configuration runs FP32 LU
    main, stats, per_ctx, plans, nprof = arm(main_prec, args.group)
    other = None if args.no_compare else arm("fp64" if main_prec == "fp32" else "fp32", args.group)[0]
    # the other refactorization schedule on the same steps: forked streams
    # (each pattern's whole refactorization on its own stream) against one
    # group (level parts forked, the tops of both trees in one launch)
    alt = None
    if not args.no_compare:
        a = arm(main_prec, not args.group)[0]
        alt = {k: a[k] for k in ("refactorization", "value", "p50_ms", "p99_ms", "launches_per_step", "omega_max")}

    # roofline of the dominant kernel over both patterns' contexts: the
    # algorithmic bytes of every instance it processed per step
    roofline = None
    if stats:
        wb = 4 if main_prec == "fp32" else 8
        dom = max(stats.items(), key=lambda kv: kv[1][1])[0]
        ph = PHASE_OF.get(dom, "refactor")
        byts = 0
        for (name, count), pat, plan in zip(groups, pats, plans):
            ab = algorithmic_bytes(plan, pat.n, pat.nnz, wb)
            byts += count * (tree_factor_bytes(plan, wb) if dom == "tree_factor_kernel" else ab[ph])
        if dom == "tree_factor_kernel":
            kms, what = stats[dom][1] / nprof, "the tree part of every instance's refactorization in one batch step"
        else:
            # a level kernel takes only some fronts of each level: the unit is
            # then the whole phase it belongs to (its kernels' time summed)
            kms = sum(v[1] for k, v in stats.items() if PHASE_OF.get(k) == ph) / nprof
            what = "the %s phase of one batch step (all 80 instances), whose largest kernel is %s" % (ph, dom)
        hbm, src = _hbm_peak()
        achieved = byts / (kms / 1000.0) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "traffic": None, "kernel": dom, "peak_source": src, "per_unit": what,
                    "algorithmic_bytes_per_unit": byts, "ms_per_unit": kms,
                    "launches_per_unit": stats[dom][0] / nprof,
                    "kernel_ms_per_step": {k: v[1] / nprof for k, v in stats.items()}}

    cpu = None
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        tasks = []
        for i in range(cores):
            name, count = groups[0] if i < max(1, (cores * 3) // 4) else groups[1]
            w = WORKLOADS[name]
            pts = [(args.seed * 1000 + j, float(mus_of[0][spread(8, len(mus_of[0]))[j % 8]])) for j in range(i, i + 40)]
            tasks.append((w["n_bus"], w["n_branch"], w["n_gen"], args.seed, pts, args.cpu_seconds))
        out, used = oracle_pool(tasks)
        t_of = {}
        for (name, _), res in zip([groups[0] if i < max(1, (cores * 3) // 4) else groups[1] for i in range(cores)], out):
            a = t_of.setdefault(name, [0, 0.0])
            a[0] += res[0]
            a[1] += res[1]
        per_inst = {name: t_of[name][1] / max(1, t_of[name][0]) for name in t_of}
        core_s_per_step = sum(count * per_inst.get(name, float("nan")) for name, count in groups)
        steps_per_s = used / core_s_per_step
        cpu = {"value": steps_per_s * sum(c for _, c in groups), "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": "%s; one process per core (spawn), each timing refactor + solve + FGMRES of its own "
                         "instances for %.0f s after an untimed analysis; batch rate = cores / (64 t_2k + 16 t_10k) "
                         "x 80" % (", ".join("%s: %d solves, %.3f s each" % (k, t_of[k][0], per_inst[k])
                                            for k in sorted(t_of)), args.cpu_seconds)}

    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if main_prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "batch", "groups": main["groups"], "precision": PREC_NAME[main_prec], "tol": args.tol,
                   "l2": "flushed between timed steps (512 MB write)",
                   "inputs": "%d inputs per instance spread over the 50-step mu schedule, cycled" % (n_in - args.warmup),
                   "note": "one step = one refactor + solve (+ refinement if needed) of all 80 instances"},
        "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "omega_max": main["omega_max"],
        "fgmres_iters_total": main["fgmres_iters_total"], "gpu_launches": main["gpu_launches"],
        "launches_per_step": main["launches_per_step"], "refactorization": main["refactorization"],
        "other_refactorization_schedule": alt,
        "clocks": main["clocks"], "roofline": roofline, "cpu_baseline": cpu,
        "fp64_arm" if main_prec == "fp32" else "fp32_arm": other,
    }
    if other is not None:
        line["fp32_vs_fp64"] = {"solves_per_s_ratio": main["value"] / other["value"],
                                "p99_ratio": main["p99_ms"] / other["p99_ms"]}
    print(json.dumps(line), flush=True)


def _hbm_peak():
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
    except Exception:
        hbm = None
    return (hbm, "measured") if hbm else (6800.0, "fallback")


# ------------------------------------------------------------------- serving

def run_serving(args):
    """Sessions with grid sizes log-uniform over 500..25,000 buses, 30..80 IPM
    iterations each, Poisson arrivals at `rate` requests/s in total; factors
    resident per session; HBM budget for admission. The value is FP32 factors
    + FP64 refinement to tol; fp64_arm replays the same sessions and arrivals
    with FP64 factors; budget_binding replays the FP32 run under a budget that
    admits only part of the sessions at a time. Each session cycles two
    pre-generated value sets (to bound input generation time)."""
    import torch
    from paper_2302_08656_gb300.serve import (GpuBackend, Server, SessionSpec, estimate_bytes,
                                              log_uniform_sizes, poisson_arrivals)

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(args.seed)
    sizes = log_uniform_sizes(rng, args.sessions, 500, 25_000)
    iters = rng.integers(30, 81, size=args.sessions)
    arrivals = poisson_arrivals(rng, args.rate, list(iters))
    specs = []
    t0 = time.perf_counter()
    for sid, B in enumerate(sizes):
        grid = make_grid(args.seed * 7919 + sid, B, int(round(1.28 * B)), max(1, int(round(0.2 * B))))
        pat = KKTPattern(grid)
        vs = [torch.from_numpy(pat.values(pat.point(sid, k, 10.0 ** -(1 + 4 * k)))).to(dev) for k in range(2)]
        bs = [torch.from_numpy(pat.rhs(sid, k)).to(dev) for k in range(2)]
        specs.append((sid, pat, vs, bs))
    gen_s = time.perf_counter() - t0

    def serve(prec, budget_gb):
        sessions = [SessionSpec(sid, pat.rowptr, pat.colidx, pat.n_primal, arrivals[sid],
                                (lambda v, b: (lambda k: (v[k % 2], b[k % 2])))(vs, bs),
                                est_bytes=estimate_bytes(pat.nnz, prec))
                    for sid, pat, vs, bs in specs]
        backend = GpuBackend(precision=prec, tol=args.tol, streams=16)
        server = Server(backend, budget_bytes=int(budget_gb * (1 << 30)), max_inflight=16, analysis_workers=12)
        sampler = ClockSampler(0)
        sampler.start()
        rep = server.run(sessions)
        clocks = sampler.stop()
        return {"precision": PREC_NAME[prec], "budget_gb": budget_gb, "value": rep.solves_per_s,
                "completed": rep.completed, "wall_s": rep.wall_s,
                "p50_ms": rep.percentile(50), "p99_ms": rep.percentile(99),
                "p50_ms_steady": rep.percentile(50, steady=True), "p99_ms_steady": rep.percentile(99, steady=True),
                "omega_max": float(max(rep.omegas)) if rep.omegas else None, "refined": rep.refined,
                "max_sessions_resident": rep.max_sessions, "max_device_bytes": rep.max_bytes,
                "admission_waits": rep.admission_waits, "failed": [[sid, k, err] for sid, k, err in rep.failed],
                "clocks": clocks}

    main = serve("fp32", args.budget_gb)
    other = None if args.no_compare else serve("fp64", args.budget_gb)
    # a budget that admits only part of the sessions at a time: about a tenth of their estimated total
    total_est = sum(estimate_bytes(pat.nnz, "fp32") for _, pat, _, _ in specs)
    small_gb = max(1.0, round(total_est / 10 / (1 << 30), 1))
    binding = None if args.no_compare else serve("fp32", small_gb)

    cpu = None
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        # one session per core, taken evenly over the size order (so the sample spans the log-uniform mix)
        order = np.argsort(sizes)
        pick = [int(order[int(round(i * (len(order) - 1) / max(1, cores - 1)))]) for i in range(cores)]
        tasks = []
        for sid in pick:
            B = sizes[sid]
            tasks.append((B, int(round(1.28 * B)), max(1, int(round(0.2 * B))), args.seed * 7919 + sid,
                          [(sid, 10.0 ** -(1 + 4 * (k % 2))) for k in range(40)], args.cpu_seconds))
        out, used = oracle_pool(tasks)
        # mean oracle time per request over the sessions, weighted by their request counts
        t_req = np.array([res[1] / max(1, res[0]) for res in out])
        wts = np.array([iters[sid] for sid in pick], dtype=np.float64)
        mean_t = float(np.sum(t_req * wts) / np.sum(wts))
        cpu = {"value": used / mean_t, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": "%d sessions spread over the size order (%d..%d buses), one process per core (spawn), "
                         "each timing its requests for %.0f s after an untimed analysis; rate = cores / mean time "
                         "per request (weighted by the sessions' request counts)"
                         % (len(pick), min(sizes[s] for s in pick), max(sizes[s] for s in pick), args.cpu_seconds)}

    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": main["completed"],
        "warmup": 0, "ms_per_step": 1000.0 * main["wall_s"] / max(1, main["completed"]), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving", "sessions": args.sessions, "buses": [500, 25000], "iterations": [30, 80],
                   "rate_per_s": args.rate, "budget_gb": args.budget_gb, "precision": "fp32_ir", "tol": args.tol,
                   "input_generation_s": gen_s},
        "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"],
        "p50_ms_steady": main["p50_ms_steady"], "p99_ms_steady": main["p99_ms_steady"],
        "omega_max": main["omega_max"], "refined": main["refined"],
        "max_sessions_resident": main["max_sessions_resident"], "max_device_bytes": main["max_device_bytes"],
        "admission_waits": main["admission_waits"], "wall_s": main["wall_s"], "failed": main["failed"],
        "clocks": main["clocks"], "fp64_arm": other, "budget_binding": binding, "cpu_baseline": cpu,
    }
    if other is not None:
        line["fp32_vs_fp64"] = {"solves_per_s_ratio": main["value"] / other["value"],
                                "p99_steady_ratio": main["p99_ms_steady"] / other["p99_ms_steady"]}
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


def run_ipm_loop(args):
    """The interior-point loop around the solver (Sec. II): one step = one whole
    ACOPF solve from the flat start on the GPU (model evaluation, a refactor +
    refine per Newton iteration, the vector steps), FP64 factors. value =
    Newton iterations per second (each is one K refactor + solve); the oracle's
    loop on the same instance is timed on one host core and its optimum is
    compared with the GPU's."""
    import torch
    import paper_2302_08656_gb300 as K
    from kktgen import flat_start, opf_data

    dev = torch.device("cuda", 0)
    w = WORKLOADS[args.workload]
    grid = make_grid(args.seed, w["n_bus"], w["n_branch"], w["n_gen"])
    data = opf_data(grid, args.seed)
    m = K.KKTModel.from_grid(grid)
    m.set_limits(data)
    prec = args.precision if args.precision == "fp64" else "fp64"      # FP32 factors do not converge here
    s = K.KKTSolver(m.rowptr, m.colidx, m.n_primal, precision=prec)
    x0h = flat_start(grid, data)
    x = torch.empty(m.n_primal, dtype=torch.float64, device=dev)
    runs = min(args.steps, 20)
    for _ in range(args.warmup):
        x.copy_(torch.from_numpy(x0h))
        m.ipm_solve(s, x)
    l0 = s.info().launches
    stream = torch.cuda.current_stream()
    ms, its, infos = [], [], []
    sampler = ClockSampler(0)
    sampler.start()
    for _ in range(runs):
        x.copy_(torch.from_numpy(x0h))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, lam, info = m.ipm_solve(s, x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(info.iters)
        infos.append(info)
    clocks = sampler.stop()
    launches = s.info().launches - l0
    xg = x.cpu().numpy()
    last = infos[-1]
    cpu, agree = None, None
    if not args.no_cpu_baseline:
        from oracle import ipm as OI
        pat = KKTPattern(grid)
        t0 = time.perf_counter()
        ref = OI.solve(pat, data, x0h)
        t_ora = time.perf_counter() - t0
        cpu = {"value": ref.iters / t_ora, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "one whole solve of the same instance by the oracle's loop (scipy sparse solves), "
                         "%d Newton iterations in %.1f s" % (ref.iters, t_ora)}
        B = grid.n_bus
        th, tr = xg[B:2 * B], ref.x[B:2 * B]
        agree = {"oracle_iterations": ref.iters, "oracle_objective": ref.objective,
                 "objective_rel_diff": abs(last.objective - ref.objective) / abs(ref.objective),
                 "max_abs_diff_V": float(np.max(np.abs(xg[:B] - ref.x[:B]))),
                 "max_abs_diff_theta": float(np.max(np.abs(th - tr))),
                 "max_abs_diff_dispatch": float(np.max(np.abs(xg[2 * B:] - ref.x[2 * B:])))}
    total_it = int(sum(its))
    line = {
        "metric": METRIC, "value": 1000.0 * total_it / sum(ms), "unit": UNIT, "n_gpus": 1, "steps": runs,
        "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + " interior-point loop", "buses": w["n_bus"], "n": m.n, "nnz": m.nnz,
                   "precision": prec, "loads_limits": "kktgen.opf_data (seeded)", "start": "flat",
                   "note": "one step = one whole ACOPF solve; value = Newton iterations (K refactor + solve) per s"},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "newton_iterations_per_solve": its[-1], "objective": last.objective, "final_error": last.err,
        "status": last.status, "fgmres_iters_per_solve": last.lin_iters, "newton_omega_max": last.lin_omega_max,
        "gpu_launches": int(launches), "clocks": clocks, "cpu_baseline": cpu, "oracle_agreement": agree,
    }
    print(json.dumps(line), flush=True)
    s.close()
    m.close()


def run_saddle(args):
    """The saddle-point specialised solve (Sec. V) on one workload: per step
    one kkt_hykkt_solve (H_g assembled and factored, conjugate gradients on
    the reduced operator, recovery), FP64 throughout; the direct path (FP32
    and FP64 refactor + refine) on the same systems beside it. value = solves
    per second of the saddle-point solve; the oracle's solve of the same
    method is timed on one host core over a bounded sample and its solutions
    compared with the device's."""
    import torch
    import paper_2302_08656_gb300 as K
    from oracle import hykkt

    dev = torch.device("cuda", 0)
    sr = tuple(args.slack_range) if args.slack_range is not None else (1e-2, 1e2)
    w, pat, mus = workload(args.workload, args.seed)
    plan_in = pool_plan(args, len(mus), args.seed)
    vals_h, rhs_h = inputs(pat, mus, plan_in, sr)
    vals = [torch.from_numpy(v).to(dev) for v in vals_h]
    rhs = [torch.from_numpy(b).to(dev) for b in rhs_h]
    xs = [torch.empty_like(b) for b in rhs]
    mE = 2 * pat.grid.n_bus
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    sp_ = K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, mE, gamma=args.gamma)
    analyze_s = time.perf_counter() - t0

    def solve(i):
        _, info = sp_.solve(vals[i], rhs[i], tol=args.cg_tol, max_iter=args.cg_max, out=xs[i],
                            raise_on_noconv=False)
        return info

    for i in range(args.warmup):
        solve(i)
    ms, its, oms, launches = [], [], [], 0
    sampler = ClockSampler(0)
    sampler.start()
    gc.disable()
    for t in range(args.steps):
        i = at(args, args.warmup + t)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = solve(i)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        its.append(info.cg_iters)
        oms.append(info.backward_err)
        launches += info.launches
    gc.enable()
    clocks = sampler.stop()
    res = [x.cpu().numpy() for x in xs[args.warmup:]]

    # per-kernel time of the factorization and solves of H_g (profiling pass)
    inner = sp_.inner()
    inner.set_profiling(True)
    inner.kernel_stats()
    nprof = min(3, args.steps)
    for t in range(nprof):
        solve(at(args, args.warmup + t))
    stats = inner.kernel_stats()
    inner.set_profiling(False)
    plan_g = inner.plan()
    roofline = roofline_of(stats, nprof, plan_g, algorithmic_bytes(plan_g, plan_g["n"], plan_g["nnz"], 8), 8,
                           args.workload + " H_g", "fp64")

    # the direct path on the same systems
    direct = {}
    for prec in (() if args.no_compare else ("fp32", "fp64")):
        s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=prec)
        for i in range(args.warmup):
            s.refactor_refine(vals[i], rhs[i], out=xs[i], tol=args.tol, raise_on_noconv=False)
        dms, dom = [], []
        for t in range(args.steps):
            i = at(args, args.warmup + t)
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, info = s.refactor_refine(vals[i], rhs[i], out=xs[i], tol=args.tol, raise_on_noconv=False)
            e1.record(stream)
            torch.cuda.synchronize()
            dms.append(e0.elapsed_time(e1))
            dom.append(info.backward_err)
        direct[PREC_NAME[prec]] = {"value": 1000.0 * len(dms) / sum(dms), "p50_ms": float(np.percentile(dms, 50)),
                                   "p99_ms": float(np.percentile(dms, 99)), "omega_max": float(max(dom))}
        s.close()

    cpu, agree = None, None
    if not args.no_cpu_baseline:
        times, errs, oom = [], [], []
        t_all = time.perf_counter()
        for k, (v, b) in enumerate(zip(vals_h[args.warmup:], rhs_h[args.warmup:])):
            Ks = pat.to_scipy(v)
            t1 = time.perf_counter()
            o = hykkt.solve(Ks, pat.n_primal, mE, b, args.oracle_gamma, tol=args.cg_tol, max_iter=100 * args.cg_max)
            times.append(time.perf_counter() - t1)
            oom.append(o.omega)
            errs.append(float(np.max(np.abs(res[k] - o.z)) / np.max(np.abs(o.z))))
            if time.perf_counter() - t_all > args.cpu_seconds:
                break
        cpu = {"value": len(times) / sum(times), "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": "%d of the %d timed inputs of %s, the oracle's saddle-point solve (scipy splu of H_g, "
                         "textbook CG) at gamma %g, block extraction untimed" % (len(times), len(res), args.workload,
                                                                                 args.oracle_gamma)}
        agree = {"inputs": len(times), "oracle_omega_max": float(max(oom)),
                 "max_rel_diff_z": float(max(errs)),
                 "note": "the graded systems do not determine z entrywise; omega of both is the check"}
    line = {
        "metric": "saddle-point specialised solves/s at backward error <= %g" % args.tol,
        "value": 1000.0 * len(ms) / sum(ms), "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + " saddle-point solve", "buses": w["n_bus"], "n": pat.n,
                   "nnz": pat.nnz, "n_primal": pat.n_primal, "m_eq": mE, "gamma": args.gamma,
                   "cg_tol": args.cg_tol, "slack_range": list(sr), "n_hg": plan_g["n"], "nnz_hg": plan_g["nnz"],
                   "nnz_lu_hg": plan_g["nnz_lu"],
                   "l2": "flushed between timed steps (512 MB write)", "analyze_s": analyze_s},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "cg_iters_mean": float(np.mean(its)), "cg_iters_max": int(max(its)), "omega_max": float(max(oms)),
        "converged_steps": int(sum(1 for o in oms if o <= args.tol)),
        "direct_path": direct, "gpu_launches": int(launches), "clocks": clocks, "cpu_baseline": cpu,
        "roofline": roofline, "inner_kernel_ms_per_call": {k: v[1] / nprof for k, v in stats.items()},
        "oracle_agreement": agree,
    }
    print(json.dumps(line), flush=True)
    sp_.close()


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
    elif args.ipm_loop:
        run_ipm_loop(args)
    elif args.saddle:
        run_saddle(args)
    elif args.assemble:
        run_ipm(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
