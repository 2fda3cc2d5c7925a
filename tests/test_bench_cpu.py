"""Host-side parts of bench.py on CPU: the oracle leg returns the solutions
that each GPU result's error is stated against, and error_vs_oracle states
that error per result."""
import os
import sys

import numpy as np
import pytest

sp = pytest.importorskip("scipy.sparse")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_leg_returns_solutions_that_meet_the_tolerance():
    w, pat, mus = bench.workload("grid200", 1)
    vals, rhs = bench.inputs(pat, mus, [(1, 0), (1, 1), (1, 2)])
    times, oms, xs = bench.cpu_run(pat, vals, rhs, 1e-10, 1e9, 3)
    assert len(times) == len(oms) == len(xs) == 3
    for v, b, x, om in zip(vals, rhs, xs, oms):
        # backward error recomputed from a scipy product, independent of the oracle's residual
        K = sp.csr_matrix((v, pat.colidx, pat.rowptr), shape=(pat.n, pat.n))
        r = b - K @ x
        knorm = float(np.max(np.asarray(abs(K).sum(axis=1)).ravel()))
        omega = np.max(np.abs(r)) / (knorm * np.max(np.abs(x)) + np.max(np.abs(b)))
        assert omega <= 1e-10 * (1 + 1e-6)
        assert om <= 1e-10


def test_error_vs_oracle_per_result():
    xo = [np.array([1.0, -2.0, 4.0]), np.array([0.5, 0.0, -0.25])]
    same = [a.copy() for a in xo]
    off = [xo[0] + np.array([0.0, 0.0, 4e-3]), xo[1] - np.array([5e-6, 0.0, 0.0])]
    e = bench.error_vs_oracle(xo, {"fp64": same, "fp32_ir": off, "absent": None})
    assert e["inputs"] == 2 and "absent" not in e
    assert e["fp64"]["max"] == 0.0 and e["fp64"]["per_result"] == [0.0, 0.0]
    assert e["fp32_ir"]["per_result"] == pytest.approx([1e-3, 1e-5])
    assert e["fp32_ir"]["max"] == pytest.approx(1e-3)
    assert e["fp32_ir"]["median"] == pytest.approx((1e-3 + 1e-5) / 2)
    # a zero oracle solution: the absolute difference is stated
    z = bench.error_vs_oracle([np.zeros(2)], {"fp64": [np.array([0.0, 3e-9])]})
    assert z["fp64"]["per_result"] == pytest.approx([3e-9])


def test_timed_steps_cycle_the_input_pool():
    """Warm-up steps use their own inputs; the timed steps cycle through the
    remaining distinct inputs of the pool, every pool input used."""
    from types import SimpleNamespace
    for steps, warmup in [(400, 3), (5, 3), (24, 4), (25, 3)]:
        a = SimpleNamespace(steps=steps, warmup=warmup)
        n = bench.pool_size(a)
        assert n == warmup + min(steps, bench.POOL_STEPS)
        idx = [bench.at(a, i) for i in range(warmup + steps)]
        assert idx[:warmup] == list(range(warmup))
        timed = idx[warmup:]
        assert all(warmup <= i < n for i in timed)
        assert set(timed) == set(range(warmup, n))
        # consecutive timed steps never repeat an input while the pool has more than one
        assert all(x != y for x, y in zip(timed, timed[1:])) or n - warmup == 1


def test_input_pool_spans_the_mu_schedule():
    """The timed inputs are spread over the whole schedule (first and last
    step included, in order); the warm-up inputs come from another seed."""
    from types import SimpleNamespace
    a = SimpleNamespace(steps=400, warmup=3)
    plan = bench.pool_plan(a, 100, 5)
    warm, timed = plan[:3], plan[3:]
    assert len(timed) == bench.POOL_STEPS
    ks = [k for _, k in timed]
    assert ks[0] == 0 and ks[-1] == 99 and ks == sorted(ks) and len(set(ks)) == len(ks)
    assert all(sd == 5 for sd, _ in timed) and all(sd != 5 for sd, _ in warm)
    short = bench.pool_plan(SimpleNamespace(steps=2, warmup=3), 100, 5)[3:]
    assert [k for _, k in short] == [0, 99]


def test_defaults_are_the_mixed_precision_70k_line():
    a = bench.parse([])
    assert a.workload == "eastern70k" and a.precision == "fp32" and a.tol == 1e-10
    assert not a.no_compare and a.warmup >= 3


def test_roofline_bytes_follow_the_algorithmic_formula():
    """Refactorization bytes: nnz(K) (value + index) + nnz(L+U) (value +
    index) + the scaling vector; the tree kernel's share counts only its
    fronts' entries and pivots."""
    plan = {"nnz_lu": 1000, "tree_nnz_k": 30, "tree_nnz_lu": 400, "tree_pivots": 20, "tree_levels": 5,
            "tree_bytes": 123456}
    ab = bench.algorithmic_bytes(plan, n=100, nnz=500, wbytes=4)
    assert ab["refactor"] == 500 * 12 + 1000 * 8 + 100 * 8
    assert ab["solve"] == 1000 * 8 + 4 * 100 * 4
    assert ab["spmv"] == 500 * 12 + 3 * 100 * 8
    assert bench.tree_factor_bytes(plan, 8) == 30 * 12 + 400 * 12 + 20 * 8
    stats = {"tree_factor_kernel": (6, 3.0), "ruiz_kernel": (21, 0.9), "scale_kernel": (3, 0.3)}
    r = bench.roofline_of(stats, 3, plan, ab, 8, "grid200", "fp64")
    assert r["kernel"] == "tree_factor_kernel" and r["launches_per_unit"] == 2
    assert r["ms_per_unit"] == pytest.approx(1.0)
    assert r["achieved"] == pytest.approx(bench.tree_factor_bytes(plan, 8) / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["multifrontal_traffic_model_bytes"] == 123456


def test_oracle_pool_runs_one_process_per_task_and_counts_solves():
    """The host-core baseline of the batch and serving workloads: spawned
    processes (none forked from a GPU process), each timing the oracle on its
    own systems within its budget."""
    tasks = [(20, 26, 4, 1, [(1, 1e-2), (2, 1e-4)], 60.0), (30, 40, 6, 2, [(3, 1e-3)], 60.0)]
    out, cores = bench.oracle_pool(tasks)
    assert cores >= 1 and len(out) == 2
    assert out[0][0] == 2 and out[1][0] == 1 and all(t > 0 for _, t in out)
