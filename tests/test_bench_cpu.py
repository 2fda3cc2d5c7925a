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
    vals, rhs = bench.inputs(pat, mus, 1, 3)
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
