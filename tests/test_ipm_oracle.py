"""Pins of the oracle's interior-point loop (oracle/ipm.py), independent of it:

* an independent NLP solver (scipy's trust-constr, a different algorithm) on
  the same problem, written from the generator's flow functions, reaches the
  same optimal cost;
* at the returned point the first-order conditions hold with the constraint
  Jacobian taken by central differences of the constraint functions (not the
  analytic one the loop uses), and the point is feasible within the bounds;
* a planted sign error in the Newton right-hand side (the barrier term of
  the bounds) breaks convergence, so the pins would see a dropped or flipped
  term.
"""
import numpy as np
import pytest

from kktgen import KKTPattern, flat_start, line_terms, make_grid, opf_data
from oracle import ipm


def _instance(B, L, G, seed):
    pat = KKTPattern(make_grid(seed, B, L, G))
    return pat, opf_data(pat.grid, seed)


def _cons(pat, data, x):
    """The constraints written again from the generator's flow functions."""
    g = pat.grid
    B, G = g.n_bus, g.n_gen
    V, th, Pg, Qg = x[:B], x[B:2 * B], x[2 * B:2 * B + G], x[2 * B + G:]
    (Pf, Qf, *_), (Pt, Qt, *_) = line_terms(g, V, th)
    gen = np.zeros((2, B))
    gen[0, g.gen_bus] = Pg
    gen[1, g.gen_bus] = Qg
    inc = np.zeros((B, g.n_branch))
    inc[g.f, np.arange(g.n_branch)] = 1.0
    out = np.zeros((B, g.n_branch))
    out[g.t, np.arange(g.n_branch)] = 1.0
    Pb = gen[0] - data.Pd - inc @ Pf - out @ Pt
    Qb = gen[1] - data.Qd - inc @ Qf - out @ Qt
    return np.concatenate([Pb, Qb]), np.concatenate([Pf ** 2 + Qf ** 2, Pt ** 2 + Qt ** 2])


@pytest.mark.parametrize("B,L,G,seed", [(5, 6, 2, 1), (9, 12, 3, 2)])
def test_same_optimum_as_an_independent_nlp_solver(B, L, G, seed):
    from scipy.optimize import Bounds, NonlinearConstraint, minimize
    pat, data = _instance(B, L, G, seed)
    g = pat.grid
    r = ipm.solve(pat, data, flat_start(g, data))
    assert r.err <= 1e-7
    lo, hi = data.bounds(g)
    cost = lambda x: float(np.sum(g.c2 * x[2 * B:2 * B + G] ** 2))                   # noqa: E731
    eq = NonlinearConstraint(lambda x: _cons(pat, data, x)[0], 0.0, 0.0)
    ineq = NonlinearConstraint(lambda x: _cons(pat, data, x)[1], -np.inf, np.concatenate([data.Smax, data.Smax]) ** 2)
    ref = minimize(cost, flat_start(g, data), method="trust-constr", constraints=[eq, ineq],
                   bounds=Bounds(lo, hi), options={"gtol": 1e-10, "xtol": 1e-12, "maxiter": 5000})
    assert np.max(np.abs(_cons(pat, data, ref.x)[0])) <= 1e-7
    # both feasible (the loop's point checked with the constraints written again here), and the
    # same cost within the loop's stopping tolerance (E_0 <= 1e-7) plus trust-constr's own accuracy
    cE, cI = _cons(pat, data, r.x)
    assert np.max(np.abs(cE)) <= 1e-7 and np.all(cI <= np.concatenate([data.Smax, data.Smax]) ** 2 + 1e-7)
    assert abs(r.objective - ref.fun) <= 1e-5 * ref.fun + 1e-7


@pytest.mark.parametrize("B,L,G,seed", [(37, 50, 8, 2), (200, 300, 40, 1)])
def test_first_order_conditions_with_finite_difference_jacobian(B, L, G, seed):
    pat, data = _instance(B, L, G, seed)
    g = pat.grid
    r = ipm.solve(pat, data, flat_start(g, data))
    assert r.err <= 1e-7 and r.iters < 60
    x = r.x
    assert abs(x[B + ipm.IPMOptions().angle_ref]) <= 1e-7          # the pin holds the reference angle at 0
    n = x.size
    # central differences of the constraints, column by column
    h = 1e-6
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        cp = np.concatenate(_cons(pat, data, x + e))
        cm = np.concatenate(_cons(pat, data, x - e))
        cols.append((cp - cm) / (2 * h))
    Jfd = np.array(cols).T
    grad = np.zeros(n)
    grad[2 * B:2 * B + G] = 2.0 * g.c2 * x[2 * B:2 * B + G]
    opt = ipm.IPMOptions()
    grad[B + opt.angle_ref] = 2.0 * opt.angle_pin * x[B + opt.angle_ref]     # the reference-angle term
    stat = grad + Jfd.T @ r.lam - r.zL + r.zU
    assert np.max(np.abs(stat)) <= 1e-6 * max(1.0, np.max(np.abs(r.lam)))
    cE, cI = _cons(pat, data, x)
    lo, hi = data.bounds(g)
    assert np.max(np.abs(cE)) <= 1e-7
    assert np.all(cI <= np.concatenate([data.Smax, data.Smax]) ** 2 + 1e-7)
    fin = np.isfinite(lo)
    assert np.all(x[fin] >= lo[fin]) and np.all(x[fin] <= hi[fin])
    # complementarity at mu -> 0 and the slack multipliers equal the flow rows' lambda
    assert np.max(np.abs(r.lam[2 * B:] - r.w)) <= 1e-7


def test_a_planted_sign_error_breaks_convergence(monkeypatch):
    """The objective gradient with the wrong sign (planted in the oracle): the
    loop then heads for the most expensive dispatch and does not reach the
    optimum within 60 iterations."""
    pat, data = _instance(37, 50, 8, 2)
    good = ipm.solve(pat, data, flat_start(pat.grid, data))
    assert good.err <= 1e-7
    orig_grad = ipm.gradient
    monkeypatch.setattr(ipm, "gradient", lambda p, x, o=ipm.IPMOptions(): -orig_grad(p, x, o))
    bad = ipm.solve(pat, data, flat_start(pat.grid, data), ipm.IPMOptions(max_iter=60))
    assert not (bad.err <= 1e-7 and abs(bad.objective - good.objective) <= 1e-6 * good.objective)
