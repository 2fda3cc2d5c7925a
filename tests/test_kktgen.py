"""Pins for the synthetic ACOPF KKT generator (problem data of Eq. 11).

J and H are checked against central finite differences of the power-flow
equations written independently in complex form (S = E conj(y (E_i - E_j)));
the matrix sizes against the paper's Table I; the inertia against eigvalsh.
"""
import os

import numpy as np
import pytest

from kktgen import KKTPattern, make_grid, mu_schedule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_grids.txt")


def _complex_constraints(grid, flow_limits, V, th, Pg, Qg):
    """Constraint functions c(x) (Eqs. 2-3) via complex power, loads and limits 0."""
    B = grid.n_bus
    E = V * np.exp(1j * th)
    y = 1.0 / (grid.r + 1j * grid.x)
    f, t = grid.f, grid.t
    Sf = E[f] * np.conj(y * (E[f] - E[t]))
    St = E[t] * np.conj(y * (E[t] - E[f]))
    inj = np.zeros(B, complex)
    np.add.at(inj, f, Sf)
    np.add.at(inj, t, St)
    gen = np.zeros(B, complex)
    np.add.at(gen, grid.gen_bus, Pg + 1j * Qg)
    bal = gen - inj
    parts = [bal.real, bal.imag]
    if flow_limits:
        parts += [np.abs(Sf) ** 2, np.abs(St) ** 2]
    return np.concatenate(parts)


def _split(grid, x):
    B, G = grid.n_bus, grid.n_gen
    return x[:B], x[B:2 * B], x[2 * B:2 * B + G], x[2 * B + G:]


@pytest.mark.parametrize("flow_limits", [True, False])
def test_jacobian_matches_finite_differences(flow_limits):
    grid = make_grid(3, 12, 16, 4)
    pat = KKTPattern(grid, flow_limits=flow_limits)
    pt = pat.point(5, 0, 1e-2)
    K = pat.to_scipy(pat.values(pt)).toarray()
    n = pat.n_primal
    J = K[n:, :n]
    assert np.array_equal(K[:n, n:], J.T)
    rng = np.random.default_rng(0)
    Pg, Qg = rng.normal(size=grid.n_gen), rng.normal(size=grid.n_gen)
    x0 = np.concatenate([pt.V, pt.theta, Pg, Qg])
    h = 1e-6
    Jfd = np.zeros_like(J)
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        cp = _complex_constraints(grid, flow_limits, *_split(grid, x0 + e))
        cm = _complex_constraints(grid, flow_limits, *_split(grid, x0 - e))
        Jfd[:, k] = (cp - cm) / (2 * h)
    scale = np.abs(J).max()
    assert np.abs(J - Jfd).max() <= 1e-6 * scale
    # every structural entry of J is present in the pattern
    assert np.all((np.abs(Jfd) > 1e-9 * scale) <= (K[n:, :n] != 0))


def test_hessian_matches_finite_differences_of_lagrangian_gradient():
    grid = make_grid(4, 10, 13, 3)
    pat = KKTPattern(grid)
    pt = pat.point(2, 1, 1e-3)
    n = pat.n_primal
    B, G = grid.n_bus, grid.n_gen
    K = pat.to_scipy(pat.values(pt)).toarray()
    H = K[:n, :n] - np.diag(pt.sigma + pt.delta_w)

    def grad_L(x):
        V, th, Pg, Qg = _split(grid, x)
        q = pat.point(2, 1, 1e-3)
        q.V, q.theta = V, th
        Kx = pat.to_scipy(pat.values(q)).toarray()
        gf = np.zeros(n)
        gf[2 * B:2 * B + G] = 2.0 * grid.c2 * Pg
        return gf + Kx[n:, :n].T @ pt.lam

    rng = np.random.default_rng(1)
    x0 = np.concatenate([pt.V, pt.theta, rng.normal(size=G), rng.normal(size=G)])
    h = 1e-6
    Hfd = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        Hfd[:, k] = (grad_L(x0 + e) - grad_L(x0 - e)) / (2 * h)
    scale = np.abs(H).max()
    assert np.abs(H - Hfd).max() <= 1e-6 * scale
    assert np.allclose(H, H.T, atol=1e-12 * scale)


def test_sizes_formula_and_symmetry():
    for (B, L, G) in [(200, 300, 40), (1000, 1280, 200)]:
        pat = KKTPattern(make_grid(1, B, L, G))
        assert pat.n == 4 * B + 2 * G + 2 * L
        assert pat.nnz == 14 * B + 42 * L + 6 * G
        K = pat.to_scipy(pat.values(pat.point(1, 0)))
        assert (K != K.T).nnz == 0
        assert np.all(np.diff(pat.rowptr) > 0)
        # columns sorted and unique within each row
        for i in range(0, pat.n, 97):
            c = pat.colidx[pat.rowptr[i]:pat.rowptr[i + 1]]
            assert np.all(np.diff(c) > 0)


def test_paper_shape_matches_table_one():
    """Without branch-flow rows the K of Eq. 11 has N = 4B + 2G and
    nnz = 14B + 24L + 6G; Table I's N and nnz are within 5 % of that."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for name, B, G, L, N, nnz in rows:
        B, G, L, N, nnz = map(int, (B, G, L, N, nnz))
        assert abs((4 * B + 2 * G) - N) / N < 0.05, name
        assert abs((14 * B + 24 * L + 6 * G) - nnz) / nnz < 0.05, name
    # the generator realises that count exactly on a small grid
    grid = make_grid(7, 300, 384, 60)
    pat = KKTPattern(grid, flow_limits=False)
    assert pat.n == 4 * 300 + 2 * 60
    assert pat.nnz == 14 * 300 + 24 * 384 + 6 * 60


def test_inertia_n_positive_m_negative():
    """K is nonsingular with inertia (n, m) thanks to dw > 0 and dc > 0."""
    for seed in (1, 2):
        grid = make_grid(seed, 8, 11, 3)
        pat = KKTPattern(grid)
        for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 3)):
            K = pat.to_scipy(pat.values(pat.point(seed, k, mu))).toarray()
            ev = np.linalg.eigvalsh(K)
            assert np.sum(ev > 0) == pat.n_primal
            assert np.sum(ev < 0) == pat.n_dual


def test_barrier_diagonal_distribution():
    pat = KKTPattern(make_grid(1, 2000, 2560, 400))
    B = pat.grid.n_bus
    for mu in (1e-1, 1e-9):
        s = pat.point(1, 3, mu).sigma
        bounded = np.concatenate([s[:B], s[2 * B:]])
        assert np.all(s[B:2 * B] == 0.0)
        assert bounded.min() >= 1e-8 * (1 - 1e-12) and bounded.max() <= 1e8 * (1 + 1e-12)
        # log-uniform: log10 is uniform on [-8, 8]
        lg = np.log10(bounded)
        assert abs(lg.mean()) < 0.5 and abs(np.median(lg)) < 0.7


def test_grid_is_connected_tree_plus_extra():
    grid = make_grid(11, 500, 640, 100)
    assert grid.f.size == 640
    assert np.unique(grid.gen_bus).size == 100
    keys = np.minimum(grid.f, grid.t) * 500 + np.maximum(grid.f, grid.t)
    assert np.unique(keys).size == keys.size and np.all(grid.f != grid.t)
    assert (grid.tree_parent >= 0).sum() == 499
    assert 0.001 <= grid.r.min() and grid.r.max() <= 0.01
    assert 0.01 <= grid.x.min() and grid.x.max() <= 0.1


def test_seeded_values_are_reproducible():
    pat = KKTPattern(make_grid(5, 50, 70, 10))
    a = pat.values(pat.point(9, 4, 1e-3))
    b = pat.values(pat.point(9, 4, 1e-3))
    c = pat.values(pat.point(9, 5, 1e-3))
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_slack_range_changes_only_the_flow_rows_diagonal():
    """With slack terms the (2,2) diagonal of every flow-limit row becomes
    -(dc + 1/sigma_s), 1/sigma_s within the requested range; every other value
    is bitwise the literal one (the slack draws use a stream of their own)."""
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    B, n = 200, pat.n_primal
    lit = pat.values(pat.point(1, 3, 1e-3))
    sl = pat.values(pat.point(1, 3, 1e-3, slack_range=(1e-2, 1e2)))
    K0, K1 = pat.to_scipy(lit), pat.to_scipy(sl)
    D = (K1 - K0).tocoo()
    D.eliminate_zeros()
    rows = np.arange(n + 2 * B, pat.n)
    assert sorted(zip(D.row.tolist(), D.col.tolist())) == [(r, r) for r in rows]
    s = -(K1.diagonal()[rows] - K0.diagonal()[rows])
    assert np.all(s >= 1e-2 * (1 - 1e-12)) and np.all(s <= 1e2 * (1 + 1e-12))
    assert np.log10(s).std() > 0.5                      # spread over the range, not one value
