"""Pins for the CPU oracle, each against something other than the oracle itself:
LAPACK's partial-pivoting LU, an independent symbolic elimination game
(networkx), dense no-pivot elimination, Sylvester's law of inertia,
closed forms, numpy / scipy solves and GMRES finite termination."""
import networkx as nx
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import oracle as O
from kktgen import KKTPattern, make_grid, mu_schedule


def dense_csr(M):
    """Structurally full CSR of a dense matrix (every entry stored)."""
    n = M.shape[0]
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    return rp, ci, M.reshape(-1).astype(np.float64)


def csr_of(S):
    S = sp.csr_matrix(S)
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64)


def factors_dense(f):
    n = f.n
    L = np.eye(n)
    U = np.zeros((n, n))
    for j in range(n):
        for s in range(f.Lp[j], f.Lp[j + 1]):
            L[f.Li[s], j] = f.Lx[s]
        for s in range(f.Up[j], f.Up[j + 1]):
            U[f.Ui[s], j] = f.Ux[s]
    return L, U


def an_floor(sv, eps=1e-14):
    return eps * np.abs(sv).max()


@pytest.fixture(scope="module")
def kkt200():
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    return pat


# ---------------------------------------------------------------- scaling

def test_ruiz_powers_of_two_and_equilibrated(kkt200):
    pat = kkt200
    v = pat.values(pat.point(1, 0, 1e-1))
    d, it = O.ruiz(pat.rowptr, pat.colidx, v, 60)
    assert it < 60                                   # converged: no factor changed
    m, e = np.frexp(d)
    assert np.all(m == 0.5)                          # exact powers of two
    sv = O.scale(pat.rowptr, pat.colidx, v, d)
    A = sp.csr_matrix((np.abs(sv), pat.colidx, pat.rowptr), shape=(pat.n, pat.n))
    rmax = A.max(axis=1).toarray().ravel()
    # at the fixed point round(-log2(r)/2) = 0, i.e. r in (1/2, 2]
    assert np.all(rmax > 0.5) and np.all(rmax <= 2.0)


def test_ruiz_diagonal_closed_form():
    a = np.array([4.0, 1.0 / 16, 3.0, 1e-10, 7e9])
    rp, ci, v = csr_of(sp.diags(a))
    d, _ = O.ruiz(rp, ci, v, 10)
    # one step gives d = 2^round(-log2(a)/2); then d^2 a is in (1/2, 2] and stays
    expect = 2.0 ** np.round(-np.log2(a) / 2)
    assert np.array_equal(d, expect)


# --------------------------------------------------------------- ordering

def _elimination_game(G, order):
    """Independent symbolic elimination (networkx): fill edges and degrees."""
    G = G.copy()
    degs, fill = [], set()
    for v in order:
        nb = list(G.neighbors(v))
        degs.append((v, {u: G.degree(u) for u in G.nodes}))
        for a in nb:
            for b in nb:
                if a < b:
                    if not G.has_edge(a, b):
                        G.add_edge(a, b)
                    fill.add((a, b))
        G.remove_node(v)
    return degs, fill


def test_min_degree_hand_cases():
    # path 0-1-2-3: degree-1 ends, lowest index first
    P = sp.diags([1.0, 1.0, 1.0], [-1, 0, 1], shape=(4, 4)) + sp.eye(4)
    rp, ci, _ = csr_of(P)
    assert list(O.min_degree(rp, ci)) == [0, 1, 2, 3]
    # star with centre 0: leaves 1, 2, 3 go first; then centre and leaf 4 both
    # have degree 1 and the lower index (the centre) wins the tie
    S = sp.lil_matrix((5, 5))
    for i in range(5):
        S[i, i] = 1
    for i in range(1, 5):
        S[0, i] = S[i, 0] = 1
    rp, ci, _ = csr_of(S)
    assert list(O.min_degree(rp, ci)) == [1, 2, 3, 0, 4]


def test_min_degree_chooses_minimum_degree_every_step(kkt200):
    pat = kkt200
    q = O.min_degree(pat.rowptr, pat.colidx)
    assert np.array_equal(np.sort(q), np.arange(pat.n))
    G = nx.Graph()
    G.add_nodes_from(range(pat.n))
    rows = np.repeat(np.arange(pat.n), np.diff(pat.rowptr))
    G.add_edges_from((int(a), int(b)) for a, b in zip(rows, pat.colidx) if a < b)
    degs, _ = _elimination_game(G, [int(v) for v in q[:400]])
    for v, dmap in degs:
        dmin = min(dmap.values())
        assert dmap[v] == dmin
        assert v == min(u for u, d in dmap.items() if d == dmin)


def test_min_degree_no_fill_on_tree():
    g = nx.random_labeled_tree(60, seed=3) if hasattr(nx, "random_labeled_tree") else nx.random_tree(60, seed=3)
    A = nx.to_scipy_sparse_array(g, nodelist=range(60)) + sp.eye(60)
    rp, ci, _ = csr_of(A)
    q = O.min_degree(rp, ci)
    _, fill = _elimination_game(g, [int(v) for v in q])
    assert all(g.has_edge(a, b) for a, b in fill)    # no new edge ever created


# --------------------------------------------------------------------- LU

def test_partial_pivoting_matches_lapack():
    """tau = 1, Q = I on a full matrix is LAPACK getrf's partial pivoting."""
    rng = np.random.default_rng(4)
    for n in (5, 17, 40):
        M = rng.normal(size=(n, n))
        rp, ci, v = dense_csr(M)
        f = O.LU(rp, ci, v, np.arange(n), None, 1.0, 0.0).factors()
        Pl, Ll, Ul = sl.lu(M)                        # M = Pl Ll Ul
        perm = np.argmax(Pl, axis=0)                 # row of M at step j
        assert np.array_equal(f.p, perm)
        L, U = factors_dense(f)
        assert np.allclose(L, Ll, atol=1e-12) and np.allclose(U, Ul, atol=1e-12 * np.abs(Ul).max())


def test_threshold_rule_hand_case():
    # column 0 = (1e-3, 1): |diag| < 0.1 * 1 -> pivot on row 1; with tau = 1e-4 keep the diagonal
    M = np.array([[1e-3, 2.0], [1.0, 5.0]])
    rp, ci, v = dense_csr(M)
    f = O.LU(rp, ci, v, np.arange(2), None, 0.1, 0.0).factors()
    assert list(f.p) == [1, 0] and f.n_offdiag == 2
    L, U = factors_dense(f)
    assert np.allclose(L, [[1, 0], [1e-3, 1]]) and np.allclose(U, [[1, 5], [0, 2 - 5e-3]])
    f = O.LU(rp, ci, v, np.arange(2), None, 1e-4, 0.0).factors()
    assert list(f.p) == [0, 1] and f.n_offdiag == 0
    L, U = factors_dense(f)
    assert np.allclose(L, [[1, 0], [1000.0, 1]]) and np.allclose(U, [[1e-3, 2], [0, 5 - 2000.0]])


def test_static_perturbation_hand_case():
    # frozen diagonal pivots on [[0, 1], [1, 0]]: u00 = 0 -> +floor; then u11 = -1/floor
    M = np.array([[0.0, 1.0], [1.0, 0.0]])
    rp, ci, v = dense_csr(M)
    floor = 1e-6
    f = O.LU(rp, ci, v, np.arange(2), np.arange(2), 0.0, floor).factors()
    assert f.n_perturbed == 1
    L, U = factors_dense(f)
    assert U[0, 0] == floor and L[1, 0] == 1.0 / floor and U[1, 1] == -1.0 / floor
    # a tiny negative pivot keeps its sign
    M = np.array([[-1e-9, 1.0], [1.0, 3.0]])
    rp, ci, v = dense_csr(M)
    f = O.LU(rp, ci, v, np.arange(2), np.arange(2), 0.0, floor).factors()
    assert f.n_perturbed == 1 and factors_dense(f)[1][0, 0] == -floor


def test_kkt_factor_reconstruction_and_symbolic_fill(kkt200):
    """Componentwise LU backward error |P A Q + E - L U| <= gamma_k |L| |U|
    (Higham, Thm. 9.3; k = longest inner product), and the pattern of L equals
    the fill graph of an independent symbolic elimination in the order q."""
    pat = kkt200
    v = pat.values(pat.point(1, 0, 1e-1))
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an)
    f = lu.factors()
    A = sp.csr_matrix((sv, pat.colidx, pat.rowptr), shape=(pat.n, pat.n)).toarray()
    PAQ = A[np.ix_(f.p, f.q)]
    L, U = factors_dense(f)
    R = L @ U - PAQ
    E = np.diag(np.diag(R)) * 0.0
    if f.n_perturbed:
        # static perturbations only move diagonal entries of U
        pert = np.abs(np.abs(np.diag(U)) - an_floor(sv)) == 0
        E = np.diag(np.where(pert, np.diag(R), 0.0))
    k = int(max(np.diff(f.Lp).max(), np.diff(f.Up).max())) + 1
    u = np.finfo(float).eps / 2
    gamma = k * u / (1 - k * u)
    assert np.all(np.abs(R - E) <= gamma * (np.abs(L) @ np.abs(U)) + 1e-300)
    # symbolic: with P = Q^T the L pattern (in original labels) is the fill graph
    assert np.array_equal(f.p, f.q)
    G = nx.Graph()
    G.add_nodes_from(range(pat.n))
    rows = np.repeat(np.arange(pat.n), np.diff(pat.rowptr))
    G.add_edges_from((int(a), int(b)) for a, b in zip(rows, pat.colidx) if a < b)
    _, fill = _elimination_game(G, [int(x) for x in f.q])
    edges = {(min(a, b), max(a, b)) for a, b in G.edges} | fill
    Lpat = set()
    for j in range(pat.n):
        for s in range(f.Lp[j], f.Lp[j + 1]):
            a, b = int(f.q[j]), int(f.p[f.Li[s]])
            Lpat.add((min(a, b), max(a, b)))
    # L pattern = every edge whose earlier end is eliminated first
    assert Lpat == edges


def test_normwise_reconstruction_when_growth_is_bounded():
    """||P A Q - L U||_F / ||A||_F <= 1e-13 on tiny KKT instances whose barrier
    diagonal and regularisation keep element growth small (Sigma in [0.1, 10],
    dw = dc = 1)."""
    for seed in (1, 2, 3):
        pat = KKTPattern(make_grid(seed, 10, 14, 3))
        pt = pat.point(seed, 0, 1e-2, delta_w=1.0, delta_c=1.0)
        pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, 0.1, 10.0), 0.0)
        v = pat.values(pt)
        an = O.analyze(pat.rowptr, pat.colidx, v)
        lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an)
        f = lu.factors()
        assert f.n_perturbed == 0
        A = sp.csr_matrix((sv, pat.colidx, pat.rowptr), shape=(pat.n, pat.n)).toarray()
        L, U = factors_dense(f)
        assert np.linalg.norm(L @ U - A[np.ix_(f.p, f.q)]) <= 1e-13 * np.linalg.norm(A)


def test_pattern_contains_dense_elimination_nonzeros():
    """Brute force: dense no-pivot elimination of P A Q with random values."""
    pat = KKTPattern(make_grid(2, 12, 15, 3))
    rng = np.random.default_rng(0)
    v = rng.uniform(1.0, 2.0, size=pat.nnz)
    A = sp.csr_matrix((v, pat.colidx, pat.rowptr), shape=(pat.n, pat.n)).toarray()
    A += np.diag(np.full(pat.n, 50.0))        # keep the dense elimination pivots away from 0
    rp, ci, vv = csr_of(sp.csr_matrix(A))
    q = O.min_degree(rp, ci)
    f = O.LU(rp, ci, vv, q, q, 0.0, 0.0).factors()
    M = A[np.ix_(f.p, f.q)].copy()
    n = pat.n
    for k in range(n):                         # textbook Doolittle, no pivoting
        M[k + 1:, k] /= M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:])
    L, U = factors_dense(f)
    struct = (np.tril(L, -1) != 0) | (np.triu(U) != 0)
    nz = np.abs(M) > 1e-12
    assert np.all(nz <= struct)
    assert np.allclose(np.tril(M, -1), np.tril(L, -1), atol=1e-12)
    assert np.allclose(np.triu(M), np.triu(U), rtol=1e-12, atol=1e-12)


def test_inertia_from_pivot_signs():
    """With P = Q^T and no perturbation, U = D L^T, so sign counts of diag(U)
    give the inertia (Sylvester): n positive, m negative."""
    for seed in (1, 2):
        pat = KKTPattern(make_grid(seed, 8, 11, 3))
        v = pat.values(pat.point(seed, 0, 1e-2))
        an = O.analyze(pat.rowptr, pat.colidx, v)
        lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an, pivot_eps=0.0)
        f = lu.factors()
        diag = f.Ux[f.Up[1:] - 1]
        ev = np.linalg.eigvalsh(pat.to_scipy(v).toarray())
        assert np.sum(diag > 0) == np.sum(ev > 0) == pat.n_primal
        assert np.sum(diag < 0) == np.sum(ev < 0) == pat.n_dual


# ------------------------------------------------- solve, residual, omega

def test_solve_matches_numpy_on_well_conditioned_kkt():
    pat = KKTPattern(make_grid(3, 30, 40, 6))
    v = pat.values(pat.point(3, 0, 1e-1, delta_w=1.0, delta_c=1.0))
    b = pat.rhs(3, 0)
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an)
    x = lu.solve_scaled(d, b)
    K = pat.to_scipy(v).toarray()
    xr = np.linalg.solve(K, b)
    assert np.linalg.cond(K) < 1e12
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)


def test_spmv_and_backward_error(kkt200):
    pat = kkt200
    v = pat.values(pat.point(1, 2, 1e-3))
    rng = np.random.default_rng(0)
    x, b = rng.normal(size=pat.n), rng.normal(size=pat.n)
    r = O.spmv_resid(pat.rowptr, pat.colidx, v, x, b)
    K = pat.to_scipy(v)
    ref = b - K @ x
    assert np.abs(r - ref).max() <= 1e-12 * (abs(K) @ np.abs(x) + np.abs(b)).max()
    # closed form on a diagonal system
    k = np.array([2.0, -4.0, 0.5])
    rp, ci, vv = csr_of(sp.diags(k))
    xd, bd = np.array([1.0, 1.0, 2.0]), np.array([2.0, -3.0, 0.0])
    om = O.backward_error(rp, ci, vv, xd, bd)
    assert om == pytest.approx(1.0 / (4.0 * 2.0 + 3.0), rel=1e-15)   # ||r|| = max(0, 1, 1)


def test_fgmres_finite_termination_two_eigenvalues():
    """M^{-1} K with two distinct eigenvalues: GMRES is exact after 2 steps."""
    n = 12
    k = np.linspace(1.0, 3.0, n)
    kp = np.where(np.arange(n) % 2 == 0, k / 2.0, k / 5.0)   # K M^{-1} = diag(2 or 5)
    rp, ci, vk = csr_of(sp.diags(k))
    _, _, vp = csr_of(sp.diags(kp))
    lu = O.LU(rp, ci, vp, np.arange(n), np.arange(n), 0.0, 0.0)
    b = np.random.default_rng(1).normal(size=n)
    x, it, om = O.fgmres(rp, ci, vk, lu, np.ones(n), b, restart=30, max_cycles=3, tol=1e-15)
    assert it == 2
    assert om <= 1e-15
    assert np.allclose(x, b / k, rtol=1e-13)


def test_fgmres_repairs_a_stale_preconditioner(kkt200):
    """Preconditioner from a different iterate (stale factors): refinement still
    reaches omega <= 1e-14 (the stale solve alone does not) and the result
    solves the new system."""
    pat = kkt200
    v0 = pat.values(pat.point(1, 0, 1e-1))
    an = O.analyze(pat.rowptr, pat.colidx, v0)
    p1 = pat.point(1, 0, 1e-1)
    p1.sigma = p1.sigma * 1.5
    v1 = pat.values(p1)
    lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v0, an)
    b = pat.rhs(1, 0)
    x0 = lu.solve_scaled(d, b)
    assert O.backward_error(pat.rowptr, pat.colidx, v1, x0, b) > 1e-14
    x, it, om = O.fgmres(pat.rowptr, pat.colidx, v1, lu, d, b, 30, 10, 1e-14)
    assert om <= 1e-14 and it >= 1
    assert O.backward_error(pat.rowptr, pat.colidx, v1, x, b) == pytest.approx(om)


def test_alg1_sequence_reaches_backward_error(kkt200):
    """Alg. 1 on the 200-bus workload: analyze on K_1, refactor + solve + refine K_2..K_10."""
    pat = kkt200
    an = O.analyze(pat.rowptr, pat.colidx, pat.values(pat.point(1, 0, 1e-1)))
    for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 10)):
        v = pat.values(pat.point(1, k, mu))
        b = pat.rhs(1, k)
        lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an)
        x, it, om = O.fgmres(pat.rowptr, pat.colidx, v, lu, d, b, 30, 10, 1e-12)
        assert om <= 1e-12


def test_jacobi_precondition_pins():
    """Jacobi sweeps with the factors (Sec. V): one sweep per factor is the
    closed form D Q diag(U)^-1 P D b; as many sweeps as unknowns reproduce the
    exact solve (L - I and U - diag(U) are nilpotent); sweeps leave a
    diagonal system's exact solution unchanged."""
    import scipy.sparse as sp
    pat = KKTPattern(make_grid(3, 30, 40, 6))
    v = pat.values(pat.point(3, 0, 1e-1, delta_w=1.0, delta_c=1.0))
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an)
    f = lu.factors()
    b = pat.rhs(3, 0)
    n = pat.n
    U = sp.csc_matrix((f.Ux, f.Ui, f.Up), shape=(n, n))
    one = O.jacobi_precondition(f, d, b, 1)
    z = np.empty(n)
    z[f.q] = ((d * b)[f.p]) / U.diagonal()
    assert np.allclose(one, d * z, rtol=1e-15, atol=0)
    full = O.jacobi_precondition(f, d, b, n)
    exact = lu.solve_scaled(d, b)
    assert np.linalg.norm(full - exact) <= 1e-10 * np.linalg.norm(exact)
    few = O.jacobi_precondition(f, d, b, 3)
    assert np.linalg.norm(few - exact) > 1e-6 * np.linalg.norm(exact)      # not exact after 3 sweeps
    rp = np.arange(4, dtype=np.int32)
    ci = np.arange(3, dtype=np.int32)
    dv = np.array([2.0, -4.0, 0.5])
    an3 = O.analyze(rp, ci, dv)
    lu3, d3, _ = O.refactor(rp, ci, dv, an3)
    bb = np.array([1.0, 2.0, 3.0])
    assert np.allclose(O.jacobi_precondition(lu3.factors(), d3, bb, 1), bb / dv, rtol=1e-15)


def test_solution_not_determined_at_fp64_on_the_literal_kkt(kkt200):
    """With -dc = -1e-10 on every constraint row and more constraint rows than
    primals (m = 2B + 2L > n = 2B + 2G), the null space of J^T is held by dc
    alone: cond(K) is far beyond 1/eps_FP64. Two backward-stable FP64 solves
    that differ only in the static-pivot threshold (1e-14 vs 1e-12 of max|DKD|)
    both reach omega <= 1e-14, yet their solutions differ by more than 1 % of
    max|x| in the dual block, whose entries reach ~|b| / dc. This is why the
    parity gates are omega and the factor entries (running error bounds), and
    why a result's difference from the oracle's x is stated, not gated."""
    pat = kkt200
    m = pat.n - pat.n_primal
    assert m > pat.n_primal
    v = pat.values(pat.point(1, 3, 1e-3))
    b = pat.rhs(1, 3)
    xs = []
    for eps in (1e-14, 1e-12):
        an = O.analyze(pat.rowptr, pat.colidx, v, pivot_eps=eps)
        lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an, pivot_eps=eps)
        x, _, om = O.fgmres(pat.rowptr, pat.colidx, v, lu, d, b, 30, 10, 1e-14)
        assert om <= 1e-14
        xs.append(x)
    y0, y1 = xs[0][pat.n_primal:], xs[1][pat.n_primal:]
    assert np.abs(y0).max() > 1e8 * np.abs(b).max()
    assert np.abs(y1 - y0).max() > 1e-2 * np.abs(y0).max()


def _exact_doolittle(A):
    """LU without pivoting of a dense float matrix over the rationals (every
    double is an exact binary fraction): multipliers below the diagonal, U on
    and above it."""
    from fractions import Fraction
    n = A.shape[0]
    M = [[Fraction(float(x)) if x != 0 else Fraction(0) for x in row] for row in A]
    for k in range(n):
        piv = M[k][k]
        rk = [(j, M[k][j]) for j in range(k + 1, n) if M[k][j] != 0]
        for i in range(k + 1, n):
            if M[i][k] != 0:
                M[i][k] = M[i][k] / piv
                lik = M[i][k]
                for j, ukj in rk:
                    M[i][j] -= lik * ukj
    return M


def _float32_doolittle(A):
    """The same elimination in single precision (operands rounded to FP32,
    every product, difference and quotient rounded to FP32)."""
    M = A.astype(np.float32)
    for k in range(M.shape[0]):
        M[k + 1:, k] = M[k + 1:, k] / M[k, k]
        M[k + 1:, k + 1:] -= np.outer(M[k + 1:, k], M[k, k + 1:]).astype(np.float32)
    return M


@pytest.mark.parametrize("seed,step,mu", [(1, 2, 1e-3), (2, 5, 1e-6), (3, 0, 1e-1), (4, 1, 1e-2), (5, 7, 1e-8)])
def test_running_error_bound_holds_against_exact_factors(seed, step, mu):
    """The first-order running error bound of every factor entry (Wilkinson's
    running error analysis; the tolerance of the GPU factor parity) against
    factors computed exactly over the rationals from the same scaled matrix
    and order. Every entry of the oracle's FP64 factors, and of an FP32
    elimination in the same order, lies within its bound for that format's
    unit roundoff, in the columns before the first pivot where the bound
    states its own invalidity (err(u_jj) >= |u_jj| / 2; here the
    rounding-noise pivot of the angle-shift direction, near the root).
    Left-looking column j depends only on columns < j, so those columns are
    exactly the entries that do not depend on such a pivot. The bound is not
    loose either: the FP32 errors reach more than half of it."""
    from fractions import Fraction
    pat = KKTPattern(make_grid(seed, 10, 14, 3))
    v = pat.values(pat.point(seed, step, mu))
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an)
    f = lu.factors()
    assert f.n_perturbed == 0
    A = sp.csr_matrix((sv, pat.colidx, pat.rowptr), shape=(pat.n, pat.n)).toarray()[np.ix_(f.p, f.q)]
    M = _exact_doolittle(A)
    M32 = _float32_doolittle(A)
    for unit, got_L, got_U in [(2.0 ** -53, lambda s, i, j: f.Lx[s], lambda s, i, j: f.Ux[s]),
                               (2.0 ** -24, lambda s, i, j: M32[i, j], lambda s, i, j: M32[i, j])]:
        eL, eU = lu.error_bound(pat.rowptr, pat.colidx, sv, unit, 0.0)
        invalid = [j for j in range(f.n) if not eU[f.Up[j + 1] - 1] < abs(f.Ux[f.Up[j + 1] - 1]) / 2]
        cut = min(invalid) if invalid else f.n
        assert cut >= f.n - 8                                   # only pivots near the root
        worst = 0.0
        for j in range(cut):
            for lo, hi, idx, bound, got in [(f.Lp[j], f.Lp[j + 1], f.Li, eL, got_L),
                                            (f.Up[j], f.Up[j + 1], f.Ui, eU, got_U)]:
                for s in range(lo, hi):
                    i = int(idx[s])
                    err = abs(Fraction(float(got(s, i, j))) - M[i][j])
                    assert err <= Fraction(float(bound[s])), (unit, i, j, float(err), bound[s])
                    if bound[s] > 0:
                        worst = max(worst, float(err / Fraction(float(bound[s]))))
        if unit == 2.0 ** -24:
            assert worst > 0.5
        else:
            assert worst > 0.05


@pytest.mark.parametrize("step,mu", [(0, 1e-1), (3, 1e-3), (7, 1e-7)])
def test_slack_terms_determine_x_and_the_fp32_threshold_needs_refinement(kkt200, step, mu):
    """With the inequality slacks' term kept in the (2,2) block (1/sigma_s in
    [1e-2, 1e2]) the solution is determined at FP64: solves without
    equilibration agree with the default within 1e-2. Factors with the FP32
    static-pivot threshold (eps = 1e-7, FP64 arithmetic) meet omega <= 1e-10
    with no refinement step, yet differ from it by more than 10 %; refined to
    omega <= 1e-15 they agree within 1e-2. Contrast with the literal matrix
    (test_solution_not_determined_at_fp64_on_the_literal_kkt)."""
    pat = kkt200
    npr = pat.n_primal
    v = pat.values(pat.point(1, step, mu, slack_range=(1e-2, 1e2)))
    b = pat.rhs(1, step)

    def solve(eps=1e-14, tol=1e-15, ruiz=10):
        an = O.analyze(pat.rowptr, pat.colidx, v, ruiz_iters=ruiz, pivot_eps=eps)
        lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an, ruiz_iters=ruiz, pivot_eps=eps)
        return O.fgmres(pat.rowptr, pat.colidx, v, lu, d, b, 30, 10, tol)

    def diff(x, y):
        return max(np.abs(x[:npr] - y[:npr]).max() / np.abs(y[:npr]).max(),
                   np.abs(x[npr:] - y[npr:]).max() / np.abs(y[npr:]).max())

    x0, _, om0 = solve()
    assert om0 <= 1e-15
    x1, _, _ = solve(ruiz=0)
    assert diff(x1, x0) < 1e-2
    xa, ita, oma = solve(eps=1e-7, tol=1e-10)
    assert ita == 0 and oma <= 1e-10 and diff(xa, x0) > 0.1
    xb, itb, omb = solve(eps=1e-7, tol=1e-15)
    assert itb > 0 and omb <= 1e-15 and diff(xb, x0) < 1e-2


def test_block_jacobi_precondition_pins():
    """Block-Jacobi sweeps with an exact substitution inside each block (the
    Gauss-Seidel end of Sec. V's iterative triangular solves): singleton
    blocks reproduce the point-Jacobi sweeps; one block is the exact solve
    after one sweep; with blocks of consecutive pivots, as many sweeps as the
    longest chain of blocks in the factors' dependencies give the exact solve,
    and fewer sweeps are closer to it than as many point sweeps; a mistake
    that keeps U's in-block entries in U_O as well (the diagonal counted
    twice) breaks the singleton pin."""
    import scipy.sparse as sp
    pat = KKTPattern(make_grid(3, 30, 40, 6))
    v = pat.values(pat.point(3, 0, 1e-1, delta_w=1.0, delta_c=1.0))
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an)
    f = lu.factors()
    b = pat.rhs(3, 0)
    n = pat.n
    exact = lu.solve_scaled(d, b)
    nrm = np.linalg.norm(exact)
    single = np.arange(n)
    for s in (1, 3):
        assert np.allclose(O.block_jacobi_precondition(f, d, b, s, single), O.jacobi_precondition(f, d, b, s),
                           rtol=1e-13, atol=1e-13 * np.abs(exact).max())
    one = O.block_jacobi_precondition(f, d, b, 1, np.zeros(n, dtype=np.int64))
    assert np.linalg.norm(one - exact) <= 1e-10 * nrm
    # blocks of 4 consecutive pivots (in the factors' order), numbered by unknown
    bpos = np.arange(n) // 4
    block_of = np.empty(n, dtype=np.int64)
    block_of[f.q] = bpos
    # longest chain of blocks: block a depends on block c if a nonzero of L (U) couples them
    L = sp.csc_matrix((f.Lx, f.Li, f.Lp), shape=(n, n)).tocoo()
    dep = {(int(bpos[r]), int(bpos[c])) for r, c, x in zip(L.row, L.col, L.data) if bpos[r] != bpos[c] and x != 0}
    nb = int(bpos.max()) + 1
    depth = np.ones(nb, dtype=np.int64)
    for a in range(nb):                                      # dependencies point to lower blocks
        for (x, y) in dep:
            if x == a:
                depth[a] = max(depth[a], depth[y] + 1)
    U = sp.csc_matrix((f.Ux, f.Ui, f.Up), shape=(n, n)).tocoo()
    depu = {(int(bpos[r]), int(bpos[c])) for r, c, x in zip(U.row, U.col, U.data) if bpos[r] != bpos[c] and x != 0}
    du = np.ones(nb, dtype=np.int64)
    for a in range(nb - 1, -1, -1):                          # upper: dependencies point to higher blocks
        for (x, y) in depu:
            if x == a:
                du[a] = max(du[a], du[y] + 1)
    s_full = int(max(depth.max(), du.max()))
    full = O.block_jacobi_precondition(f, d, b, s_full, block_of)
    assert np.linalg.norm(full - exact) <= 1e-10 * nrm
    # fewer sweeps: larger blocks absorb dependency chains, so the block sweeps
    # are closer to the exact solve than as many point sweeps
    for s in (2, 3):
        eb = np.linalg.norm(O.block_jacobi_precondition(f, d, b, s, block_of) - exact)
        ep = np.linalg.norm(O.jacobi_precondition(f, d, b, s) - exact)
        print("sweeps %d: block %.2e point %.2e (of %.2e)" % (s, eb, ep, nrm))
        assert eb < ep and ep > 1e-6 * nrm
    # the planted mistake, in the oracle: U's in-block entries also kept in U_O
    real = O._block_parts

    def wrong(f_, block_of_):
        LD, LO, UD, UO = real(f_, block_of_)
        return LD, LO, UD, (UO + UD).tocsr()
    good = O.block_jacobi_precondition(f, d, b, 2, single)
    O._block_parts = wrong
    try:
        bad = O.block_jacobi_precondition(f, d, b, 2, single)
    finally:
        O._block_parts = real
    assert np.allclose(good, O.jacobi_precondition(f, d, b, 2), rtol=1e-13, atol=1e-13 * np.abs(exact).max())
    assert not np.allclose(bad, O.jacobi_precondition(f, d, b, 2), rtol=1e-6)
