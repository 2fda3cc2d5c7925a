"""Jacobi-sweep preconditioner (approximate triangular solves with the
factors, Sec. V) on the GPU against the oracle's plain restatement of the
same sweeps (oracle.jacobi_precondition), and as the preconditioner of the
FGMRES refinement.

Point-Jacobi sweeps do not depend on the elimination order beyond the
factors themselves, so the library's postordered factors and the oracle's
factors of the same order give the same operator. Tolerance, derived from the
arithmetic: the two factorizations differ entrywise by at most eb_gpu +
eb_ora (the oracle's first-order running error bounds, as in the factor
parity tests), and every sweep adds the rounding of a sum of at most n_row
products. Carried to first order through the sweeps,
  e_y <- E_L |y| + |L - I| e_y + g (|L - I| |y| + |c|),
  e_x <- (e_y + E_U |x| + |U - D| e_x + g (|U - D| |x| + |y|)) / |D| + |x| E_D / |D|,
with E_L, E_U, E_D the bounds of L - I, U - D and D, and g = 64 u; the
results must agree within D e_x entrywise (in the original index space).
After one sweep this bound is sharp (most entries within ~1e-14 relative);
over more sweeps worst-case growth makes it loose, so the sweeps themselves
are pinned by a fixed-point property instead: L - I and U - diag(U) are
nilpotent, so n sweeps must reproduce the exact triangular solves (which
test_gpu_parity.py compares with the oracle) -- an entry of the factors that
a sweep missed, doubled or misplaced breaks it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid, mu_schedule


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(_dev())


@pytest.mark.parametrize("sweeps", [1])
@pytest.mark.parametrize("B,L,G,seed", [(200, 300, 40, 1), (37, 50, 8, 5)])
def test_jacobi_sweeps_match_oracle(sweeps, B, L, G, seed):
    pat = KKTPattern(make_grid(seed, B, L, G))
    pt = pat.point(seed, 0, 1e-1, delta_w=1.0, delta_c=1.0)
    pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, 0.1, 10.0), 0.0)
    v = pat.values(pt)
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an)
    b = pat.rhs(seed, 0)
    f = lu.factors()
    ref = O.jacobi_precondition(f, d, b, sweeps)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, user_perm=an.q, precond="jacobi",
                    jacobi_sweeps=sweeps)
    s.refactor(_t(v))
    z = s.precondition(_t(b)).cpu().numpy()
    tol = _sweep_bound(pat, lu, f, sv, d, b, sweeps)
    assert np.all(np.abs(z - ref) <= tol), float(np.max(np.abs(z - ref) / np.maximum(tol, 1e-300)))
    s.close()


def _sweep_bound(pat, lu, f, sv, d, b, sweeps):
    import scipy.sparse as sp
    n = f.n
    u = 2.0 ** -53
    g = 64 * u
    floor = 1e-14 * np.abs(sv).max()
    eL, eU = lu.error_bound(pat.rowptr, pat.colidx, sv, u, floor)
    eL, eU = 2 * eL, 2 * eU                                  # gpu + oracle
    Ls = sp.csc_matrix((f.Lx, f.Li, f.Lp), shape=(n, n)).tocsr()
    EL = sp.csc_matrix((eL, f.Li, f.Lp), shape=(n, n)).tocsr()
    U = sp.csc_matrix((f.Ux, f.Ui, f.Up), shape=(n, n))
    EUf = sp.csc_matrix((eU, f.Ui, f.Up), shape=(n, n))
    du = U.diagonal()
    ed = EUf.diagonal()
    Us = (U - sp.diags(du)).tocsr()
    EU = (EUf - sp.diags(ed)).tocsr()
    aL, aU = abs(Ls), abs(Us)
    c = (d * b)[f.p]
    y = np.zeros(n)
    ey = np.zeros(n)
    for _ in range(sweeps):
        ey = EL @ np.abs(y) + aL @ ey + g * (aL @ np.abs(y) + np.abs(c))
        y = c - Ls @ y
    x = np.zeros(n)
    ex = np.zeros(n)
    for _ in range(sweeps):
        xn = (y - Us @ x) / du
        ex = (ey + EU @ np.abs(x) + aU @ ex + g * (aU @ np.abs(x) + np.abs(y))) / np.abs(du) + np.abs(xn) * ed / np.abs(du)
        x = xn
    e = np.empty(n)
    e[f.q] = ex
    return np.asarray(d) * e



@pytest.mark.parametrize("B,L,G,seed", [(30, 40, 6, 3), (37, 50, 8, 5)])
def test_enough_sweeps_give_the_exact_solve(B, L, G, seed):
    pat = KKTPattern(make_grid(seed, B, L, G))
    pt = pat.point(seed, 0, 1e-1, delta_w=1.0, delta_c=1.0)
    pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, 0.1, 10.0), 0.0)
    v = pat.values(pt)
    b = pat.rhs(seed, 0)
    ex = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    ex.refactor(_t(v))
    x = ex.solve(_t(b)).cpu().numpy()
    jac = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precond="jacobi", jacobi_sweeps=pat.n)
    jac.refactor(_t(v))
    z = jac.precondition(_t(b)).cpu().numpy()
    assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)
    ex.close()
    jac.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fgmres_with_jacobi_preconditioner(precision):
    """Refinement preconditioned by the sweeps. With as many sweeps as
    unknowns the preconditioner is the exact solve and the refinement meets
    the tolerance at once. With few sweeps the sweeps of these factors do not
    make a useful preconditioner (measured: FGMRES(30) with 10 restarts stalls
    even on a well-conditioned 200-bus system), and the call must say so:
    KKT_E_NOCONV with the omega it reached, and the omega is the oracle's."""
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    pt = pat.point(1, 0, 1e-1, delta_w=1.0, delta_c=1.0)
    pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, 0.1, 10.0), 0.0)
    v = pat.values(pt)
    b = pat.rhs(1, 0)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision, precond="jacobi",
                    jacobi_sweeps=pat.n)
    s.refactor(_t(v))
    x, info = s.refine(_t(b), tol=1e-10)
    assert O.backward_error(pat.rowptr, pat.colidx, v, x.cpu().numpy(), b) <= 1e-10
    s.close()
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision, precond="jacobi", jacobi_sweeps=8,
                    max_cycles=2)
    for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 3)):
        vk = pat.values(pat.point(1, k, mu))
        bk = pat.rhs(1, k)
        s.refactor(_t(vk))
        xk, ik = s.refine(_t(bk), tol=1e-10, raise_on_noconv=False)
        omk = O.backward_error(pat.rowptr, pat.colidx, vk, xk.cpu().numpy(), bk)
        print("mu %.0e: 8 Jacobi sweeps, FGMRES iters %d omega %.2e" % (mu, ik.iters, omk))
        assert ik.iters > 0
        assert omk <= 1e-10 or ik.backward_err > 1e-10
        assert ik.backward_err == pytest.approx(omk, rel=1e-2, abs=1e-14)
    s.close()


# ---- block-Jacobi sweeps (each front's pivots a block, exact inside the sweep)

def _fronts_of(pat, s, q):
    """Block of every unknown: the library's fronts (host analysis,
    kkt_plan_fronts, in step order) mapped through its step permutation."""
    _, w = K.plan_fronts(pat.rowptr, pat.colidx, user_perm=q)
    perm = s.perm()                                          # step -> unknown
    block_of = np.empty(pat.n, dtype=np.int64)
    block_of[perm] = np.repeat(np.arange(w.size), w)
    return block_of


def _block_bound(pat, lu, f, sv, d, b, block_of):
    """First-order bound of |GPU - oracle| for one block sweep per factor,
    y = L_D^{-1} c, x = U_D^{-1} y, block by block: with E the sum of both
    factorizations' running error bounds and g = 64 u for the rounding of a
    substitution of at most 64 pivots (reciprocal and product included),
      e_y = |L_D^{-1}| (E_L |y| + g (|L_D| |y| + |c|)),
      e_x = |U_D^{-1}| (e_y + E_U |x| + g (|U_D| |x| + |y|)),
    the blocks' inverses formed densely; in the original numbering, times d."""
    import scipy.sparse as sp
    n = f.n
    u = 2.0 ** -53
    g = 64 * u
    floor = 1e-14 * np.abs(sv).max()
    eL, eU = lu.error_bound(pat.rowptr, pat.colidx, sv, u, floor)
    L = (sp.csc_matrix((f.Lx, f.Li, f.Lp), shape=(n, n)) + sp.eye(n)).tocsr()
    EL = sp.csc_matrix((2 * eL, f.Li, f.Lp), shape=(n, n)).tocsr()
    U = sp.csc_matrix((f.Ux, f.Ui, f.Up), shape=(n, n)).tocsr()
    EU = sp.csc_matrix((2 * eU, f.Ui, f.Up), shape=(n, n)).tocsr()
    blk = np.asarray(block_of)[f.q]
    c = (d * b)[f.p]
    y, ey, x, ex = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    order = np.argsort(blk, kind="stable")
    bounds = np.flatnonzero(np.diff(blk[order])) + 1
    for idx in np.split(order, bounds):
        idx = np.sort(idx)
        Lk, ELk = L[idx][:, idx].toarray(), EL[idx][:, idx].toarray()
        Uk, EUk = U[idx][:, idx].toarray(), EU[idx][:, idx].toarray()
        y[idx] = np.linalg.solve(Lk, c[idx])
        ey[idx] = np.abs(np.linalg.inv(Lk)) @ (ELk @ np.abs(y[idx]) + g * (np.abs(Lk) @ np.abs(y[idx]) + np.abs(c[idx])))
        x[idx] = np.linalg.solve(Uk, y[idx])
        ex[idx] = np.abs(np.linalg.inv(Uk)) @ (ey[idx] + EUk @ np.abs(x[idx]) +
                                               g * (np.abs(Uk) @ np.abs(x[idx]) + np.abs(y[idx])))
    e = np.empty(n)
    e[f.q] = ex
    return np.asarray(d) * e


@pytest.mark.parametrize("B,L,G,seed", [(200, 300, 40, 1), (37, 50, 8, 5)])
def test_block_jacobi_sweep_matches_oracle(B, L, G, seed):
    pat = KKTPattern(make_grid(seed, B, L, G))
    pt = pat.point(seed, 0, 1e-1, delta_w=1.0, delta_c=1.0)
    pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, 0.1, 10.0), 0.0)
    v = pat.values(pt)
    an = O.analyze(pat.rowptr, pat.colidx, v)
    lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an)
    b = pat.rhs(seed, 0)
    f = lu.factors()
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, user_perm=an.q, precond="block", jacobi_sweeps=1)
    s.refactor(_t(v))
    block_of = _fronts_of(pat, s, an.q)
    ref = O.block_jacobi_precondition(f, d, b, 1, block_of)
    z = s.precondition(_t(b)).cpu().numpy()
    tol = _block_bound(pat, lu, f, sv, d, b, block_of)
    assert np.all(np.abs(z - ref) <= tol), float(np.max(np.abs(z - ref) / np.maximum(tol, 1e-300)))
    # one block sweep is not one point sweep (the fronts hold more than one
    # pivot): the two differ beyond the bound on a large share of the entries
    apart = np.abs(ref - O.jacobi_precondition(f, d, b, 1)) > tol
    print("bound median %.1e of |z|, block vs point apart on %d of %d entries"
          % (np.median(tol / np.maximum(np.abs(ref), 1e-300)), apart.sum(), pat.n))
    assert apart.sum() > pat.n // 10
    s.close()


@pytest.mark.parametrize("B,L,G,seed", [(30, 40, 6, 3), (200, 300, 40, 1)])
def test_block_sweeps_reach_the_exact_solve_sooner(B, L, G, seed):
    """As many block sweeps as the assembly tree has levels reproduce the
    exact GPU solve (a front depends only on fronts of lower levels in L and
    of higher levels in U); point sweeps need as many as the longest
    dependency chain of single pivots."""
    pat = KKTPattern(make_grid(seed, B, L, G))
    pt = pat.point(seed, 0, 1e-1, delta_w=1.0, delta_c=1.0)
    pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, 0.1, 10.0), 0.0)
    v = pat.values(pt)
    b = pat.rhs(seed, 0)
    ex = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    ex.refactor(_t(v))
    x = ex.solve(_t(b)).cpu().numpy()
    levels = ex.plan()["n_levels"]
    blk = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precond="block", jacobi_sweeps=levels)
    blk.refactor(_t(v))
    z = blk.precondition(_t(b)).cpu().numpy()
    assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)
    pj = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precond="jacobi", jacobi_sweeps=levels)
    pj.refactor(_t(v))
    zp = pj.precondition(_t(b)).cpu().numpy()
    print("%d levels: block %.2e, point %.2e" % (levels, np.linalg.norm(z - x) / np.linalg.norm(x),
                                                 np.linalg.norm(zp - x) / np.linalg.norm(x)))
    assert np.linalg.norm(zp - x) > 1e3 * np.linalg.norm(z - x)
    for h in (ex, blk, pj):
        h.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fgmres_with_block_sweeps(precision):
    """Refinement preconditioned by block sweeps on the interior-point inputs
    of a 200-bus system (15 tree levels): with as many sweeps as levels the
    preconditioner is the exact solve and the tolerance is met at once; with
    4 sweeps FGMRES iterates, and the backward error it reports (met or not)
    is the oracle's."""
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    levels = K.plan(pat.rowptr, pat.colidx)["n_levels"]
    for sweeps in (levels, 4):
        s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision, precond="block",
                        jacobi_sweeps=sweeps)
        for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 3)):
            v = pat.values(pat.point(1, k, mu))
            b = pat.rhs(1, k)
            s.refactor(_t(v))
            x, info = s.refine(_t(b), tol=1e-10, raise_on_noconv=False)
            om = O.backward_error(pat.rowptr, pat.colidx, v, x.cpu().numpy(), b)
            print("%s mu %.0e: %d block sweeps, FGMRES iters %d omega %.2e" % (precision, mu, sweeps, info.iters, om))
            assert info.backward_err == pytest.approx(om, rel=1e-2, abs=1e-14)
            if sweeps == levels:
                assert om <= 1e-10 and info.iters <= (1 if precision == "fp64" else 30)
            else:
                assert info.iters > 0 and (om <= 1e-10 or info.backward_err > 1e-10)
        s.close()
