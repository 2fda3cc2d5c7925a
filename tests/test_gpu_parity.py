"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

* equilibration factors: bitwise equal (power-of-two arithmetic is exact);
* factors, entrywise: |f_gpu - f_ora| <= eb_gpu + eb_ora, where eb is the
  first-order running error bound of each entry (Wilkinson's running error
  analysis of the left-looking elimination, computed by the oracle for a
  format of unit roundoff u: 2^-53 for FP64, 2^-24 for the FP32 path). Both
  computations lie within eb of the exact factors of the same D K D, so they
  lie within the sum of each other. The bound holds for any summation order,
  so it covers the GPU's multifrontal grouping of the same updates;
* a pivot with |u_jj| < 1e-10 (|L||U|)_jj is rounding noise (cancellation of
  terms 1e10 times larger than the result; the angle-shift direction of K is
  held only by dw): first-order analysis does not apply to it or to what
  depends on it -- its own value, its L column and the rows and columns of its
  elimination-tree ancestors -- so those entries are checked through the
  solution's backward error instead (in FP32 the noise is large enough that
  the two sides may even decide its static perturbation differently);
* static-pivot decisions identical on every determined pivot;
* amalgamation zeros stored by the GPU are exactly 0;
* solve / refine: normwise backward error omega on the unscaled K.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def compare_factors(f, gpu, floor, eb, noise_rel=1e-10, gfloor=None):
    """Entrywise comparison of the GPU factors with the oracle's (keyed by
    original indices) against per-entry tolerances eb = (ebL, ebU) aligned
    with the oracle's Lx / Ux. floor / gfloor: the static-pivot value of the
    oracle / of the GPU (the same FP64 floor, rounded once to FP32 for FP32
    factors). Where the two sides decide a pivot differently, the side that
    kept its pivot must hold it further than the pivot's bound from the floor
    to count as a mismatch: closer, either decision is consistent with the
    data. Returns (worst L error / tol, worst U error / tol,
    perturbation-decision mismatches on determined pivots, noise pivots,
    entries compared, entries total, pivots left undecided)."""
    gfloor = floor if gfloor is None else gfloor
    n = f.n
    lr, lc, lv, ur, uc, uv = gpu
    ebL, ebU = eb
    Labs = sp.csc_matrix((np.abs(f.Lx), f.Li, f.Lp), shape=(n, n)) + sp.identity(n, format="csc")
    Uabs = sp.csc_matrix((np.abs(f.Ux), f.Ui, f.Up), shape=(n, n))
    Sd = np.asarray((Labs @ Uabs).diagonal()).ravel()
    udiag = f.Ux[f.Up[1:] - 1]
    noise = np.abs(udiag) < noise_rel * Sd
    parent = np.full(n, -1)
    has = np.diff(f.Lp) > 0
    parent[has] = np.minimum.reduceat(f.Li, f.Lp[:-1][has])
    anc = np.zeros(n, bool)                       # strict ancestors of noise pivots
    for p in np.nonzero(noise)[0]:
        q = parent[p]
        while q >= 0 and not anc[q]:
            anc[q] = True
            q = parent[q]
    lcol = np.repeat(np.arange(n), np.diff(f.Lp))
    ucol = np.repeat(np.arange(n), np.diff(f.Up))

    def lookup(rows, cols, grow, gcol, gval, what):
        okey = rows.astype(np.int64) * n + cols
        gkey = grow.astype(np.int64) * n + gcol
        order = np.argsort(gkey)
        gk, gv = gkey[order], gval[order]
        assert np.unique(gk).size == gk.size, what + ": duplicate GPU entries"
        pos = np.searchsorted(gk, okey)
        ok = (pos < gk.size) & (gk[np.minimum(pos, gk.size - 1)] == okey)
        assert np.all(ok), what + ": oracle entry missing on the GPU"
        extra = np.ones(gk.size, bool)
        extra[pos] = False
        assert np.all(gv[extra] == 0.0), what + ": nonzero outside the structure"
        return gv[pos]

    gL = lookup(f.p[f.Li], f.q[lcol], lr, lc, lv, "L")
    gU = lookup(f.p[f.Ui], f.q[ucol], ur, uc, uv, "U")
    mL = ~(anc[lcol] | noise[lcol])
    ndiag = np.zeros(f.Ux.size, bool)              # a noise pivot's own value is rounding noise too
    ndiag[(f.Up[1:] - 1)[noise]] = True
    mU = ~(anc[f.Ui] | ndiag)
    eL = np.abs(gL - f.Lx)[mL] / np.maximum(ebL[mL], 1e-300)
    eU = np.abs(gU - f.Ux)[mU] / np.maximum(ebU[mU], 1e-300)
    gdiag = gU[f.Up[1:] - 1]
    det = ~(anc | noise)
    po = np.abs(udiag) == floor
    pg = np.abs(gdiag) == gfloor
    kept = np.where(po, np.abs(gdiag), np.abs(udiag))          # the value of the side that did not perturb
    undecided = (po != pg) & (np.abs(kept - floor) <= ebU[f.Up[1:] - 1] + abs(gfloor - floor))
    mism = int(np.sum((po != pg) & det & ~undecided))
    return (float(eL.max()) if eL.size else 0.0, float(eU.max()) if eU.size else 0.0, mism,
            int(noise.sum()), int(mL.sum() + mU.sum()), int(f.Lx.size + f.Ux.size), int(undecided.sum()))


@pytest.fixture(scope="module")
def grid200():
    return KKTPattern(make_grid(1, 200, 300, 40))


def test_ruiz_scaling_is_bitwise_equal(grid200):
    pat = grid200
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 4)):
        v = pat.values(pat.point(1, k, mu))
        s.refactor(_t(v))
        torch.cuda.synchronize()
        d_gpu = s.scaling()
        d_ora, _ = O.ruiz(pat.rowptr, pat.colidx, v, 10)
        assert np.array_equal(d_gpu, d_ora)
    s.close()


def test_ruiz_scaling_bitwise_over_wide_magnitudes(grid200):
    """Symmetric row/column factors 10^U(-75, 75) spread |k| over ~300 decades:
    many iterations change d (all after the first run on exponent keys) and the
    result still equals the oracle's bit for bit."""
    pat = grid200
    rng = np.random.default_rng(11)
    sc = 10.0 ** rng.uniform(-75, 75, size=pat.n)
    rows = np.repeat(np.arange(pat.n), np.diff(pat.rowptr))
    v = pat.values(pat.point(1, 2, 1e-3)) * sc[rows] * sc[pat.colidx]
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    s.refactor(_t(v))
    torch.cuda.synchronize()
    d_ora, it = O.ruiz(pat.rowptr, pat.colidx, v, 10)
    assert it >= 4
    assert np.array_equal(s.scaling(), d_ora)
    s.close()


def test_ruiz_scaling_bitwise_with_a_subnormal_entry(grid200):
    """A subnormal entry (in a row whose maximum is a normal entry) sends every
    iteration down the by-values path; d still equals the oracle's."""
    pat = grid200
    v = pat.values(pat.point(1, 1, 1e-2)).copy()
    i = 7
    lo, hi = pat.rowptr[i], pat.rowptr[i + 1]
    q = lo + int(np.argmin(np.abs(v[lo:hi])))                  # not the row maximum
    j = pat.colidx[q]
    v[q] = 1e-310
    qs = pat.rowptr[j] + int(np.searchsorted(pat.colidx[pat.rowptr[j]:pat.rowptr[j + 1]], i))
    v[qs] = 1e-310                                              # keep K symmetric
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    s.refactor(_t(v))
    torch.cuda.synchronize()
    d_ora, _ = O.ruiz(pat.rowptr, pat.colidx, v, 10)
    assert np.array_equal(s.scaling(), d_ora)
    s.close()


def _parity_case(pat, seed, steps, precision="fp64", point_kw=None, clip_sigma=None):
    v0 = pat.values(pat.point(seed, 0, 1e-1, **(point_kw or {})))
    an = O.analyze(pat.rowptr, pat.colidx, v0)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, user_perm=an.q, precision=precision)
    eps = 1e-14 if precision == "fp64" else 1e-7
    u_gpu = 2.0 ** -53 if precision == "fp64" else 2.0 ** -24
    out = []
    for k, mu in enumerate(mu_schedule(1e-1, 1e-8, steps)):
        pt = pat.point(seed, k, mu, **(point_kw or {}))
        if clip_sigma:
            pt.sigma = np.where(pt.sigma > 0, np.clip(pt.sigma, *clip_sigma), 0.0)
        v = pat.values(pt)
        lu, d, sv = O.refactor(pat.rowptr, pat.colidx, v, an, pivot_eps=eps)
        f = lu.factors()
        floor = eps * np.abs(sv).max()
        s.refactor(_t(v))
        torch.cuda.synchronize()
        bL64, bU64 = lu.error_bound(pat.rowptr, pat.colidx, sv, 2.0 ** -53, floor)
        bLg, bUg = lu.error_bound(pat.rowptr, pat.colidx, sv, u_gpu, floor)
        gfloor = floor if precision == "fp64" else float(np.float32(floor))
        eL, eU, mism, nnoise, ncmp, ntot, nund = compare_factors(f, s.export_factors(), floor,
                                                                 (bL64 + bLg, bU64 + bUg), gfloor=gfloor)
        b = pat.rhs(seed, k)
        x = s.solve(_t(b))
        torch.cuda.synchronize()
        om = O.backward_error(pat.rowptr, pat.colidx, v, x.cpu().numpy(), b)
        xo = lu.solve_scaled(d, b)
        om_o = O.backward_error(pat.rowptr, pat.colidx, v, xo, b)
        info = s.info()
        print("step %d: factor err/tol L %.2e U %.2e  compared %d of %d  noise pivots %d  pert mismatches %d  "
              "undecided pivots %d  perturbed gpu %d oracle %d  omega gpu %.2e oracle %.2e"
              % (k, eL, eU, ncmp, ntot, nnoise, mism, nund, info.n_perturbed, f.n_perturbed, om, om_o))
        out.append(dict(eL=eL, eU=eU, mism=mism, om=om, om_o=om_o, pg=info.n_perturbed, po=f.n_perturbed,
                        noise=nnoise, undecided=nund))
    s.close()
    return out


def _assert_parity(r, omega=1e-12):
    assert r["eL"] <= 1.0 and r["eU"] <= 1.0, r
    assert r["mism"] == 0, r
    # the unrefined solve is as backward stable as the oracle's
    assert r["om"] <= max(omega, 10.0 * r["om_o"]), r


def test_fp64_factors_match_oracle_200bus(grid200):
    for r in _parity_case(grid200, 1, 10):
        _assert_parity(r)
        assert r["om_o"] <= 1e-12


@pytest.mark.parametrize("B,L,G,seed", [(2, 1, 1, 3), (5, 6, 2, 4), (37, 50, 8, 5), (1000, 1280, 200, 6)])
def test_fp64_factors_match_oracle_sizes(B, L, G, seed):
    """Degenerate (2 buses), tiny, ragged and multi-tile cases."""
    pat = KKTPattern(make_grid(seed, B, L, G))
    for r in _parity_case(pat, seed, 3):
        _assert_parity(r)


def test_fp64_factors_match_oracle_25k():
    """Full size of the 25,000-bus workload (panel fronts and tiled Schur
    updates included), every determined factor entry."""
    pat = KKTPattern(make_grid(1, 25_000, 32_000, 5_000))
    for r in _parity_case(pat, 1, 2):
        _assert_parity(r)


def test_fp64_factors_bounded_growth_25k():
    """Same 25k structure with well-conditioned values: no noise pivots, so
    every entry is compared."""
    pat = KKTPattern(make_grid(2, 25_000, 32_000, 5_000))
    for r in _parity_case(pat, 2, 1, point_kw=dict(delta_w=1.0, delta_c=1.0), clip_sigma=(0.1, 10.0)):
        _assert_parity(r)
        assert r["noise"] == 0


def test_fp32_factors_close_to_fp64_oracle():
    """FP32 factors (FP32 accumulation) against the FP64 oracle: the same
    entrywise rule with the FP32 unit roundoff for the GPU side."""
    pat = KKTPattern(make_grid(2, 200, 300, 40))
    for r in _parity_case(pat, 2, 2, precision="fp32", point_kw=dict(delta_w=1.0, delta_c=1.0),
                          clip_sigma=(0.1, 10.0)):
        assert r["eL"] <= 1.0 and r["eU"] <= 1.0, r
        assert r["pg"] == 0 and r["po"] == 0


@pytest.mark.parametrize("B,L,G,seed,steps", [(200, 300, 40, 2, 4), (25_000, 32_000, 5_000, 1, 2)])
def test_fp32_factors_against_fp64_oracle_on_graded_values(B, L, G, seed, steps):
    """FP32 factors on the graded inputs themselves: literal dw = 1e-8 and
    dc = 1e-10, Sigma log-uniform over [1e-8, 1e8] down the mu schedule, static
    pivots at eps = 1e-7 on both sides. Every determined entry lies within the
    sum of the FP64 and FP32 running error bounds of the oracle's, and every
    static-pivot decision agrees except where the oracle's pivot lies within
    that bound of the floor (either decision is then consistent with the
    data)."""
    pat = KKTPattern(make_grid(seed, B, L, G))
    res = _parity_case(pat, seed, steps, precision="fp32")
    for r in res:
        assert r["eL"] <= 1.0 and r["eU"] <= 1.0, r
        assert r["mism"] == 0, r
    assert sum(r["po"] for r in res) > 0          # the graded values do meet the floor


def test_fp32_error_per_result_and_refinement(grid200):
    """Per result: ||x32 - x64|| / ||x64|| before and after refinement, and omega."""
    pat = grid200
    v0 = pat.values(pat.point(1, 0, 1e-1))
    an = O.analyze(pat.rowptr, pat.colidx, v0)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, user_perm=an.q, precision="fp32")
    for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 5)):
        v = pat.values(pat.point(1, k, mu))
        b = pat.rhs(1, k)
        lu, d, _ = O.refactor(pat.rowptr, pat.colidx, v, an)
        x64, _, om64 = O.fgmres(pat.rowptr, pat.colidx, v, lu, d, b, 30, 10, 1e-14)
        s.refactor(_t(v))
        x0 = s.solve(_t(b)).cpu().numpy()
        x1, info = s.refine(_t(b), tol=1e-10)
        x1 = x1.cpu().numpy()
        om0 = O.backward_error(pat.rowptr, pat.colidx, v, x0, b)
        om1 = O.backward_error(pat.rowptr, pat.colidx, v, x1, b)
        e0 = np.linalg.norm(x0 - x64) / np.linalg.norm(x64)
        e1 = np.linalg.norm(x1 - x64) / np.linalg.norm(x64)
        print("step %d: fp32 solve: err %.2e omega %.2e | refined: err %.2e omega %.2e iters %d"
              % (k, e0, om0, e1, om1, info.iters))
        assert om1 <= 1e-10
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
def test_refine_reaches_backward_error(grid200, precision, tol):
    pat = grid200
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision)
    for k, mu in enumerate(mu_schedule(1e-1, 1e-8, 10)):
        v = pat.values(pat.point(1, k, mu))
        b = pat.rhs(1, k)
        s.refactor(_t(v))
        x, info = s.refine(_t(b), tol=tol)
        om = O.backward_error(pat.rowptr, pat.colidx, v, x.cpu().numpy(), b)
        # both evaluations of omega (GPU, oracle) meet the tolerance; they are
        # not compared with each other: at omega ~ 1e-17 the residual is
        # rounding noise whose value depends on the summation order
        assert om <= tol and info.backward_err <= tol
    s.close()


def test_solve_matches_numpy_on_well_conditioned_system():
    pat = KKTPattern(make_grid(3, 30, 40, 6))
    v = pat.values(pat.point(3, 0, 1e-1, delta_w=1.0, delta_c=1.0))
    b = pat.rhs(3, 0)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    s.refactor(_t(v))
    x = s.solve(_t(b)).cpu().numpy()
    xr = np.linalg.solve(pat.to_scipy(v).toarray(), b)
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)
    s.close()


def test_residual_matches_oracle(grid200):
    pat = grid200
    v = pat.values(pat.point(1, 3, 1e-3))
    rng = np.random.default_rng(0)
    x, b = rng.normal(size=pat.n), rng.normal(size=pat.n)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    s.refactor(_t(v))
    r, om = s.residual(_t(b), _t(x))
    ro = O.spmv_resid(pat.rowptr, pat.colidx, v, x, b)
    scale = (abs(pat.to_scipy(v)) @ np.abs(x) + np.abs(b)).max()
    assert np.abs(r.cpu().numpy() - ro).max() <= 1e-13 * scale
    assert om == pytest.approx(O.backward_error(pat.rowptr, pat.colidx, v, x, b), rel=1e-10)
    s.close()


def test_static_perturbation_on_zero_pivot():
    """A 2x2 saddle point [[0, 1], [1, 0]]: the first pivot is exactly 0 and is
    replaced by +eps*max|A|; refinement still solves the system."""
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    v = np.array([0.0, 1.0, 1.0, 0.0])
    s = K.KKTSolver(rp, ci, 1, ordering="natural")
    s.refactor(_t(v))
    torch.cuda.synchronize()
    assert s.info().n_perturbed == 1
    b = np.array([2.0, 3.0])
    x, info = s.refine(_t(b), tol=1e-14)
    assert np.allclose(x.cpu().numpy(), [3.0, 2.0], rtol=1e-12)
    s.close()


def test_call_order_errors():
    pat = KKTPattern(make_grid(1, 10, 12, 2))
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    b = _t(np.ones(pat.n))
    with pytest.raises(K.KKTError) as e:
        s.solve(b)
    assert e.value.status == 4
    s.close()


def test_host_step_equals_device_path(grid200):
    pat = grid200
    v = pat.values(pat.point(1, 2, 1e-4))
    b = pat.rhs(1, 2)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    xh, info = s.step_host(v, b, tol=1e-12)
    s.refactor(_t(v))
    xd, _ = s.refine(_t(b), tol=1e-12)
    assert np.array_equal(xh, xd.cpu().numpy())
    assert O.backward_error(pat.rowptr, pat.colidx, v, xh, b) <= 1e-12
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_eastern70k_backward_error_through_the_timed_call(precision):
    """Full size of the 70,000-bus workload through kkt_refactor_refine (the call
    the benchmark times): the oracle's normwise backward error of the returned
    x, computed on the host from K and b alone, meets the 1e-10 tolerance, and
    the library's own figure (a different summation order of the residual)
    meets it too."""
    from kktgen import WORKLOADS
    w = WORKLOADS["eastern70k"]
    pat = KKTPattern(make_grid(3, w["n_bus"], w["n_branch"], w["n_gen"]))
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision)
    for k, mu in ((0, 1e-1), (1, 1e-9)):
        v = pat.values(pat.point(3, k, mu))
        b = pat.rhs(3, k)
        x, info = s.refactor_refine(_t(v), _t(b), tol=1e-10)
        om = O.backward_error(pat.rowptr, pat.colidx, v, x.cpu().numpy(), b)
        assert info.status == 0
        assert om <= 1e-10, om
        assert info.backward_err <= 1e-10, info.backward_err
    s.close()


@pytest.mark.parametrize("bad,where", [(np.nan, "offdiag"), (np.inf, "diag"), (-np.inf, "offdiag")])
def test_nan_or_inf_in_k_reports_numeric(grid200, bad, where):
    """A NaN or Inf planted in K's values (a host-made input; nothing faults):
    the refactorization flags it (kkt_get_info status KKT_E_NUMERIC), refine
    returns KKT_E_NUMERIC instead of a solution, and the next refactorization
    with finite values runs normally on the same context."""
    pat = grid200
    v_ok = pat.values(pat.point(1, 0, 1e-1))
    v = v_ok.copy()
    i = 23
    lo, hi = pat.rowptr[i], pat.rowptr[i + 1]
    cols = pat.colidx[lo:hi]
    j = i if where == "diag" else int(cols[cols != i][0])
    v[lo + int(np.searchsorted(cols, j))] = bad
    v[pat.rowptr[j] + int(np.searchsorted(pat.colidx[pat.rowptr[j]:pat.rowptr[j + 1]], i))] = bad
    b = pat.rhs(1, 0)
    for precision in ("fp64", "fp32"):
        s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision)
        s.refactor(_t(v))
        torch.cuda.synchronize()
        assert s.info().status == 8
        with pytest.raises(K.KKTError) as e:
            s.refine(_t(b), tol=1e-10)
        assert e.value.status == 8
        with pytest.raises(K.KKTError) as e:
            s.refactor_refine(_t(v), _t(b), tol=1e-10)
        assert e.value.status == 8
        x, info = s.refactor_refine(_t(v_ok), _t(b), tol=1e-10)
        assert info.status == 0
        assert O.backward_error(pat.rowptr, pat.colidx, v_ok, x.cpu().numpy(), b) <= 1e-10
        s.close()


def test_nan_solution_is_never_reported_converged(grid200):
    """kkt_residual's omega of a NaN x is NaN (maxima on bit patterns), so a
    tolerance test on it fails."""
    pat = grid200
    v = pat.values(pat.point(1, 2, 1e-3))
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    s.refactor(_t(v))
    x = np.full(pat.n, np.nan)
    _, om = s.residual(_t(pat.rhs(1, 2)), _t(x))
    assert not (om <= 1e-10)
    s.close()
