"""The allocation-free backward-error entry point against the context-based
one (kkt_residual): same residual and omega on two calls in a row.

It exists for callers that cannot allocate device memory when they need the
check (a framework owning all device memory, a fixed-budget serving loop, or
no analysis context yet); its scratch is a fixed array the library declares
in device memory. Collected last on purpose (file name), so that a run that
stops at the first failure has run every other test before it."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def grid1k():
    return KKTPattern(make_grid(1, 1000, 1280, 200))


def test_noalloc_backward_error_matches_context_path(grid1k):
    dev = _dev()
    pat = grid1k
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    rp = torch.from_numpy(pat.rowptr).to(dev)
    ci = torch.from_numpy(pat.colidx).to(dev)
    rng = np.random.default_rng(7)
    for call in range(2):
        v = pat.values(pat.point(3, call, 1e-2))
        vd = torch.from_numpy(v).to(dev)
        x = torch.from_numpy(rng.normal(size=pat.n)).to(dev)
        b = torch.from_numpy(rng.normal(size=pat.n)).to(dev)
        s.refactor(vd)
        r_ref, om_ref = s.residual(b, x)
        r = torch.full((pat.n,), np.nan, dtype=torch.float64, device=dev)
        om = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
        K.backward_error_noalloc(rp, ci, vd, x, b, r, om)
        torch.cuda.synchronize()
        rr = r.cpu().numpy()
        scale = (abs(pat.to_scipy(v)) @ np.abs(x.cpu().numpy()) + np.abs(b.cpu().numpy())).max()
        assert np.abs(rr - r_ref.cpu().numpy()).max() <= 1e-13 * scale
        assert float(om.item()) == pytest.approx(om_ref, rel=1e-12)
    s.close()


def test_noalloc_nan_in_x_gives_nan_omega_like_the_context_path(grid1k):
    """One NaN entry of x: omega is NaN on both paths (a NaN solution must not
    pass a tolerance test); the rows that do not touch that column keep their
    finite residual."""
    dev = _dev()
    pat = grid1k
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    v = pat.values(pat.point(3, 0, 1e-2))
    vd = torch.from_numpy(v).to(dev)
    rng = np.random.default_rng(8)
    xh = rng.normal(size=pat.n)
    j = pat.n // 3
    xh[j] = np.nan
    x = torch.from_numpy(xh).to(dev)
    b = torch.from_numpy(rng.normal(size=pat.n)).to(dev)
    s.refactor(vd)
    r_ref, om_ref = s.residual(b, x)
    assert math.isnan(om_ref)
    r = torch.zeros(pat.n, dtype=torch.float64, device=dev)
    om = torch.zeros(1, dtype=torch.float64, device=dev)
    K.backward_error_noalloc(torch.from_numpy(pat.rowptr).to(dev), torch.from_numpy(pat.colidx).to(dev),
                             vd, x, b, r, om)
    torch.cuda.synchronize()
    assert math.isnan(float(om.item()))
    rr = r.cpu().numpy()
    touches = np.zeros(pat.n, bool)
    rows = np.repeat(np.arange(pat.n), np.diff(pat.rowptr))
    touches[rows[pat.colidx == j]] = True
    assert np.all(np.isnan(rr[touches])) and np.all(np.isfinite(rr[~touches]))
    s.close()


def test_noalloc_checks_the_pattern_on_the_device(grid1k):
    """A column index outside [0, n) and a row pointer beyond nnz are caught by
    the kernel's own checks before any read: the affected rows get NaN, omega
    is NaN, the other rows are untouched, and the next valid call is exact."""
    dev = _dev()
    pat = grid1k
    v = pat.values(pat.point(3, 1, 1e-2))
    vd = torch.from_numpy(v).to(dev)
    rng = np.random.default_rng(9)
    x = torch.from_numpy(rng.normal(size=pat.n)).to(dev)
    b = torch.from_numpy(rng.normal(size=pat.n)).to(dev)
    rp_ok = torch.from_numpy(pat.rowptr).to(dev)
    ci_ok = torch.from_numpy(pat.colidx).to(dev)
    r = torch.zeros(pat.n, dtype=torch.float64, device=dev)
    om = torch.zeros(1, dtype=torch.float64, device=dev)

    ci_bad = pat.colidx.copy()
    row_c = 17
    ci_bad[pat.rowptr[row_c]] = pat.n + 5                       # column outside [0, n)
    K.backward_error_noalloc(rp_ok, torch.from_numpy(ci_bad).to(dev), vd, x, b, r, om)
    torch.cuda.synchronize()
    rr = r.cpu().numpy()
    assert math.isnan(float(om.item()))
    assert np.isnan(rr[row_c]) and np.isfinite(np.delete(rr, row_c)).all()

    rp_bad = pat.rowptr.copy()
    row_p = 40
    rp_bad[row_p + 1] = pat.nnz + 100                            # beyond nnz: rows 40 and 41 break the rule
    K.backward_error_noalloc(torch.from_numpy(rp_bad).to(dev), ci_ok, vd, x, b, r, om)
    torch.cuda.synchronize()
    rr = r.cpu().numpy()
    assert math.isnan(float(om.item()))
    assert np.isnan(rr[[row_p, row_p + 1]]).all() and np.isfinite(np.delete(rr, [row_p, row_p + 1])).all()

    K.backward_error_noalloc(rp_ok, ci_ok, vd, x, b, r, om)     # the scratch holds nothing stale
    torch.cuda.synchronize()
    assert np.isfinite(r.cpu().numpy()).all() and math.isfinite(float(om.item()))


def test_noalloc_rejects_too_many_rows_and_null_pointers():
    _dev()
    lib = K._native.lib()
    assert lib.kkt_backward_error_noalloc(8_388_609, 1, 1, 1, 1, 1, 1, 1, 1, None) == 1
    assert lib.kkt_backward_error_noalloc(10, 1, None, 1, 1, 1, 1, 1, 1, None) == 1
    assert lib.kkt_backward_error_noalloc(0, 1, 1, 1, 1, 1, 1, 1, 1, None) == 1
    assert lib.kkt_backward_error_noalloc(10, -1, 1, 1, 1, 1, 1, 1, 1, None) == 1
