"""The allocation-free backward-error entry point against the context-based
one (kkt_residual): same residual and omega on two calls in a row.

It exists for callers that cannot allocate device memory when they need the
check (a framework owning all device memory, a fixed-budget serving loop, or
no analysis context yet); its scratch is a fixed array the library declares
in device memory. Collected last on purpose (file name), so that a run that
stops at the first failure has run every other test before it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid


def test_noalloc_backward_error_matches_context_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    pat = KKTPattern(make_grid(1, 1000, 1280, 200))
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


def test_noalloc_rejects_too_many_rows_and_null_pointers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = K._native.lib()
    assert lib.kkt_backward_error_noalloc(8_388_609, 1, 1, 1, 1, 1, 1, 1, None) == 1
    assert lib.kkt_backward_error_noalloc(10, None, 1, 1, 1, 1, 1, 1, None) == 1
    assert lib.kkt_backward_error_noalloc(0, 1, 1, 1, 1, 1, 1, 1, None) == 1
