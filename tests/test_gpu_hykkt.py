"""The saddle-point specialised solve on the GPU (kkt_hykkt_*, Sec. V) against
the oracle (oracle/hykkt.py) and the direct solve of K: entrywise where K
determines the solution, by the backward error on the graded-like inputs,
and its error reports on host-made inputs."""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, KKTPoint, make_grid
from oracle import hykkt


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(_dev())


def _benign(pat, seed, step, dc=1e-3):
    p = pat.point(seed, step, 1e-3, delta_w=1.0, delta_c=dc, slack_range=(0.1, 10.0))
    sig = np.where(p.sigma > 0, np.clip(p.sigma, 0.1, 10.0), 0.0)
    return KKTPoint(p.V, p.theta, p.lam, sig, p.mu, p.delta_w, p.delta_c, p.slack_inv)


@pytest.mark.parametrize("gamma", [300.0, 900.0])
def test_matches_oracle_and_direct_solve_where_determined(gamma):
    pat = KKTPattern(make_grid(2, 120, 170, 24))
    mE = 2 * pat.grid.n_bus
    s = K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, mE, gamma=gamma)
    for step in range(3):
        v = pat.values(_benign(pat, 4, step))
        b = pat.rhs(4, step)
        Ks = pat.to_scipy(v)
        ref = spla.spsolve(Ks.tocsc(), b)
        o = hykkt.solve(Ks, pat.n_primal, mE, b, gamma, tol=1e-13, max_iter=2000)
        z, info = s.solve(_t(v), _t(b), tol=1e-13, max_iter=2000)
        z = z.cpu().numpy()
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(z - ref)) <= 1e-8 * scale
        assert np.max(np.abs(z - o.z)) <= 1e-8 * scale
        assert info.backward_err <= 1e-13 and hykkt.backward_error(Ks, z, b) <= 1e-13
        assert abs(info.cg_iters - o.cg_iters) <= 1          # same iteration, rounding apart
        assert info.status == 0 and info.cg_resid <= 1e-13
    pl = s.inner().plan()                       # the borrowed context factoring H_g
    assert pl["n"] == pat.n_primal and pl["nnz"] >= pat.n_primal
    s.close()


@pytest.mark.parametrize("buses,lines,gens,gamma", [(200, 300, 40, 1e4), (200, 300, 40, 1e8),
                                                     (25_000, 32_000, 5_000, 1e8), (70_000, 88_000, 10_000, 1e8)])
def test_graded_like_inputs_reach_the_backward_error(buses, lines, gens, gamma):
    """The interior-point form with the slacks' term (1/sigma_s on [1e-2, 1e2]),
    literal dw = 1e-8, dc = 1e-10, Sigma over [1e-8, 1e8]: omega <= 1e-10 for
    the whole K, as the oracle reaches on the same systems (200 buses)."""
    pat = KKTPattern(make_grid(1, buses, lines, gens))
    mE = 2 * pat.grid.n_bus
    s = K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, mE, gamma=gamma)
    for k, mu in enumerate([1e-1, 1e-5, 1e-8]):
        v = pat.values(pat.point(1, k, mu, slack_range=(1e-2, 1e2)))
        b = pat.rhs(1, k)
        z, info = s.solve(_t(v), _t(b), tol=1e-12, max_iter=500)
        om = hykkt.backward_error(pat.to_scipy(v), z.cpu().numpy(), b)
        print("%d buses, gamma %.0e, mu %.0e: %d CG iterations, omega %.2e (library %.2e)" % (buses, gamma, mu, info.cg_iters, om,
                                                                                 info.backward_err))
        assert om <= 1e-10 and info.backward_err == pytest.approx(om, rel=1e-3, abs=1e-18)
        if buses <= 200 and gamma <= 1e6:
            # the oracle's LU of H_g (unequilibrated, threshold pivoting) loses
            # about kappa(H_g) u, which grows with gamma: at 1e8 it ends near
            # 1e-10 on these systems, so it is held to the bound only below
            o = hykkt.solve(pat.to_scipy(v), pat.n_primal, mE, b, gamma, tol=1e-12, max_iter=500)
            assert o.omega <= 1e-10
    s.close()


def test_errors_on_host_made_inputs():
    dev = _dev()
    pat = KKTPattern(make_grid(2, 120, 170, 24))
    mE = 2 * pat.grid.n_bus
    v = pat.values(_benign(pat, 4, 0))
    b = pat.rhs(4, 0)
    # gamma d_E >= 1 (d_E = 1e-3): refused as numeric
    s = K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, mE, gamma=2000.0)
    with pytest.raises(K.KKTError) as e:
        s.solve(_t(v), _t(b))
    assert e.value.status == 8
    s.close()
    # too few iterations: KKT_E_NOCONV with the information filled
    s = K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, mE, gamma=300.0)
    z, info = s.solve(_t(v), _t(b), tol=1e-14, max_iter=2, raise_on_noconv=False)
    assert info.status == 6 and info.cg_iters == 2 and info.cg_resid > 1e-14
    with pytest.raises(K.KKTError) as e:
        s.solve(_t(v), _t(b), tol=1e-14, max_iter=2)
    assert e.value.status == 6
    s.close()
    # a (2,2) block that is not diagonal: refused by the analysis
    n = pat.n
    rp, ci = pat.rowptr.astype(np.int64), pat.colidx.astype(np.int64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    extra_r = np.array([pat.n_primal, pat.n_primal + 1])
    extra_c = np.array([pat.n_primal + 1, pat.n_primal])
    r2 = np.concatenate([rows, extra_r])
    c2 = np.concatenate([ci, extra_c])
    order = np.lexsort((c2, r2))
    r2, c2 = r2[order], c2[order]
    rp2 = np.concatenate([[0], np.cumsum(np.bincount(r2, minlength=n))]).astype(np.int32)
    with pytest.raises(K.KKTError) as e:
        K.SaddlePointSolver(rp2, c2.astype(np.int32), pat.n_primal, mE, gamma=300.0)
    assert e.value.status == 5
    # arguments
    with pytest.raises(ValueError):
        K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, 0)
    h = C.c_void_p()
    assert K._native.lib().kkt_hykkt_analyze(n, pat.n_primal, mE, None, None, 1.0, C.byref(h)) == 1
    s = K.SaddlePointSolver(pat.rowptr, pat.colidx, pat.n_primal, mE, gamma=300.0)
    bt, vt = _t(b), _t(v)
    with pytest.raises(ValueError):
        s.solve(vt, bt, out=bt)
    info = K._native.HykktInfo()
    assert K._native.lib().kkt_hykkt_solve(s._h, vt.data_ptr(), bt.data_ptr(), bt.data_ptr(), 1e-12, 10,
                                           C.byref(info), None) == 1
    s.close()
    del dev


def test_no_inequality_rows_on_the_device():
    """K without inequality rows (n = n_primal + m_eq): the device path with
    nothing to condense equals the direct solve and the oracle."""
    import scipy.sparse as sp
    pat = KKTPattern(make_grid(2, 120, 170, 24))
    mE = 2 * pat.grid.n_bus
    m = pat.n_primal + mE
    Ks = pat.to_scipy(pat.values(_benign(pat, 6, 1)))
    Ke = sp.csr_matrix(Ks[:m, :m])
    Ke.sort_indices()
    b = pat.rhs(6, 1)[:m]
    ref = spla.spsolve(Ke.tocsc(), b)
    o = hykkt.solve(Ke, pat.n_primal, mE, b, 300.0, tol=1e-13, max_iter=2000)
    s = K.SaddlePointSolver(Ke.indptr.astype(np.int32), Ke.indices.astype(np.int32), pat.n_primal, mE, gamma=300.0)
    z, info = s.solve(_t(Ke.data), _t(b), tol=1e-13, max_iter=2000)
    z = z.cpu().numpy()
    assert np.max(np.abs(z - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert np.max(np.abs(z - o.z)) <= 1e-8 * np.max(np.abs(ref))
    assert info.backward_err <= 1e-13 and abs(info.cg_iters - o.cg_iters) <= 1
    s.close()
