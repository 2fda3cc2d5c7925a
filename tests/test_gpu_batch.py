"""Batched refactorization: instances sharing one pattern in one launch per
level, and several different contexts refactored concurrently. Every batched
result must equal, bit for bit, the result of the same instance processed
alone (the kernels are deterministic: fixed reduction and assembly orders)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-10)])
def test_batch_equals_single_instances(precision, tol):
    dev = _dev()
    pat = KKTPattern(make_grid(4, 2000, 2560, 400))
    B = 6
    vals = [pat.values(pat.point(100 + i, i, 10.0 ** -(1 + i))) for i in range(B)]
    rhs = [pat.rhs(100 + i, i) for i in range(B)]
    sb = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=B, precision=precision)
    vd = torch.from_numpy(np.concatenate(vals)).to(dev)
    bd = torch.from_numpy(np.concatenate(rhs)).to(dev)
    for _ in range(2):                                   # twice: graphs are captured on the first call
        sb.refactor(vd)
        xb, infos = sb.refine(bd, tol=tol)
    xb = xb.cpu().numpy().reshape(B, pat.n)
    single = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision)
    for i in range(B):
        single.refactor(torch.from_numpy(vals[i]).to(dev))
        xs, info = single.refine(torch.from_numpy(rhs[i]).to(dev), tol=tol)
        assert np.array_equal(xb[i], xs.cpu().numpy()), i
        assert infos[i].backward_err <= tol
        assert O.backward_error(pat.rowptr, pat.colidx, vals[i], xb[i], rhs[i]) <= tol
    sb.close()
    single.close()


def test_concurrent_contexts_equal_sequential():
    dev = _dev()
    pats = [KKTPattern(make_grid(5, 500, 640, 100)), KKTPattern(make_grid(6, 1500, 1920, 300))]
    ctxs = [K.KKTSolver(p.rowptr, p.colidx, p.n_primal) for p in pats]
    vals = [torch.from_numpy(p.values(p.point(7, 2, 1e-3))).to(dev) for p in pats]
    rhs = [torch.from_numpy(p.rhs(7, 2)).to(dev) for p in pats]
    outs = [torch.empty_like(b) for b in rhs]
    for _ in range(2):
        K.refactor_batched(ctxs, vals)
        K.solve_batched(ctxs, rhs, outs)
    torch.cuda.synchronize()
    for c, v, b, x in zip(ctxs, vals, rhs, outs):
        c.refactor(v)
        xs = c.solve(b)
        torch.cuda.synchronize()
        assert np.array_equal(x.cpu().numpy(), xs.cpu().numpy())
    for c in ctxs:
        c.close()


def test_full_batch_64x2k_equals_single_instances():
    """The 64 x 2,000-bus batch of the benchmark (FP32 factors + FP64 refinement;
    with 64 instances the tree threshold per instance drops to 38 fronts, a
    different schedule from a single context's): every instance meets the
    tolerance, and sampled instances equal single-context solves bit for bit
    and meet it by the oracle's own backward error."""
    dev = _dev()
    pat = KKTPattern(make_grid(8, 2000, 2560, 400))
    B, tol = 64, 1e-10
    vals = [pat.values(pat.point(200 + i, i % 7, 10.0 ** -(1 + i % 7))) for i in range(B)]
    rhs = [pat.rhs(200 + i, i % 7) for i in range(B)]
    sb = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=B, precision="fp32")
    vd = torch.from_numpy(np.concatenate(vals)).to(dev)
    bd = torch.from_numpy(np.concatenate(rhs)).to(dev)
    sb.refactor(vd)
    xb, infos = sb.refine(bd, tol=tol)
    xb = xb.cpu().numpy().reshape(B, pat.n)
    assert all(i.status == 0 and i.backward_err <= tol for i in infos)
    single = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision="fp32")
    for i in (0, 17, 38, 63):
        single.refactor(torch.from_numpy(vals[i]).to(dev))
        xs, info = single.refine(torch.from_numpy(rhs[i]).to(dev), tol=tol)
        assert np.array_equal(xb[i], xs.cpu().numpy()), i
        assert O.backward_error(pat.rowptr, pat.colidx, vals[i], xb[i], rhs[i]) <= tol
    sb.close()
    single.close()
