"""Refactorization of uneven sizes in one launch (kkt_group_*): patterns of
different sizes, some batched, refactored together -- level parts on forked
streams, the tops of all assembly trees in one persistent launch whose
tickets interleave the members by height. Every member's factors and
solutions must equal, bit for bit, those of the same member refactored
alone (same kernels and per-context order; only the scheduling differs), and
the solutions meet the tolerance by the oracle's backward error."""
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


MEMBERS = [(500, 640, 100, 1), (2000, 2560, 400, 4), (5000, 6400, 1000, 2)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_group_refactor_equals_each_member_alone(precision):
    dev = _dev()
    pats = [KKTPattern(make_grid(10 + i, B, L, G)) for i, (B, L, G, _) in enumerate(MEMBERS)]
    counts = [c for *_, c in MEMBERS]
    grouped = [K.KKTSolver(p.rowptr, p.colidx, p.n_primal, count=c, precision=precision, tree_min_fronts=152 * c)
               for p, c in zip(pats, counts)]
    alone = [K.KKTSolver(p.rowptr, p.colidx, p.n_primal, count=c, precision=precision, tree_min_fronts=152 * c)
             for p, c in zip(pats, counts)]
    assert all(s.plan()["tree_levels"] > 0 for s in grouped)
    group = K.KKTGroup(grouped)
    for step in range(2):                                   # twice: graphs are captured on the first call
        vals_h = [[p.values(p.point(100 * step + 10 * g + i, step, 10.0 ** -(1 + 3 * step + i)))
                   for i in range(c)] for g, (p, c) in enumerate(zip(pats, counts))]
        rhs_h = [[p.rhs(100 * step + 10 * g + i, step) for i in range(c)] for g, (p, c) in enumerate(zip(pats, counts))]
        vals = [torch.from_numpy(np.concatenate(v)).to(dev) for v in vals_h]
        rhs = [torch.from_numpy(np.concatenate(b)).to(dev) for b in rhs_h]
        group.refactor(vals)
        for s, v in zip(alone, vals):
            s.refactor(v)
        torch.cuda.synchronize()
        for g, (sg, sa, p, c) in enumerate(zip(grouped, alone, pats, counts)):
            assert sg.info().status == 0 and sa.info().status == 0
            fg, fa = sg.export_factors(), sa.export_factors()
            for a, b in zip(fg, fa):
                assert np.array_equal(a, b), "member %d factors differ" % g
            xg, ig = sg.refine(rhs[g], tol=1e-10)
            xa, ia = sa.refine(rhs[g], tol=1e-10)
            assert np.array_equal(xg.cpu().numpy(), xa.cpu().numpy()), "member %d solutions differ" % g
            xs = xg.cpu().numpy().reshape(c, p.n)
            for i in range(c):
                assert O.backward_error(p.rowptr, p.colidx, vals_h[g][i], xs[i], rhs_h[g][i]) <= 1e-10
    group.close()
    for s in grouped + alone:
        s.close()


def test_group_arguments():
    _dev()
    p = KKTPattern(make_grid(1, 200, 300, 40))
    a = K.KKTSolver(p.rowptr, p.colidx, p.n_primal)
    b = K.KKTSolver(p.rowptr, p.colidx, p.n_primal, precision="fp32")
    with pytest.raises(ValueError):
        K.KKTGroup([a, b])                                   # mixed precision
    with pytest.raises(ValueError):
        K.KKTGroup([a, a])                                   # a member twice
    lib = K._native.lib()
    arr = K._ptr_array([a.handle.value, b.handle.value])
    import ctypes as C
    h = C.c_void_p()
    assert lib.kkt_group_create(arr, 2, C.byref(h)) == 1     # the library refuses mixed precision too
    assert lib.kkt_group_create(arr, 0, C.byref(h)) == 1
    g = K.KKTGroup([a])
    with pytest.raises(ValueError):
        g.refactor([])
    g.close()
    a.close()
    b.close()
