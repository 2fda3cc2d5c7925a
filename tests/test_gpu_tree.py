"""The persistent tree kernels (narrow top of the assembly tree) against the
level-launched kernels, and their bounded waits.

Both schedules apply the same operations in the same order to every entry
(assembly: original entry, then the children in order; elimination: updates
in pivot order, one reciprocal per pivot), so factors and solutions must be
bitwise identical, whatever share of the tree the persistent kernels take.
Their agreement with the oracle is covered by test_gpu_parity.py, which runs
the default schedule.

Failure detection: a test hook makes the first unit of the refactorization
kernel wait on a flag that nothing sets; the bounded wait must expire, the
call must report KKT_E_TIMEOUT and the context must stay usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid, WORKLOADS

KKT_E_TIMEOUT = 7


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _run(pat, vals, rhs, precision, tree_min_fronts, count=1):
    dev = _dev()
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=count, precision=precision,
                    tree_min_fronts=tree_min_fronts)
    plan = s.plan()
    s.refactor(torch.from_numpy(vals).to(dev))
    x = s.solve(torch.from_numpy(rhs).to(dev)).cpu().numpy()
    f = s.export_factors()
    info = s.info()
    s.close()
    return plan, f, x, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("B,L,G,seed", [(200, 300, 40, 1), (2000, 2560, 400, 4), (30, 40, 6, 3)])
def test_tree_and_level_schedules_bitwise_equal(precision, B, L, G, seed):
    pat = KKTPattern(make_grid(seed, B, L, G))
    v = pat.values(pat.point(seed, 2, 1e-4))
    b = pat.rhs(seed, 2)
    runs = [_run(pat, v, b, precision, t) for t in (0, 152, 10 ** 9)]
    assert runs[0][0]["tree_levels"] == 0
    assert runs[2][0]["tree_levels"] == runs[2][0]["n_levels"]
    for plan, f, x, info in runs[1:]:
        assert info.status == 0
        assert info.n_perturbed == runs[0][3].n_perturbed
        for a, c in zip(f, runs[0][1]):
            assert np.array_equal(a, c)
        assert np.array_equal(x, runs[0][2])


def test_tree_batched_instances_equal_single():
    pat = KKTPattern(make_grid(4, 2000, 2560, 400))
    count = 5
    vals = np.concatenate([pat.values(pat.point(100 + i, 1, 1e-3)) for i in range(count)])
    rhs = np.concatenate([pat.rhs(100 + i, 1) for i in range(count)])
    _, _, xb, info = _run(pat, vals, rhs, "fp64", 10 ** 9, count=count)
    assert info.status == 0
    for i in range(count):
        _, _, xi, _ = _run(pat, vals[i * pat.nnz:(i + 1) * pat.nnz], rhs[i * pat.n:(i + 1) * pat.n], "fp64", 0)
        assert np.array_equal(xb[i * pat.n:(i + 1) * pat.n], xi)


def test_bounded_wait_expires_and_context_recovers():
    dev = _dev()
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    v = torch.from_numpy(pat.values(pat.point(1, 0, 1e-1))).to(dev)
    b = torch.from_numpy(pat.rhs(1, 0)).to(dev)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, spin_limit=20000)
    assert s.plan()["tree_levels"] > 0
    s.refactor(v)
    x_ok, info = s.refine(b, tol=1e-12)
    assert info.status == 0
    s.debug_stall()
    s.refactor(v)
    assert s.info().status == KKT_E_TIMEOUT
    with pytest.raises(K.KKTError) as e:
        s.refine(b, tol=1e-12)
    assert e.value.status == KKT_E_TIMEOUT
    s.refactor(v)                                   # the context is usable again
    x, info = s.refine(b, tol=1e-12)
    assert info.status == 0 and info.backward_err <= 1e-12
    assert torch.equal(x, x_ok)
    s.close()


def test_no_tree_part_rejects_the_stall_hook():
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    _dev()
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, tree_min_fronts=0)
    with pytest.raises(K.KKTError) as e:
        s.debug_stall()
    assert e.value.status == 4
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("count,tmf", [(1, 2432), (1, 10 ** 9), (3, 10 ** 9), (1, 0)])
def test_fused_refactor_refine_equals_separate_calls(precision, count, tmf):
    """kkt_refactor_refine (the forward substitution of the first solve inside
    the refactorization) gives the same bits as kkt_refactor + kkt_refine."""
    dev = _dev()
    pat = KKTPattern(make_grid(4, 2000, 2560, 400))
    vals = np.concatenate([pat.values(pat.point(40 + i, 3, 1e-5)) for i in range(count)])
    rhs = np.concatenate([pat.rhs(40 + i, 3) for i in range(count)])
    v = torch.from_numpy(vals).to(dev)
    b = torch.from_numpy(rhs).to(dev)
    a = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=count, precision=precision, tree_min_fronts=tmf)
    f = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=count, precision=precision, tree_min_fronts=tmf)
    for _ in range(2):                                 # second call replays the captured graphs
        a.refactor(v)
        xa, ia = a.refine(b, tol=1e-10)
        xf, if_ = f.refactor_refine(v, b, tol=1e-10)
        assert torch.equal(xa, xf)
        ia = ia if count > 1 else [ia]
        if_ = if_ if count > 1 else [if_]
        for p, q in zip(ia, if_):
            assert p.backward_err == q.backward_err and p.iters == q.iters and p.status == q.status == 0
    a.close()
    f.close()


@pytest.fixture(scope="module")
def grid8k():
    return KKTPattern(make_grid(5, 8000, 10240, 1600))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_warp_class_staged_children_bitwise(grid8k, precision):
    """8,000-bus grid: levels 1-2 (1,583 and 856 fronts) are factored a warp per
    front with the children's blocks staged by cp.async, 67 of those fronts in
    more than one staging chunk; the same bits as the all-tree schedule."""
    pat = grid8k
    v = pat.values(pat.point(8, 2, 1e-4))
    b = pat.rhs(8, 2)
    runs = [_run(pat, v, b, precision, t) for t in (0, 10 ** 9)]
    for plan, f, x, info in runs:
        assert info.status == 0
    for a, c in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(a, c)
    assert np.array_equal(runs[0][2], runs[1][2])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_forward_in_the_warp_class_equals_separate(grid8k, precision):
    """kkt_refactor_refine on the 8,000-bus grid with every level launched: the
    forward step runs inside the leaf and warp kernels (children's vectors staged
    with their blocks) and gives the bits of kkt_refactor + kkt_refine."""
    dev = _dev()
    pat = grid8k
    v = torch.from_numpy(pat.values(pat.point(9, 3, 1e-5))).to(dev)
    b = torch.from_numpy(pat.rhs(9, 3)).to(dev)
    a = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision, tree_min_fronts=0)
    f = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision=precision, tree_min_fronts=0)
    a.refactor(v)
    xa, ia = a.refine(b, tol=1e-10)
    xf, if_ = f.refactor_refine(v, b, tol=1e-10)
    assert torch.equal(xa, xf)
    assert ia.backward_err == if_.backward_err and ia.status == if_.status == 0
    a.close()
    f.close()


def test_warp_class_child_past_the_staging_area_bitwise():
    """The 70,000-bus system with every level launched: on levels 5-7 some warp-class
    fronts have a child whose block exceeds the staging area and is read from
    global memory; factors and solution equal the all-tree schedule's."""
    w = WORKLOADS["eastern70k"]
    pat = KKTPattern(make_grid(2, w["n_bus"], w["n_branch"], w["n_gen"]))
    v = pat.values(pat.point(2, 1, 1e-3))
    b = pat.rhs(2, 1)
    runs = [_run(pat, v, b, "fp64", t) for t in (0, 10 ** 9)]
    for plan, f, x, info in runs:
        assert info.status == 0
    assert runs[0][0]["tree_levels"] == 0
    for a, c in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(a, c)
    assert np.array_equal(runs[0][2], runs[1][2])
