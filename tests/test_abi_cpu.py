"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function include/kkt.h declares, validates its inputs, and its analysis
agrees with the oracle's symbolic counts."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2302_08656_gb300 as K
from paper_2302_08656_gb300 import _native
from kktgen import KKTPattern, make_grid

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "kkt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kkt_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _native.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_native.SIGNATURES)


def test_status_strings_and_defaults():
    lib = _native.lib()
    for s in range(9):
        assert lib.kkt_status_string(s)
    o = _native.Options()
    lib.kkt_default_options(C.byref(o))
    assert o.precision == 0 and o.restart == 30 and o.ruiz_iters == 10 and o.max_cycles == 10


def test_plan_matches_oracle_symbolic_counts():
    """Same elimination order => same structural L+U count (integer, exact)."""
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    q = O.min_degree(pat.rowptr, pat.colidx)
    v = pat.values(pat.point(1, 0))
    an = O.analyze(pat.rowptr, pat.colidx, v)
    assert np.array_equal(an.q, q)
    lu, _, _ = O.refactor(pat.rowptr, pat.colidx, v, an)
    f = lu.factors()
    info = K.plan(pat.rowptr, pat.colidx, user_perm=q)
    assert info["nnz_lu"] == f.Lx.size + f.Ux.size
    assert info["n"] == pat.n and info["nnz"] == pat.nnz
    assert info["stored_factor"] >= info["nnz_lu"]


@pytest.mark.parametrize("B,L,G,seed", [(30, 40, 6, 3), (200, 300, 40, 1), (2000, 2560, 400, 4)])
def test_own_ordering_equals_the_oracle_minimum_degree(B, L, G, seed):
    """The library's minimum degree (quotient graph, binary heap) and the
    oracle's (explicit elimination graph, degree buckets) are independent
    implementations of one rule (exact degree, lowest index first): the plan
    of the library's own ordering is the plan of the oracle's order."""
    pat = KKTPattern(make_grid(seed, B, L, G))
    q = O.min_degree(pat.rowptr, pat.colidx)
    own = K.plan(pat.rowptr, pat.colidx)
    given = K.plan(pat.rowptr, pat.colidx, user_perm=q)
    for key in ("nnz_lu", "stored_factor", "n_fronts", "n_levels", "max_front", "flops"):
        assert own[key] == given[key], key


@pytest.mark.parametrize("B", [2, 3, 50])
def test_plan_small_and_degenerate_grids(B):
    pat = KKTPattern(make_grid(7, B, max(B - 1, 1) + (B // 3), max(1, B // 5)))
    info = K.plan(pat.rowptr, pat.colidx)
    assert info["n"] == pat.n and info["n_levels"] >= 1 and info["n_fronts"] >= 1


def test_plan_rejects_bad_patterns():
    # missing diagonal
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([1, 0], np.int32)
    with pytest.raises(K.KKTError) as e:
        K.plan(rp, ci)
    assert e.value.status == 5
    # unsymmetric pattern
    rp = np.array([0, 2, 3], np.int32)
    ci = np.array([0, 1, 1], np.int32)
    with pytest.raises(K.KKTError) as e:
        K.plan(rp, ci)
    assert e.value.status == 5
    # unsymmetric with equal row and column counts (a 3-cycle off the diagonal)
    rp = np.array([0, 2, 4, 6], np.int32)
    ci = np.array([0, 1, 1, 2, 0, 2], np.int32)
    with pytest.raises(K.KKTError) as e:
        K.plan(rp, ci)
    assert e.value.status == 5
    # unsorted columns
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([1, 0, 0, 1], np.int32)
    with pytest.raises(K.KKTError) as e:
        K.plan(rp, ci)
    assert e.value.status == 5
    # a user permutation that is not a permutation
    pat = KKTPattern(make_grid(1, 10, 12, 2))
    bad = np.zeros(pat.n, np.int32)
    with pytest.raises(K.KKTError) as e:
        K.plan(pat.rowptr, pat.colidx, user_perm=bad)
    assert e.value.status == 1
    # bad options
    with pytest.raises(K.KKTError):
        K.plan(pat.rowptr, pat.colidx, restart=0)


def test_one_by_one_and_diagonal_plans():
    rp = np.array([0, 1], np.int32)
    ci = np.array([0], np.int32)
    info = K.plan(rp, ci)
    assert info["n_fronts"] == 1 and info["nnz_lu"] == 1
    n = 100
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    info = K.plan(rp, ci)
    assert info["nnz_lu"] == n and info["n_levels"] == 1


def test_plan_tree_part_follows_the_option():
    """The persistent kernels take the narrow top of the tree: none with
    tree_min_fronts = 0, every level with a huge threshold, a contiguous top
    part in between; the option is validated."""
    pat = KKTPattern(make_grid(4, 2000, 2560, 400))
    none = K.plan(pat.rowptr, pat.colidx, tree_min_fronts=0)
    dflt = K.plan(pat.rowptr, pat.colidx)
    full = K.plan(pat.rowptr, pat.colidx, tree_min_fronts=10 ** 9)
    assert none["tree_levels"] == 0 and none["tree_units"] == 0
    assert 0 < dflt["tree_levels"] < dflt["n_levels"]
    assert full["tree_levels"] == full["n_levels"] and full["tree_units"] >= full["n_fronts"]
    assert none["nnz_lu"] == dflt["nnz_lu"] == full["nnz_lu"]
    with pytest.raises(K.KKTError):
        K.plan(pat.rowptr, pat.colidx, tree_min_fronts=-1)
    with pytest.raises(K.KKTError):
        K.plan(pat.rowptr, pat.colidx, spin_limit=0)


def test_out_of_range_options_are_refused():
    """Every option outside its documented range is refused with KKT_E_ARG by
    the host-only plan (the same check runs in kkt_analyze)."""
    pat = KKTPattern(make_grid(1, 10, 12, 2))
    bad = [dict(ruiz_iters=-1), dict(ruiz_iters=65), dict(restart=0), dict(restart=10 ** 6), dict(max_cycles=-1),
           dict(max_pivots=0), dict(max_pivots=65), dict(relax_pivots=0), dict(tree_min_fronts=-1),
           dict(spin_limit=0), dict(precond=3), dict(jacobi_sweeps=0), dict(ordering=3),
           dict(static_pivot_eps=float("nan")), dict(static_pivot_eps=1.0), dict(relax_zeros=-0.1),
           dict(relax_zeros=float("nan")), dict(relax_zeros=1.5)]
    for opts in bad:
        with pytest.raises(K.KKTError) as e:
            K.plan(pat.rowptr, pat.colidx, **opts)
        assert e.value.status == 1, opts
    # documented defaults-selecting values and the ends of the ranges are accepted
    for opts in [dict(static_pivot_eps=-1.0), dict(static_pivot_eps=0.0), dict(relax_zeros=0.0),
                 dict(relax_zeros=1.0), dict(max_pivots=64), dict(ruiz_iters=0)]:
        K.plan(pat.rowptr, pat.colidx, **opts)
    with pytest.raises(ValueError):
        K.plan(pat.rowptr, pat.colidx, precision="fp16")


def test_plan_fronts_matches_the_plan():
    """The host-only front query: one entry per front, pivots summing to n,
    every front at least as large as its pivot block, and the panels
    (F w + w (F - w) values each) adding up to the plan's stored factor."""
    pat = KKTPattern(make_grid(2, 300, 390, 60))
    for mp in (8, 16, 32):
        p = K.plan(pat.rowptr, pat.colidx, max_pivots=mp)
        F, w = K.plan_fronts(pat.rowptr, pat.colidx, max_pivots=mp)
        assert F.size == w.size == p["n_fronts"]
        assert int(w.sum()) == pat.n and np.all(w >= 1) and np.all(F >= w) and int(w.max()) <= mp
        assert int(F.max()) == p["max_front"]
        assert int(np.sum(F.astype(np.int64) * w + w * (F - w))) == p["stored_factor"]
        h = K.front_histogram(pat.rowptr, pat.colidx, max_pivots=mp)
        assert h["fronts"] == F.size and sum(b["fronts"] for b in h["buckets"]) == F.size
        assert abs(sum(b["flops"] for b in h["buckets"]) - h["flops"]) <= 1e-9 * h["flops"]
