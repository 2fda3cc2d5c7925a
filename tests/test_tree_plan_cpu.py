"""Ordering checks of the persistent tree kernels' plan (tree_plan.cpp,
compiled here with g++ into tests/tree_plan_dump.cpp). A unit of the
persistent kernels takes a ticket in plan order and waits only on units
with smaller tickets, which is what guarantees forward progress without
any assumption on how many blocks are resident. Checked:

* the tree part is exactly the levels from `split` up, level by level, and
  within a level the fronts are ordered by the last index among their
  children;
* every factorization unit comes after every unit of its children's fronts;
  in the fused order every forward unit comes after the factorization units
  of its own front and the forward units of its children;
* every parent front has a larger index than its children (the backward
  solve runs the fronts in reverse); children below the tree part (factored
  by the level launches before the tree kernels) are never waited on;
* every front has nt x nt factorization units and one forward unit.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from kktgen import KKTPattern, make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_08656_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def dump_tool(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers not available")
    exe = str(tmp_path_factory.mktemp("tree") / "tree_plan_dump")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(ROOT, "tests", "tree_plan_dump.cpp"), os.path.join(CSRC, "analysis.cpp"),
                    os.path.join(CSRC, "tree_plan.cpp"), "-o", exe], check=True)
    return exe


def _plan(tool, tmp_path, pat, max_pivots, min_fronts):
    src, out = str(tmp_path / "in"), str(tmp_path / "out")
    np.asarray([pat.n], np.int32).tofile(src + ".n")
    np.asarray(pat.rowptr, np.int32).tofile(src + ".rp")
    np.asarray(pat.colidx, np.int32).tofile(src + ".ci")
    subprocess.run([tool, src, out, str(max_pivots), str(min_fronts)], check=True)
    r = {k: np.fromfile(out + "." + k, dtype=np.int64)
         for k in ["head", "fr", "kid", "unit", "fused", "level", "sn_parent", "child_ptr", "child_list", "asm_ptr",
                   "sn_first", "sn_front", "bwd_chain", "bwd_chain_ptr"]}
    r["fr"] = r["fr"].reshape(-1, 6)
    r["unit"] = r["unit"].reshape(-1, 3)
    r["fused"] = r["fused"].reshape(-1, 3)
    return r


@pytest.mark.parametrize("buses,max_pivots,min_fronts", [(2000, 16, 2432), (2000, 8, 100000), (500, 16, 64),
                                                         (2000, 16, 0)])
def test_tree_plan_orders_every_dependency_first(dump_tool, tmp_path, buses, max_pivots, min_fronts):
    pat = KKTPattern(make_grid(3, buses, int(1.28 * buses), buses // 5))
    P = _plan(dump_tool, tmp_path, pat, max_pivots, min_fronts)
    split, n_levels, ns, nq, alg_bytes = (int(x) for x in P["head"])
    fr, kid, level, sn_parent = P["fr"], P["kid"], P["level"], P["sn_parent"]
    if min_fronts == 0:
        assert nq == 0 and split == n_levels
        return
    # the tree part: exactly the fronts of levels >= split, level by level
    sn = fr[:, 0]
    assert sorted(sn.tolist()) == [s for s in range(ns) if level[s] >= split]
    lev = level[sn]
    assert np.all(np.diff(lev) >= 0)
    q_of = np.full(ns, -1)
    q_of[sn] = np.arange(nq)
    # within a level, ordered by the last tree index among the children
    key = []
    for q in range(nq):
        kids = kid[fr[q, 4]:fr[q, 5]]
        key.append(max(kids.max(), -1) if kids.size else -1)
    key = np.asarray(key)
    for l in range(split, n_levels):
        ks = key[lev == l]
        if l > split:
            assert np.all(np.diff(ks) >= 0)
    for q in range(nq):
        s = sn[q]
        # parents and children
        assert fr[q, 1] == (q_of[sn_parent[s]] if sn_parent[s] >= 0 else -1)
        if fr[q, 1] >= 0:
            assert fr[q, 1] > q
        ch = P["child_list"][P["child_ptr"][s]:P["child_ptr"][s + 1]]
        assert kid[fr[q, 4]:fr[q, 5]].tolist() == [int(q_of[c]) for c in ch]      # -1 below the tree part
        assert all((q_of[c] >= 0) == (level[c] >= split) for c in ch)
    # factorization units: nt x nt per front, every child's units first
    unit = P["unit"]
    first_u = np.full(nq, -1)
    last_u = np.full(nq, -1)
    for u, (q, ti, tj) in enumerate(unit):
        if first_u[q] < 0:
            first_u[q] = u
        last_u[q] = u
    for q in range(nq):
        nt = fr[q, 2]
        mine = unit[first_u[q]:last_u[q] + 1]
        assert fr[q, 3] == nt * nt and len(mine) == nt * nt and np.all(mine[:, 0] == q)
        assert sorted(zip(mine[:, 1], mine[:, 2])) == [(i, j) for i in range(nt) for j in range(nt)]
        for c in kid[fr[q, 4]:fr[q, 5]]:
            if c >= 0:
                assert last_u[c] < first_u[q]
    # fused order: the forward unit after its front's factorization units and its children's forward units
    fused = P["fused"]
    pos_fwd = np.full(nq, -1)
    last_fac = np.full(nq, -1)
    first_fac = np.full(nq, -1)
    for u, (q, ti, tj) in enumerate(fused):
        if ti < 0:
            assert pos_fwd[q] < 0
            pos_fwd[q] = u
        else:
            last_fac[q] = u
            if first_fac[q] < 0:
                first_fac[q] = u
    assert np.all(pos_fwd >= 0) and len(fused) == len(unit) + nq
    for q in range(nq):
        assert last_fac[q] < pos_fwd[q]
        for c in kid[fr[q, 4]:fr[q, 5]]:
            if c >= 0:
                assert pos_fwd[c] < pos_fwd[q] and last_fac[c] < first_fac[q]
    # backward chains: every front exactly once; a chain starts at a root or
    # at a front whose parent has two or more children in the tree part and
    # continues through single tree children; the chain holding a chain's
    # first front's parent comes earlier
    chain, cptr = P["bwd_chain"], P["bwd_chain_ptr"]
    assert cptr[0] == 0 and cptr[-1] == nq and np.all(np.diff(cptr) > 0)
    assert sorted(chain.tolist()) == list(range(nq))
    tree_kids = [[c for c in kid[fr[q, 4]:fr[q, 5]] if c >= 0] for q in range(nq)]
    chain_of = np.empty(nq, dtype=np.int64)
    for ci in range(len(cptr) - 1):
        members = chain[cptr[ci]:cptr[ci + 1]]
        chain_of[members] = ci
        top = members[0]
        assert fr[top, 1] < 0 or len(tree_kids[fr[top, 1]]) >= 2
        for a_, b_ in zip(members[:-1], members[1:]):
            assert tree_kids[a_] == [b_]
        assert len(tree_kids[members[-1]]) != 1
    for ci in range(len(cptr) - 1):
        top = chain[cptr[ci]]
        if fr[top, 1] >= 0:
            assert chain_of[fr[top, 1]] < ci
            assert chain[cptr[chain_of[fr[top, 1]] + 1] - 1] == fr[top, 1]     # the parent ends its chain
    # the forward substitution runs the chains in reverse (bottom front first,
    # chains from the last to the first): a bottom front's children in the
    # tree part are tops of chains with larger indices (earlier forward
    # tickets), and the only child of every later front is the front before it
    for ci in range(len(cptr) - 1):
        members = chain[cptr[ci]:cptr[ci + 1]]
        for c in tree_kids[members[-1]]:
            assert chain_of[c] > ci and chain[cptr[chain_of[c]]] == c
        for lower, upper in zip(members[::-1][:-1], members[::-1][1:]):
            assert tree_kids[upper] == [lower]


@pytest.mark.parametrize("buses,max_pivots,min_fronts", [(2000, 16, 2432), (500, 8, 100000)])
def test_tree_algorithmic_bytes_follow_their_definition(dump_tool, tmp_path, buses, max_pivots, min_fronts):
    """The algorithmic bytes of one refactorization of the tree part (the
    roofline numerator of tree_factor_kernel), recomputed from the fronts:
    per front, its original entries (value + 8 bytes of position and source
    index), its factor panel (F w + w m values), its own contribution block
    written (m^2) and its children's contribution blocks read; 8-byte values."""
    pat = KKTPattern(make_grid(5, buses, int(1.28 * buses), buses // 5))
    P = _plan(dump_tool, tmp_path, pat, max_pivots, min_fronts)
    split, n_levels, ns, nq, alg_bytes = (int(x) for x in P["head"])
    assert nq > 0
    es = 8
    w = np.diff(P["sn_first"])
    F = P["sn_front"]
    m = F - w
    expect = 0
    for s in P["fr"][:, 0]:
        expect += (P["asm_ptr"][s + 1] - P["asm_ptr"][s]) * (es + 8)
        expect += (F[s] * w[s] + w[s] * m[s]) * es + m[s] * m[s] * es
        for c in P["child_list"][P["child_ptr"][s]:P["child_ptr"][s + 1]]:
            expect += m[c] * m[c] * es
    assert alg_bytes == expect
