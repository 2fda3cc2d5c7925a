"""Structural checks of the library's host analysis (analysis.cpp, compiled
here with g++ into tests/analysis_dump.cpp) against definitions computed
independently on the CPU:

* the front row sets equal the pivots plus the union of their exact column
  structures, taken from an elimination game on the permuted pattern;
* every original entry is assembled exactly once, into the front of its
  earlier step, at the local position of its row and column;
* every contribution-block row maps to the same row of the parent front,
  children lists and levels are consistent, storage offsets match the
  front sizes;
* the sliced copy of the pattern holds every entry exactly once, a row's
  entries in CSR order down its lane, slice widths equal to the longest row
  of the slice, rows sorted by length within each window.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from kktgen import KKTPattern, make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_08656_gb300", "csrc")


@pytest.fixture(scope="module")
def dump_tool(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("analysis") / "analysis_dump")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "analysis_dump.cpp"),
                    os.path.join(CSRC, "analysis.cpp"), "-o", exe], check=True)
    return exe


def _plan(tool, tmp_path, rowptr, colidx, max_pivots):
    n = rowptr.size - 1
    src, out = str(tmp_path / "in"), str(tmp_path / "out")
    np.asarray([n], np.int32).tofile(src + ".n")
    np.asarray(rowptr, np.int32).tofile(src + ".rp")
    np.asarray(colidx, np.int32).tofile(src + ".ci")
    subprocess.run([tool, src, out, str(max_pivots)], check=True)
    names = ["perm", "sn_first", "sn_parent", "sn_front", "rows_ptr", "rows", "child_ptr", "child_list",
             "level_ptr", "level_fronts", "asm_ptr", "asm_pos", "asm_src", "rel_ptr", "rel", "cb_split",
             "panel_off", "cb_off", "stats", "sell_off", "sell_row", "sell_ci", "sell_src", "csr2sell"]
    return {k: np.fromfile(out + "." + k, dtype=np.int64) for k in names}


def _column_structures(rowptr, colidx, iperm):
    """Elimination game on the pattern relabelled by iperm: struct[j] = rows > j
    of column j of the factor."""
    n = rowptr.size - 1
    adj = [set() for _ in range(n)]
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    for i, j in zip(rows, colidx):
        if i != j:
            a, b = int(iperm[i]), int(iperm[j])
            adj[a].add(b)
            adj[b].add(a)
    struct = []
    for j in range(n):
        s = {k for k in adj[j] if k > j}
        struct.append(s)
        for k in s:
            adj[k] |= s
            adj[k].discard(k)
    return struct


def _random_symmetric(n, deg, seed):
    rng = np.random.default_rng(seed)
    pairs = set()
    for i in range(n):
        for j in rng.integers(0, n, size=deg):
            if i != j:
                pairs.add((min(i, int(j)), max(i, int(j))))
    rows = [[i] for i in range(n)]
    for a, b in pairs:
        rows[a].append(b)
        rows[b].append(a)
    rowptr = np.zeros(n + 1, np.int32)
    colidx = []
    for i in range(n):
        r = sorted(rows[i])
        colidx.extend(r)
        rowptr[i + 1] = rowptr[i] + len(r)
    return rowptr, np.asarray(colidx, np.int32)


CASES = [("kkt 200 buses", 16), ("kkt 200 buses", 4), ("kkt 60 buses", 1), ("random 400", 16), ("random 400", 3)]


@pytest.mark.parametrize("case,max_pivots", CASES)
def test_plan_structure(dump_tool, tmp_path, case, max_pivots):
    if case == "kkt 200 buses":
        pat = KKTPattern(make_grid(1, 200, 300, 40))
        rowptr, colidx = pat.rowptr, pat.colidx
    elif case == "kkt 60 buses":
        pat = KKTPattern(make_grid(4, 60, 80, 12))
        rowptr, colidx = pat.rowptr, pat.colidx
    else:
        rowptr, colidx = _random_symmetric(400, 3, 7)
    n, nnz = rowptr.size - 1, colidx.size
    P = _plan(dump_tool, tmp_path, rowptr, colidx, max_pivots)
    perm = P["perm"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    iperm = np.empty(n, np.int64)
    iperm[perm] = np.arange(n)
    ns = int(P["stats"][0])
    first, parent, front = P["sn_first"], P["sn_parent"], P["sn_front"]
    rows_ptr, rows = P["rows_ptr"], P["rows"]
    assert first.size == ns + 1 and first[0] == 0 and first[-1] == n
    width = np.diff(first)
    assert np.all(width >= 1) and np.all(width <= max_pivots)
    struct = _column_structures(rowptr, colidx, iperm)
    assert int(P["stats"][2]) == sum(len(s) for s in struct)            # nnz(L), diagonal excluded
    front_of = np.repeat(np.arange(ns), width)
    for s in range(ns):
        R = rows[rows_ptr[s]:rows_ptr[s + 1]]
        w, F = int(width[s]), int(front[s])
        assert R.size == F and np.all(np.diff(R) > 0)
        piv = np.arange(first[s], first[s + 1])
        assert np.array_equal(R[:w], piv)
        union = set()
        for j in piv:
            union |= struct[j]
        assert set(R[w:].tolist()) == {i for i in union if i > piv[-1]}
        if F > w:
            assert parent[s] == front_of[R[w]]                          # the etree parent of the last pivot
        else:
            assert parent[s] == -1
    # assembly: every entry once, into the front of its earlier step, at (row, column)
    asm_ptr, asm_pos, asm_src = P["asm_ptr"], P["asm_pos"], P["asm_src"]
    assert np.array_equal(np.sort(asm_src), np.arange(nnz))
    entry_row = np.repeat(np.arange(n), np.diff(rowptr))
    for s in range(ns):
        R = rows[rows_ptr[s]:rows_ptr[s + 1]]
        F = int(front[s])
        for at in range(asm_ptr[s], asm_ptr[s + 1]):
            p = asm_src[at]
            r, c = iperm[entry_row[p]], iperm[colidx[p]]
            assert front_of[min(r, c)] == s
            a, b = asm_pos[at] % F, asm_pos[at] // F
            assert R[a] == r and R[b] == c
    # contribution rows into the parent, the ones on the parent's pivots first
    rel_ptr, rel, cb_split = P["rel_ptr"], P["rel"], P["cb_split"]
    for s in range(ns):
        w, F, q = int(width[s]), int(front[s]), int(parent[s])
        assert rel_ptr[s + 1] - rel_ptr[s] == F - w
        if q < 0:
            continue
        R = rows[rows_ptr[s]:rows_ptr[s + 1]]
        Rq = rows[rows_ptr[q]:rows_ptr[q + 1]]
        loc = rel[rel_ptr[s]:rel_ptr[s + 1]]
        assert np.array_equal(Rq[loc], R[w:])
        assert cb_split[s] == int(np.sum(loc < width[q]))
    # children lists and levels
    child_ptr, child_list = P["child_ptr"], P["child_list"]
    for s in range(ns):
        assert list(child_list[child_ptr[s]:child_ptr[s + 1]]) == [k for k in range(ns) if parent[k] == s]
    level_ptr, level_fronts = P["level_ptr"], P["level_fronts"]
    assert np.array_equal(np.sort(level_fronts), np.arange(ns))
    lev = np.empty(ns, np.int64)
    for l in range(level_ptr.size - 1):
        lev[level_fronts[level_ptr[l]:level_ptr[l + 1]]] = l
    for s in range(ns):
        kids = child_list[child_ptr[s]:child_ptr[s + 1]]
        assert lev[s] == (1 + max(lev[k] for k in kids) if kids.size else 0)
    # storage offsets
    F, w = front.astype(np.int64), width.astype(np.int64)
    assert np.array_equal(np.diff(P["panel_off"]), F * w + w * (F - w))
    assert np.array_equal(np.diff(P["cb_off"]), (F - w) ** 2)


@pytest.mark.parametrize("B,L,G,seed", [(2, 1, 1, 3), (37, 50, 8, 5), (1500, 1920, 300, 6)])
def test_sliced_copy_of_the_pattern(dump_tool, tmp_path, B, L, G, seed):
    pat = KKTPattern(make_grid(seed, B, L, G))
    p = _plan(dump_tool, tmp_path, pat.rowptr, pat.colidx, 16)
    n, nnz = pat.n, pat.nnz
    off, row, ci, src, c2s = p["sell_off"], p["sell_row"], p["sell_ci"], p["sell_src"], p["csr2sell"]
    ns = (n + 31) // 32
    assert off.size == ns + 1 and row.size == 32 * ns and off[0] == 0
    lens = np.diff(pat.rowptr)
    # every row once, lanes past the last row empty
    assert sorted(row[row >= 0].tolist()) == list(range(n)) and np.all(row[n:] == -1)
    assert np.all(row[:n] >= 0)
    slots = 0
    for s_ in range(ns):
        r = row[32 * s_:32 * s_ + 32]
        width = (off[s_ + 1] - off[s_]) // 32
        assert (off[s_ + 1] - off[s_]) % 32 == 0
        assert width == max(lens[x] for x in r if x >= 0)
        for l, x in enumerate(r):
            for k in range(width):
                o = off[s_] + 32 * k + l
                if x >= 0 and k < lens[x]:
                    assert src[o] == pat.rowptr[x] + k and ci[o] == pat.colidx[src[o]] and c2s[src[o]] == o
                    slots += 1
                else:
                    assert src[o] == -1 and ci[o] == -1
    assert slots == nnz and ci.size == off[-1]
    # rows are sorted by decreasing length (then index) within each window of 4096 rows
    order = row[:n]
    for w0 in range(0, n, 4096):
        seg = order[w0:w0 + 4096]
        assert sorted(seg.tolist()) == list(range(w0, min(n, w0 + 4096)))
        key = [(-lens[x], x) for x in seg]
        assert key == sorted(key)
