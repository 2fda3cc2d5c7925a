"""The host plan of the saddle-point specialised solve (hykkt_plan.cpp,
compiled here with g++ into tests/hykkt_plan_dump.cpp), against definitions
written independently with scipy: the blocks of K, the pattern of
H_g = H + J_I^T D_I^{-1} J_I + gamma J_E^T J_E, and its values summed from the
plan's term lists; and the patterns it must refuse."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from kktgen import KKTPattern, make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_08656_gb300", "csrc")
KEYS = ["dpos", "je_p", "je_c", "je_v", "ji_p", "ji_c", "ji_v", "jet_p", "jet_c", "jet_v", "jit_p", "jit_c", "jit_v",
        "hg_p", "hg_c", "term_ptr", "term"]


@pytest.fixture(scope="module")
def tool(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("hykkt") / "hykkt_plan_dump")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "hykkt_plan_dump.cpp"),
                    os.path.join(CSRC, "hykkt_plan.cpp"), "-o", exe], check=True)
    return exe


def _run(tool, tmp_path, n, rowptr, colidx, n_primal, m_eq):
    src, out = str(tmp_path / "in"), str(tmp_path / "out")
    np.asarray([n], np.int32).tofile(src + ".n")
    np.asarray(rowptr, np.int32).tofile(src + ".rp")
    np.asarray(colidx, np.int32).tofile(src + ".ci")
    r = subprocess.run([tool, src, out, str(n_primal), str(m_eq)])
    if r.returncode != 0:
        return r.returncode, None
    P = {k: np.fromfile(out + "." + k, dtype=np.int64) for k in KEYS}
    P["term"] = P["term"].reshape(-1, 3)
    return 0, P


@pytest.mark.parametrize("buses,lines,gens,gamma", [(120, 170, 24, 300.0), (200, 300, 40, 1e8), (3, 2, 1, 20.0)])
def test_plan_reproduces_the_blocks_and_H_g(tool, tmp_path, buses, lines, gens, gamma):
    pat = KKTPattern(make_grid(2, buses, lines, gens))
    n, npr, mE = pat.n, pat.n_primal, 2 * pat.grid.n_bus
    st, P = _run(tool, tmp_path, n, pat.rowptr, pat.colidx, npr, mE)
    assert st == 0
    rng = np.random.default_rng(buses)
    rp, ci = np.asarray(pat.rowptr, np.int64), np.asarray(pat.colidx, np.int64)
    vals = rng.standard_normal(rp[-1])
    rows = np.repeat(np.arange(n), np.diff(rp))
    # the (2,2) diagonal: negative, so that d = -diag > 0
    dual_diag = (rows >= npr) & (ci == rows)
    vals[dual_diag] = -rng.uniform(0.5, 2.0, dual_diag.sum())
    K = sp.csr_matrix((vals, ci, rp), shape=(n, n))
    H, JE, JI = K[:npr, :npr], K[npr:npr + mE, :npr], K[npr + mE:, :npr]
    d = -K.diagonal()[npr:]
    dE, dI = d[:mE], d[mE:]
    # blocks: positions point at K's entries of the right row and column
    assert np.array_equal(ci[P["dpos"]], np.arange(npr, n)) and np.array_equal(rows[P["dpos"]], np.arange(npr, n))
    for name, m, off in (("je", mE, npr), ("ji", n - npr - mE, npr + mE)):
        p_, c_, v_ = P[name + "_p"], P[name + "_c"], P[name + "_v"]
        assert p_.size == m + 1 and np.array_equal(ci[v_], c_) and np.all(c_ < npr)
        assert np.array_equal(rows[v_], off + np.repeat(np.arange(m), np.diff(p_)))
        # transpose: the same (row, column, position) triples
        tp, tc, tv = P[name + "t_p"], P[name + "t_c"], P[name + "t_v"]
        fwd = sorted(zip(np.repeat(np.arange(m), np.diff(p_)).tolist(), c_.tolist(), v_.tolist()))
        bwd = sorted(zip(tc.tolist(), np.repeat(np.arange(npr), np.diff(tp)).tolist(), tv.tolist()))
        assert fwd == bwd
    # pattern of H_g: struct(H) + struct(J_I^T J_I) + struct(J_E^T J_E) + the diagonal, each row sorted
    S = lambda A: (abs(A) > 0).astype(np.int64)                    # noqa: E731
    pattern = (S(H) + S(JI).T @ S(JI) + S(JE).T @ S(JE) + sp.eye(npr, dtype=np.int64)).tocsr()
    pattern.sort_indices()
    assert np.array_equal(P["hg_p"], pattern.indptr) and np.array_equal(P["hg_c"], pattern.indices)
    # values from the term lists
    t = P["term"]
    a, b, k = t[:, 0], t[:, 1], t[:, 2]
    tv = np.where(k == -1, vals[a], np.where(k == -2, gamma * vals[a] * vals[np.maximum(b, 0)],
                                             vals[a] * vals[np.maximum(b, 0)] / dI[np.maximum(k, 0)] if dI.size else 0))
    ent = np.add.reduceat(tv, P["term_ptr"][:-1]) if tv.size else np.zeros(0)
    ent[np.diff(P["term_ptr"]) == 0] = 0.0                      # the diagonal with no term
    Hg = sp.csr_matrix((ent, P["hg_c"], P["hg_p"]), shape=(npr, npr))
    ref = (H + JI.T @ sp.diags(1.0 / dI) @ JI + gamma * (JE.T @ JE)) if dI.size else (H + gamma * (JE.T @ JE))
    diff = abs(Hg - ref).max()
    assert diff <= 1e-13 * max(1.0, abs(ref).max())
    # every term of an entry lies in its row and column
    e_row = np.repeat(np.repeat(np.arange(npr), np.diff(P["hg_p"])), np.diff(P["term_ptr"]))
    e_col = np.repeat(P["hg_c"], np.diff(P["term_ptr"]))
    h = k == -1
    assert np.array_equal(rows[a[h]], e_row[h]) and np.array_equal(ci[a[h]], e_col[h])
    pr = ~h
    assert np.array_equal(ci[a[pr]], e_row[pr]) and np.array_equal(ci[b[pr]], e_col[pr])
    assert np.array_equal(rows[a[pr]], rows[b[pr]])              # a pair lies in one dual row
    del dE


def _coo_to_csr(n, r, c):
    order = np.lexsort((c, r))
    r, c = np.asarray(r)[order], np.asarray(c)[order]
    rp = np.concatenate([[0], np.cumsum(np.bincount(r, minlength=n))]).astype(np.int32)
    return rp, c.astype(np.int32)


def test_plan_refuses_what_the_method_cannot_take(tool, tmp_path):
    pat = KKTPattern(make_grid(2, 20, 28, 4))
    n, npr, mE = pat.n, pat.n_primal, 2 * pat.grid.n_bus
    rp = np.asarray(pat.rowptr, np.int64)
    rows = np.repeat(np.arange(n), np.diff(rp))
    cols = np.asarray(pat.colidx, np.int64)
    # (2,2) block not diagonal
    r2, c2 = _coo_to_csr(n, np.concatenate([rows, [npr, npr + 1]]), np.concatenate([cols, [npr + 1, npr]]))
    assert _run(tool, tmp_path, n, r2, c2, npr, mE)[0] == 2
    # a dual row without its diagonal
    keep = ~((rows == npr + 3) & (cols == npr + 3))
    r3, c3 = _coo_to_csr(n, rows[keep], cols[keep])
    assert _run(tool, tmp_path, n, r3, c3, npr, mE)[0] == 3
    # a column out of range, row pointers not monotone
    c4 = np.asarray(pat.colidx, np.int32).copy()
    c4[5] = n
    assert _run(tool, tmp_path, n, pat.rowptr, c4, npr, mE)[0] == 1
    r5 = np.asarray(pat.rowptr, np.int32).copy()
    r5[3], r5[4] = r5[4], r5[3]
    assert _run(tool, tmp_path, n, r5, pat.colidx, npr, mE)[0] == 1
    # the unmodified pattern is taken
    assert _run(tool, tmp_path, n, pat.rowptr, pat.colidx, npr, mE)[0] == 0
