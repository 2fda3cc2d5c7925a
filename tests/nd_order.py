"""Test-side nested-dissection ordering of a KKT pattern: recursive coordinate
bisection of the buses' positions, each cut's vertex separator (the vertices
of one half adjacent to the other) ordered after both halves. Given to the
library as a user permutation (the refactorization accepts any elimination
order, Sec. III), so that the tree height and fill of a dissection order can
be compared with the library's own minimum-degree order."""
import numpy as np
import scipy.sparse as sp


def kkt_coordinates(pat):
    """A position for every row of the KKT matrix: a variable or balance row at
    its bus, a generator at its bus, a flow-limit row at its line's midpoint."""
    g = pat.grid
    mid = 0.5 * (g.xy[g.f] + g.xy[g.t])
    parts = [g.xy, g.xy, g.xy[g.gen_bus], g.xy[g.gen_bus], g.xy, g.xy]
    if pat.flow_limits:
        parts += [mid, mid]
    return np.concatenate(parts)


def nested_dissection(pat, leaf=64):
    n = pat.n
    A = sp.csr_matrix((np.ones(pat.nnz), pat.colidx, pat.rowptr), shape=(n, n))
    xy = kkt_coordinates(pat)
    out = []
    stack = [(np.arange(n), False)]
    # iterative post-order: a part is emitted after its two halves, then its separator
    while stack:
        idx, expanded = stack.pop()
        if expanded:
            out.append(idx)
            continue
        if idx.size <= leaf:
            out.append(idx)
            continue
        ax = 0 if np.ptp(xy[idx, 0]) >= np.ptp(xy[idx, 1]) else 1
        med = np.median(xy[idx, ax])
        left, right = idx[xy[idx, ax] <= med], idx[xy[idx, ax] > med]
        if left.size == 0 or right.size == 0:
            out.append(idx)
            continue
        touches = np.asarray(A[left][:, right].sum(axis=1)).ravel() > 0
        sep, left = left[touches], left[~touches]
        stack.append((sep, True))
        stack.append((right, False))
        stack.append((left, False))
    return np.concatenate(out).astype(np.int32)
