"""Seeded synthetic transmission grids shaped like the paper's test systems.

The paper evaluates on the TAMU synthetic Northeast (25,000 buses, 32,230
branches, 4,834 generators) and Eastern (70,000 buses, 88,270 branches,
10,390 generators) grids (Table I). Those data sets are not available here, so
this module draws grids with the same bus / branch / generator counts and the
sparse, irregular, nearly planar connectivity the paper describes for these
KKT matrices (Sec. II).

Recipe (the paper is silent on every constant; these are the readings used):

* buses at uniform random points of the unit square;
* candidate lines = k-nearest-neighbour pairs (k = 8), so every line is local;
* a random spanning tree by Kruskal's algorithm over the candidates in random
  order (components that the candidates leave apart are joined by their
  closest pair of buses);
* extra lines drawn uniformly, without repetition, from the candidates not in
  the tree, until the branch count is reached;
* branch resistance r ~ U[0.001, 0.01] pu and reactance x ~ U[0.01, 0.1] pu;
* generators at distinct uniformly drawn buses, quadratic cost coefficient
  c2 ~ U[0.01, 0.1].

``locality=False`` draws extra lines between uniformly random bus pairs
instead (a stress case whose fill behaves like an expander graph).

Nothing here performs any linear-solver arithmetic: the module only produces
problem data.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial import cKDTree


@dataclass
class Grid:
    n_bus: int
    n_branch: int
    n_gen: int
    xy: np.ndarray          # (B, 2) bus coordinates
    f: np.ndarray           # (L,) from-bus of each branch
    t: np.ndarray           # (L,) to-bus of each branch
    r: np.ndarray           # (L,) series resistance, pu
    x: np.ndarray           # (L,) series reactance, pu
    gen_bus: np.ndarray     # (G,) bus of each generator (distinct)
    c2: np.ndarray          # (G,) quadratic cost coefficient
    tree_parent: np.ndarray  # (B,) parent in the spanning tree, -1 at the root
    tree_order: np.ndarray   # (B,) breadth-first order of the spanning tree
    tree_edge_dir: np.ndarray  # (B,) for non-root buses: the branch to the parent

    @property
    def g(self) -> np.ndarray:
        return self.r / (self.r * self.r + self.x * self.x)

    @property
    def b(self) -> np.ndarray:
        return -self.x / (self.r * self.r + self.x * self.x)


def _find(parent: np.ndarray, a: int) -> int:
    root = a
    while parent[root] != root:
        root = parent[root]
    while parent[a] != root:
        nxt = parent[a]
        parent[a] = root
        a = nxt
    return root


def make_grid(seed: int, n_bus: int, n_branch: int | None = None,
              n_gen: int | None = None, knn: int = 8,
              locality: bool = True) -> Grid:
    """Draw one grid. Unstated counts default to L = 1.28 B and G = 0.2 B."""
    B = int(n_bus)
    L = int(round(1.28 * B)) if n_branch is None else int(n_branch)
    G = max(1, int(round(0.2 * B))) if n_gen is None else int(n_gen)
    if B < 2 or L < B - 1 or G > B:
        raise ValueError("need B >= 2, L >= B-1 and G <= B")
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x6772_6964]))
    xy = rng.random((B, 2))
    k = min(knn + 1, B)
    tree = cKDTree(xy)
    _, nb = tree.query(xy, k=k)
    a = np.repeat(np.arange(B), k - 1)
    c = nb[:, 1:].reshape(-1)
    lo, hi = np.minimum(a, c), np.maximum(a, c)
    keep = lo != hi
    cand = np.unique(lo[keep].astype(np.int64) * B + hi[keep])
    cand = cand[rng.permutation(cand.size)]

    # Kruskal in random order = a uniformly random spanning forest of the kNN graph.
    uf = np.arange(B)
    in_tree = np.zeros(cand.size, dtype=bool)
    n_comp = B
    cu, cv = (cand // B).astype(np.int64), (cand % B).astype(np.int64)
    for e in range(cand.size):
        ru, rv = _find(uf, int(cu[e])), _find(uf, int(cv[e]))
        if ru != rv:
            uf[ru] = rv
            in_tree[e] = True
            n_comp -= 1
            if n_comp == 1:
                break
    tree_u = list(cu[in_tree])
    tree_v = list(cv[in_tree])
    # join leftover components by their closest bus pair
    while n_comp > 1:
        roots = np.array([_find(uf, i) for i in range(B)])
        comp_ids, sizes = np.unique(roots, return_counts=True)
        small = comp_ids[np.argmin(sizes)]
        members = np.nonzero(roots == small)[0]
        best = (np.inf, -1, -1)
        kk = min(B, 32)
        while best[1] < 0:
            d, idx = tree.query(xy[members], k=kk)
            for row, m in enumerate(members):
                for dist, j in zip(d[row], idx[row]):
                    if roots[j] != small and dist < best[0]:
                        best = (dist, int(m), int(j))
            kk = min(B, kk * 4)
        _, u, v = best
        uf[_find(uf, u)] = _find(uf, v)
        tree_u.append(u)
        tree_v.append(v)
        n_comp -= 1

    tree_u = np.array(tree_u, dtype=np.int64)
    tree_v = np.array(tree_v, dtype=np.int64)
    n_extra = L - (B - 1)
    if locality:
        rest = cand[~in_tree]
        tree_keys = np.minimum(tree_u, tree_v) * B + np.maximum(tree_u, tree_v)
        rest = rest[~np.isin(rest, tree_keys)]
        if rest.size < n_extra:
            raise ValueError("not enough nearest-neighbour candidates for the branch count")
        extra = rest[rng.choice(rest.size, size=n_extra, replace=False)]
    else:
        used = set((np.minimum(tree_u, tree_v) * B + np.maximum(tree_u, tree_v)).tolist())
        extra_l = []
        while len(extra_l) < n_extra:
            p, q = rng.integers(0, B, size=2)
            if p == q:
                continue
            key = int(min(p, q)) * B + int(max(p, q))
            if key not in used:
                used.add(key)
                extra_l.append(key)
        extra = np.array(extra_l, dtype=np.int64)
    f = np.concatenate([tree_u, extra // B]).astype(np.int64)
    t = np.concatenate([tree_v, extra % B]).astype(np.int64)
    r = rng.uniform(0.001, 0.01, size=L)
    x = rng.uniform(0.01, 0.1, size=L)
    gen_bus = np.sort(rng.choice(B, size=G, replace=False)).astype(np.int64)
    c2 = rng.uniform(0.01, 0.1, size=G)

    # breadth-first spanning-tree order from bus 0 (used for the angle walk)
    adj_ptr = np.zeros(B + 1, dtype=np.int64)
    ends = np.concatenate([tree_u, tree_v])
    others = np.concatenate([tree_v, tree_u])
    eid = np.concatenate([np.arange(B - 1), np.arange(B - 1)])
    order = np.argsort(ends, kind="stable")
    np.add.at(adj_ptr, ends + 1, 1)
    adj_ptr = np.cumsum(adj_ptr)
    adj = others[order]
    adj_e = eid[order]
    parent = np.full(B, -1, dtype=np.int64)
    pedge = np.full(B, -1, dtype=np.int64)
    seen = np.zeros(B, dtype=bool)
    bfs = np.empty(B, dtype=np.int64)
    bfs[0] = 0
    seen[0] = True
    head, tail = 0, 1
    while head < tail:
        u = bfs[head]
        head += 1
        for p in range(adj_ptr[u], adj_ptr[u + 1]):
            v = adj[p]
            if not seen[v]:
                seen[v] = True
                parent[v] = u
                pedge[v] = adj_e[p]
                bfs[tail] = v
                tail += 1
    if tail != B:
        raise RuntimeError("spanning tree does not reach every bus")
    return Grid(B, L, G, xy, f, t, r, x, gen_bus, c2, parent, bfs, pedge)
