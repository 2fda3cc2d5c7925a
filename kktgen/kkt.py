"""ACOPF KKT matrices K_k (Eq. 11) on a synthetic grid, in full symmetric CSR.

Formulation (Eqs. 1-4, written in polar voltages, no shunts, unit taps):

* primal x = (V_1..V_B, theta_1..theta_B, Pg_1..Pg_G, Qg_1..Qg_G), n = 2B + 2G;
* equalities g(x) = 0: active and reactive power balance at every bus,
  Pbal_i = sum_{gens at i} Pg - Pd_i - sum_{lines at i} P_line (flow leaving i),
  and likewise for Q;
* inequalities h(x) <= h+: apparent-power limits P^2 + Q^2 <= Smax^2 at both
  ends of every branch (set ``flow_limits=False`` for the paper's Table I
  shape, which has no such rows);
* objective F(x) = sum c2 Pg^2.

After the interior-point method eliminates the bound multipliers and the
inequality slacks, the Newton system is the symmetric indefinite

    K = [[H + Sigma + dw I,  J^T],
         [J,              -dc I]]

with H the Hessian of the Lagrangian (Sec. II), J the constraint Jacobian
(m x n), Sigma the barrier diagonal D_y = mu Y^-2 and dw, dc the usual
primal / dual regularisations. Eq. 11 prints the (2,1) block as J^T and the
(2,2) block as 0; the reading used here puts J (m x n) below H and a -dc
diagonal in the (2,2) block so the matrix is nonsingular at every mu.

Barrier reading: for every bounded primal (V, Pg, Qg) the slack-like
variable y_i is drawn log-uniform on [sqrt(mu/1e8), sqrt(mu/1e-8)], so that
Sigma_i = mu / y_i^2 is log-uniform on [1e-8, 1e8] at every mu. Angles are
unbounded and get only dw.

All K_k of one grid share one sparsity pattern (Sec. II); ``KKTPattern``
holds it and ``KKTPattern.values`` fills it for one interior-point step.
This module holds problem data only; no linear-solver arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .grid import Grid


def branch_terms(Vi, Vj, ti, tj, g, b):
    """Flow P, Q leaving bus i on a line to bus j, with gradients and Hessians.

    Local variable order is (Vi, Vj, theta_i, theta_j). With
    A = g cos(ti-tj) + b sin(ti-tj) and A' = dA/dti:
        P = g Vi^2 - Vi Vj A
        Q = -b Vi^2 + Vi Vj A'
    Returns P, Q (L,), dP, dQ (4, L), HP, HQ (4, 4, L).
    """
    th = ti - tj
    c, s = np.cos(th), np.sin(th)
    A = g * c + b * s
    Ap = -g * s + b * c          # dA/dti
    Bq = -Ap                      # g s - b c
    P = g * Vi * Vi - Vi * Vj * A
    Q = -b * Vi * Vi - Vi * Vj * Bq
    ViVj = Vi * Vj
    z = np.zeros_like(Vi)
    dP = np.stack([2 * g * Vi - Vj * A, -Vi * A, -ViVj * Ap, ViVj * Ap])
    dQ = np.stack([-2 * b * Vi - Vj * Bq, -Vi * Bq, -ViVj * A, ViVj * A])
    HP = np.array([
        [2 * g + z, -A, -Vj * Ap, Vj * Ap],
        [-A, z, -Vi * Ap, Vi * Ap],
        [-Vj * Ap, -Vi * Ap, ViVj * A, -ViVj * A],
        [Vj * Ap, Vi * Ap, -ViVj * A, ViVj * A],
    ])
    HQ = np.array([
        [-2 * b + z, -Bq, -Vj * A, Vj * A],
        [-Bq, z, -Vi * A, Vi * A],
        [-Vj * A, -Vi * A, -ViVj * Ap, ViVj * Ap],
        [Vj * A, Vi * A, ViVj * Ap, -ViVj * Ap],
    ])
    return P, Q, dP, dQ, HP, HQ


_SWAP = np.array([1, 0, 3, 2])   # (Vj, Vi, tj, ti) -> (Vi, Vj, ti, tj)


def line_terms(grid: Grid, V, theta):
    """From-end and to-end flows of every branch in local order (Vi, Vj, ti, tj)."""
    i, j = grid.f, grid.t
    g, b = grid.g, grid.b
    Pf, Qf, dPf, dQf, HPf, HQf = branch_terms(V[i], V[j], theta[i], theta[j], g, b)
    Pt, Qt, dPt, dQt, HPt, HQt = branch_terms(V[j], V[i], theta[j], theta[i], g, b)
    dPt, dQt = dPt[_SWAP], dQt[_SWAP]
    HPt, HQt = HPt[_SWAP][:, _SWAP], HQt[_SWAP][:, _SWAP]
    return (Pf, Qf, dPf, dQf, HPf, HQf), (Pt, Qt, dPt, dQt, HPt, HQt)


@dataclass
class KKTPoint:
    """One interior-point iterate: everything K_k depends on."""
    V: np.ndarray
    theta: np.ndarray
    lam: np.ndarray
    sigma: np.ndarray     # (n,) barrier diagonal, 0 on angles
    mu: float
    delta_w: float
    delta_c: float
    slack_inv: np.ndarray = None   # (m,) 1/sigma_s on inequality rows (0 elsewhere), or None


class KKTPattern:
    """The fixed sparsity pattern of K for one grid, and its value assembly."""

    def __init__(self, grid: Grid, flow_limits: bool = True):
        self.grid = grid
        self.flow_limits = bool(flow_limits)
        B, L, G = grid.n_bus, grid.n_branch, grid.n_gen
        self.n_primal = n = 2 * B + 2 * G
        self.n_dual = m = 2 * B + (2 * L if flow_limits else 0)
        self.n = N = n + m
        i, j = grid.f, grid.t
        loc = np.stack([i, j, B + i, B + j])                       # (4, L)
        self._loc = loc
        rows, cols = [], []
        # H: one dense 4x4 block per line
        for a in range(4):
            for c in range(4):
                rows.append(loc[a]); cols.append(loc[c])
        # primal diagonal
        rows.append(np.arange(n)); cols.append(np.arange(n))
        # J rows: balance rows (from- and to-end contributions), generators, flow rows
        jr, jc = [], []
        rP, rQ = n + np.arange(B), n + B + np.arange(B)
        for a in range(4):
            jr += [rP[i], rP[j], rQ[i], rQ[j]]
            jc += [loc[a]] * 4
        gb = grid.gen_bus
        jr += [rP[gb], rQ[gb]]
        jc += [2 * B + np.arange(G), 2 * B + G + np.arange(G)]
        if flow_limits:
            rF, rT = n + 2 * B + np.arange(L), n + 2 * B + L + np.arange(L)
            for a in range(4):
                jr += [rF, rT]
                jc += [loc[a], loc[a]]
        jr = np.concatenate(jr); jc = np.concatenate(jc)
        rows += [jr, jc]; cols += [jc, jr]
        rows.append(n + np.arange(m)); cols.append(n + np.arange(m))
        r = np.concatenate(rows).astype(np.int64)
        c = np.concatenate(cols).astype(np.int64)
        keys, inv = np.unique(r * N + c, return_inverse=True)
        self._inv = inv
        self._n_trip = r.size
        self.nnz = keys.size
        self.colidx = (keys % N).astype(np.int32)
        counts = np.bincount((keys // N).astype(np.int64), minlength=N)
        self.rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)

    # ------------------------------------------------------------------ draws
    def point(self, seed: int, step: int, mu: float = 1e-1,
              delta_w: float = 1e-8, delta_c: float = 1e-10, slack_range=None) -> KKTPoint:
        """Seeded iterate (V, theta, lambda, Sigma) for interior-point step ``step``.

        slack_range = (lo, hi): keep the inequality slacks' term in the (2,2)
        block, -(dc + 1/sigma_s) on every flow-limit row instead of -dc, with
        1/sigma_s = s_s / z_s log-uniform on [lo, hi] (the range of Sigma,
        (1e-8, 1e8), is the reading that matches the barrier diagonal). None:
        the literal -dc. Drawn from a stream of its own: every other value is
        the same with or without it."""
        g = self.grid
        rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(step), 0x6b6b74]))
        V = rng.uniform(0.95, 1.05, size=g.n_bus)
        dth = rng.normal(0.0, 0.1, size=g.n_bus)
        theta = np.zeros(g.n_bus)
        for v in g.tree_order[1:]:
            theta[v] = theta[g.tree_parent[v]] + dth[v]
        lam = rng.normal(0.0, 1.0, size=self.n_dual)
        lo, hi = np.log(np.sqrt(mu / 1e8)), np.log(np.sqrt(mu / 1e-8))
        y = np.exp(rng.uniform(lo, hi, size=self.n_primal))
        sigma = mu / (y * y)
        sigma[g.n_bus:2 * g.n_bus] = 0.0
        slack_inv = None
        if slack_range is not None:
            r2 = np.random.default_rng(np.random.SeedSequence([int(seed), int(step), 0x736c6b]))
            slack_inv = np.zeros(self.n_dual)
            a, b = np.log(float(slack_range[0])), np.log(float(slack_range[1]))
            slack_inv[2 * g.n_bus:] = np.exp(r2.uniform(a, b, size=self.n_dual - 2 * g.n_bus))
        return KKTPoint(V, theta, lam, sigma, float(mu), float(delta_w), float(delta_c), slack_inv)

    def rhs(self, seed: int, step: int) -> np.ndarray:
        rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(step), 0x726873]))
        return rng.normal(0.0, 1.0, size=self.n)

    # --------------------------------------------------------------- assembly
    def jacobian_blocks(self, V, theta):
        """Per-triplet Jacobian values in the order the pattern lists J."""
        g = self.grid
        (Pf, Qf, dPf, dQf, _, _), (Pt, Qt, dPt, dQt, _, _) = line_terms(g, V, theta)
        vals = []
        for a in range(4):
            vals += [-dPf[a], -dPt[a], -dQf[a], -dQt[a]]
        vals += [np.ones(g.n_gen), np.ones(g.n_gen)]
        if self.flow_limits:
            for a in range(4):
                vals += [2 * Pf * dPf[a] + 2 * Qf * dQf[a], 2 * Pt * dPt[a] + 2 * Qt * dQt[a]]
        return np.concatenate(vals)

    def hessian_blocks(self, V, theta, lam):
        """4x4 Hessian-of-Lagrangian block of every line (constraint part)."""
        g = self.grid
        B, L = g.n_bus, g.n_branch
        i, j = g.f, g.t
        (Pf, Qf, dPf, dQf, HPf, HQf), (Pt, Qt, dPt, dQt, HPt, HQt) = line_terms(g, V, theta)
        lP, lQ = lam[:B], lam[B:2 * B]
        Hb = -(lP[i] * HPf + lP[j] * HPt + lQ[i] * HQf + lQ[j] * HQt)
        if self.flow_limits:
            lF, lT = lam[2 * B:2 * B + L], lam[2 * B + L:]
            for (P, Q, dP, dQ, HP, HQ), lw in (((Pf, Qf, dPf, dQf, HPf, HQf), lF),
                                              ((Pt, Qt, dPt, dQt, HPt, HQt), lT)):
                outer = dP[:, None, :] * dP[None, :, :] + dQ[:, None, :] * dQ[None, :, :]
                Hb = Hb + lw * 2.0 * (outer + P * HP + Q * HQ)
        return Hb

    def values(self, pt: KKTPoint) -> np.ndarray:
        """CSR values of K at one iterate (same order as ``colidx``)."""
        g = self.grid
        B, G = g.n_bus, g.n_gen
        Hb = self.hessian_blocks(pt.V, pt.theta, pt.lam)
        trip = [Hb.reshape(16, -1).reshape(-1)]
        diag = pt.sigma + pt.delta_w
        diag = diag.copy()
        diag[2 * B:2 * B + G] += 2.0 * g.c2               # objective Hessian
        trip.append(diag)
        jv = self.jacobian_blocks(pt.V, pt.theta)
        trip += [jv, jv]
        dual = np.full(self.n_dual, -pt.delta_c)
        if pt.slack_inv is not None:
            dual -= pt.slack_inv
        trip.append(dual)
        w = np.concatenate(trip)
        assert w.size == self._n_trip
        return np.bincount(self._inv, weights=w, minlength=self.nnz)

    def to_scipy(self, vals):
        import scipy.sparse as sp
        return sp.csr_matrix((vals, self.colidx, self.rowptr), shape=(self.n, self.n))


def mu_schedule(mu0: float, mu1: float, steps: int) -> np.ndarray:
    """Geometric barrier schedule mu0 -> mu1 over ``steps`` steps (continuation mu -> 0)."""
    if steps == 1:
        return np.array([mu0])
    return np.geomspace(mu0, mu1, steps)


# Workloads (sizes from the paper's Table I grids and the configurations used
# for parity and measurement).
WORKLOADS = {
    "grid200": dict(n_bus=200, n_branch=300, n_gen=40, steps=10, mu0=1e-1, mu1=1e-8),
    "northeast25k": dict(n_bus=25_000, n_branch=32_000, n_gen=5_000, steps=100, mu0=1e-1, mu1=1e-9),
    "eastern70k": dict(n_bus=70_000, n_branch=88_000, n_gen=10_000, steps=100, mu0=1e-1, mu1=1e-9),
    "batch2k": dict(n_bus=2_000, n_branch=2_560, n_gen=400, steps=50, mu0=1e-1, mu1=1e-9),
    "batch10k": dict(n_bus=10_000, n_branch=12_800, n_gen=2_000, steps=50, mu0=1e-1, mu1=1e-9),
}
