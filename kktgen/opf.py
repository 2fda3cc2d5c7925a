"""Seeded loads and limits that turn a synthetic grid into an ACOPF instance
(Eqs. 1-4): the data an interior-point run needs beyond the network itself.
Problem data only; no solver arithmetic.

Readings (the paper is silent on every constant; its TAMU grids are absent):
* loads Pd_i ~ U[0.02, 0.08] pu at every bus, Qd_i = Pd_i * U[0.1, 0.3]
  (light loading, so the flat start is close and every instance is feasible);
* generators: Pmin = 0, Pmax_k = 1.6 * sum(Pd) / G * U[0.8, 1.2],
  Qmax_k = Pmax_k / 2, Qmin_k = -Qmax_k;
* voltage magnitudes within [0.9, 1.1]; angles free;
* line limits |S| <= Smax = 1 pu at both ends (the squared limit is the
  flow rows' bound).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .grid import Grid


@dataclass
class OPFData:
    Pd: np.ndarray      # (B,)
    Qd: np.ndarray      # (B,)
    Vmin: np.ndarray    # (B,)
    Vmax: np.ndarray    # (B,)
    Pmin: np.ndarray    # (G,)
    Pmax: np.ndarray    # (G,)
    Qmin: np.ndarray    # (G,)
    Qmax: np.ndarray    # (G,)
    Smax: np.ndarray    # (L,)

    def bounds(self, grid: Grid):
        """Lower and upper bounds of the primal vector (V, theta, Pg, Qg);
        -inf / +inf on the angles."""
        B = grid.n_bus
        lo = np.concatenate([self.Vmin, np.full(B, -np.inf), self.Pmin, self.Qmin])
        hi = np.concatenate([self.Vmax, np.full(B, np.inf), self.Pmax, self.Qmax])
        return lo, hi


def opf_data(grid: Grid, seed: int) -> OPFData:
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x6f7066]))
    B, L, G = grid.n_bus, grid.n_branch, grid.n_gen
    Pd = rng.uniform(0.02, 0.08, size=B)
    Qd = Pd * rng.uniform(0.1, 0.3, size=B)
    Pmax = 1.6 * Pd.sum() / max(G, 1) * rng.uniform(0.8, 1.2, size=G)
    Qmax = 0.5 * Pmax
    return OPFData(Pd=Pd, Qd=Qd, Vmin=np.full(B, 0.9), Vmax=np.full(B, 1.1), Pmin=np.zeros(G), Pmax=Pmax,
                   Qmin=-Qmax, Qmax=Qmax, Smax=np.ones(L))


def flat_start(grid: Grid, data: OPFData) -> np.ndarray:
    """The usual initial point: |V| = 1, angles 0, generation at mid-range."""
    B = grid.n_bus
    return np.concatenate([np.ones(B), np.zeros(B), 0.5 * (data.Pmin + data.Pmax), 0.5 * (data.Qmin + data.Qmax)])
