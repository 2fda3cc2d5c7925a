"""Oracle of the saddle-point specialised solve (TEST INFRASTRUCTURE: only the
test suite, the smoke check and the benchmark's CPU baseline use it).

Sec. V names a solver specialised to the saddle-point structure of the KKT
systems as a way forward, without giving its method. This oracle follows the
hybrid direct-iterative approach to such systems from the literature on GPU
ACOPF solvers, written out plainly in NumPy / SciPy (FP64), in the order of
its steps. With the unknowns ordered (x, y_E, y_I) -- primal, then the dual
rows of the equality constraints (the power balance), then those of the
inequality constraints (line flows) --

    K = [ H     J_E^T  J_I^T ]        the (2,2) block diagonal:
        [ J_E  -D_E    0     ]        D_E = diag(d_E) >= 0 (regularization),
        [ J_I   0     -D_I   ]        D_I = diag(d_I) > 0 (regularization and slacks)

  condense  the inequality rows: y_I = D_I^{-1} (J_I x - r_I), so
            H' = H + J_I^T D_I^{-1} J_I,  r' = r_x + J_I^T D_I^{-1} r_I;
  augment   add gamma J_E^T times the equality rows to the first block row:
            H_g = H' + gamma J_E^T J_E,  r'' = r' + gamma J_E^T r_E,
            H_g x + J_E^T C y_E = r'' with C = I - gamma D_E (diagonal, > 0);
  Schur     eliminating x = H_g^{-1} (r'' - J_E^T C y_E) from the equality
            rows J_E x - D_E y_E = r_E gives (S C + D_E) y_E = J_E H_g^{-1} r'' - r_E,
            S = J_E H_g^{-1} J_E^T; with y_E = C^{-1/2} w the operator becomes
            the symmetric C^{1/2} S C^{1/2} + D_E, solved by conjugate gradients
            (each product one solve with H_g: factored once, here by a sparse LU);
  recover   x = H_g^{-1} (r'' - J_E^T C y_E), y_I = D_I^{-1} (J_I x - r_I).

The method is exact for any gamma >= 0 with gamma d_E < 1; gamma trades the
conjugate-gradient iterations (fewer as gamma grows) against the conditioning
of H_g. scipy.sparse.linalg.splu factors H_g (a library primitive); the
conjugate gradients are the textbook iteration.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class Blocks:
    H: sp.csr_matrix
    JE: sp.csr_matrix
    JI: sp.csr_matrix
    dE: np.ndarray
    dI: np.ndarray


def blocks(K, n_primal: int, m_eq: int) -> Blocks:
    """The blocks of K (scipy sparse, square); the (2,2) block must be diagonal."""
    K = sp.csr_matrix(K)
    n = K.shape[0]
    p, e = n_primal, n_primal + m_eq
    D = K[p:, p:]
    if (D - sp.diags(D.diagonal())).count_nonzero():
        raise ValueError("the (2,2) block is not diagonal")
    d = -D.diagonal()
    return Blocks(H=K[:p, :p].tocsr(), JE=K[p:e, :p].tocsr(), JI=K[e:, :p].tocsr(), dE=d[:m_eq].copy(),
                  dI=d[m_eq:].copy())


@dataclass
class Result:
    z: np.ndarray
    cg_iters: int
    cg_resid: float          # ||b' - A' w|| / ||b'|| at exit
    omega: float             # normwise backward error of z for K


def backward_error(K, z, b) -> float:
    K = sp.csr_matrix(K)
    r = b - K @ z
    kn = np.max(np.asarray(abs(K).sum(axis=1)).ravel())
    den = kn * np.max(np.abs(z)) + np.max(np.abs(b))
    return float(np.max(np.abs(r)) / den) if den > 0 else float(np.max(np.abs(r)))


def solve(K, n_primal: int, m_eq: int, b, gamma: float, tol: float = 1e-12, max_iter: int = 200) -> Result:
    B = blocks(K, n_primal, m_eq)
    if np.any(B.dI <= 0):
        raise ValueError("the inequality rows need D_I > 0")
    C = 1.0 - gamma * B.dE
    if np.any(C <= 0):
        raise ValueError("gamma d_E must stay below 1")
    p, e = n_primal, n_primal + m_eq
    b = np.asarray(b, dtype=np.float64)
    rx, rE, rI = b[:p], b[p:e], b[e:]
    # condense the inequality rows
    Hp = B.H + B.JI.T @ sp.diags(1.0 / B.dI) @ B.JI
    rp = rx + B.JI.T @ (rI / B.dI)
    # augment with gamma J_E^T J_E
    Hg = (Hp + gamma * (B.JE.T @ B.JE)).tocsc()
    r2 = rp + gamma * (B.JE.T @ rE)
    lu = spla.splu(Hg)
    sq = np.sqrt(C)

    def op(w):                               # (C^{1/2} S C^{1/2} + D_E) w
        return sq * (B.JE @ lu.solve(B.JE.T @ (sq * w))) + B.dE * w

    rhs = sq * (B.JE @ lu.solve(r2) - rE)
    # conjugate gradients from w = 0
    w = np.zeros(m_eq)
    r = rhs.copy()
    d = r.copy()
    rr = float(r @ r)
    nb = float(np.linalg.norm(rhs))
    it = 0
    while it < max_iter and np.sqrt(rr) > tol * nb:
        q = op(d)
        a = rr / float(d @ q)
        w += a * d
        r -= a * q
        rn = float(r @ r)
        d = r + (rn / rr) * d
        rr = rn
        it += 1
    yE = w / sq
    x = lu.solve(r2 - B.JE.T @ (C * yE))
    yI = (B.JI @ x - rI) / B.dI
    z = np.concatenate([x, yE, yI])
    return Result(z=z, cg_iters=it, cg_resid=float(np.sqrt(rr) / nb) if nb > 0 else 0.0,
                  omega=backward_error(K, z, b))
