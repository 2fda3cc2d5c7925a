"""Pins of the oracle's saddle-point specialised solve (oracle/hykkt.py), on
the CPU: against a direct solve of the whole system where it is well
determined, its invariances, the algebra of its reduced operator, brute
force on a tiny grid, and a planted mistake that the checks catch."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from kktgen import KKTPattern, KKTPoint, make_grid
from oracle import hykkt


def _benign(pat, seed, step, dc=1e-3):
    """Sigma clipped to [0.1, 10], dw = 1, dc = 1e-3, slacks' term on [0.1, 10]:
    a well determined K (the graded inputs are not, see the GPU tests)."""
    p = pat.point(seed, step, 1e-3, delta_w=1.0, delta_c=dc, slack_range=(0.1, 10.0))
    sig = np.where(p.sigma > 0, np.clip(p.sigma, 0.1, 10.0), 0.0)
    return KKTPoint(p.V, p.theta, p.lam, sig, p.mu, p.delta_w, p.delta_c, p.slack_inv)


@pytest.fixture(scope="module")
def pat():
    return KKTPattern(make_grid(2, 120, 170, 24))


@pytest.mark.parametrize("gamma", [300.0, 900.0])
def test_matches_the_direct_solve_of_K(pat, gamma):
    """gamma large enough: H' is indefinite on these matrices (its Lagrangian
    Hessian part), and gamma J_E^T J_E makes the reduced operator positive
    definite (from gamma ~ 300 here; with gamma = 0 the conjugate gradients
    stall -- the reason for augmenting)."""
    mE = 2 * pat.grid.n_bus
    for step in range(3):
        K = pat.to_scipy(pat.values(_benign(pat, 4, step)))
        b = pat.rhs(4, step)
        ref = spla.spsolve(K.tocsc(), b)
        r = hykkt.solve(K, pat.n_primal, mE, b, gamma, tol=1e-14, max_iter=2000)
        assert np.max(np.abs(r.z - ref)) <= 1e-8 * np.max(np.abs(ref))
        assert r.omega <= 1e-13
        assert r.cg_iters <= mE                   # CG on an mE x mE SPD operator


def test_gamma_trades_iterations_not_the_answer(pat):
    """The method is exact for every admissible gamma; larger gamma, fewer
    conjugate-gradient iterations (the augmented operator clusters)."""
    mE = 2 * pat.grid.n_bus
    K = pat.to_scipy(pat.values(_benign(pat, 7, 1)))
    b = pat.rhs(7, 1)
    runs = [hykkt.solve(K, pat.n_primal, mE, b, g, tol=1e-13, max_iter=3000) for g in (300.0, 600.0, 900.0)]
    for r in runs[1:]:
        assert np.max(np.abs(r.z - runs[0].z)) <= 1e-8 * np.max(np.abs(runs[0].z))
    its = [r.cg_iters for r in runs]
    assert its[0] > its[1] > its[2]


def test_reduced_operator_is_symmetric_positive_definite(pat):
    """C^{1/2} J_E H_g^{-1} J_E^T C^{1/2} + D_E, formed densely from the blocks:
    symmetric, positive definite, and equal to the Schur complement of the
    augmented system (computed independently as a dense block elimination)."""
    mE = 2 * pat.grid.n_bus
    K = pat.to_scipy(pat.values(_benign(pat, 5, 2)))
    B = hykkt.blocks(K, pat.n_primal, mE)
    g = 300.0
    Hp = (B.H + B.JI.T @ sp.diags(1.0 / B.dI) @ B.JI).toarray()
    Hg = Hp + g * (B.JE.T @ B.JE).toarray()
    C = 1.0 - g * B.dE
    JE = B.JE.toarray()
    A = np.diag(np.sqrt(C)) @ JE @ np.linalg.solve(Hg, JE.T) @ np.diag(np.sqrt(C)) + np.diag(B.dE)
    assert np.allclose(A, A.T, rtol=1e-9, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    # dense block elimination of [[Hg, JE^T C], [JE, -D_E]]: Schur = D_E + JE Hg^-1 JE^T C
    M = np.block([[Hg, JE.T * C], [JE, -np.diag(B.dE)]])
    n = Hg.shape[0]
    S = -(M[n:, n:] - M[n:, :n] @ np.linalg.solve(M[:n, :n], M[:n, n:]))
    assert np.allclose(np.diag(np.sqrt(C)) @ S @ np.diag(1.0 / np.sqrt(C)), A, rtol=1e-8, atol=1e-10 * np.abs(A).max())


def test_brute_force_tiny_grid():
    """Three buses, two lines, one generator: dense numpy solve of K."""
    p = KKTPattern(make_grid(1, 3, 2, 1))
    mE = 2 * p.grid.n_bus
    for step in range(4):
        K = p.to_scipy(p.values(_benign(p, 9, step, dc=1e-2)))
        b = p.rhs(9, step)
        ref = np.linalg.solve(K.toarray(), b)
        r = hykkt.solve(K, p.n_primal, mE, b, 20.0, tol=1e-15, max_iter=100)
        assert np.allclose(r.z, ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())


def test_planted_sign_error_is_caught(pat, monkeypatch):
    """A sign error in the inequality rows' coupling (J_I negated: the
    condensed matrix is unchanged, its right-hand side and the recovery of
    y_I are not) must fail the backward-error check the tests above rely on."""
    mE = 2 * pat.grid.n_bus
    K = pat.to_scipy(pat.values(_benign(pat, 4, 0)))
    b = pat.rhs(4, 0)
    good = hykkt.solve(K, pat.n_primal, mE, b, 10.0, tol=1e-14, max_iter=2000)
    assert good.omega <= 1e-13
    real = hykkt.blocks

    def wrong(K_, p_, m_):
        B = real(K_, p_, m_)
        B.JI = -B.JI                                  # the planted mistake
        return B

    monkeypatch.setattr(hykkt, "blocks", wrong)
    bad = hykkt.solve(K, pat.n_primal, mE, b, 10.0, tol=1e-14, max_iter=2000)
    assert bad.omega > 1e-6


def test_no_inequality_rows(pat):
    """The degenerate case without inequality rows (K = [H J_E^T; J_E -D_E]):
    nothing is condensed, the method is the augmented Schur complement alone."""
    mE = 2 * pat.grid.n_bus
    K = pat.to_scipy(pat.values(_benign(pat, 6, 1)))
    m = pat.n_primal + mE
    Ke = K[:m, :m].tocsr()
    b = pat.rhs(6, 1)[:m]
    ref = spla.spsolve(Ke.tocsc(), b)
    r = hykkt.solve(Ke, pat.n_primal, mE, b, 300.0, tol=1e-14, max_iter=2000)
    assert np.max(np.abs(r.z - ref)) <= 1e-8 * np.max(np.abs(ref)) and r.omega <= 1e-13
