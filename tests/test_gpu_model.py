"""GPU model evaluation (the KKT values of an interior-point iterate, Eq. 11
from the ACOPF model of Eqs. 1-4) against the seeded generator's assembly,
which test_kktgen.py pins to central differences of an independent
complex-power formulation.

Tolerance: the two assemblies form every term with different roundings
(device vs host trigonometric functions, different operation orders) and sum
the terms in different orders. Each term is a short sum of products whose
magnitudes are bounded per line by the line admittance Y = |g| + |b| and the
multipliers (|V| <= 1.05): Hessian entries by 2.2 Y (sum of |balance
multipliers|) + 61 Y^2 (sum of |flow multipliers|), balance-Jacobian entries
by 3.2 Y, flow-Jacobian entries by 30 Y^2. An entry must agree within
64 u times the sum of those bounds over the terms landing on it, plus
64 u |diagonal part| (u = 2^-53): a first-order rounding bound with a
generous constant, independent of any cancellation inside a term."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _term_bounds(pat, pt):
    """Per nonzero: the sum of the magnitude bounds of the terms landing on it,
    laid out like the generator's triplets (16 Hessian blocks of L, the
    primal diagonal, the Jacobian and its transpose, the dual diagonal)."""
    g = pat.grid
    B, L, G = g.n_bus, g.n_branch, g.n_gen
    Y = np.abs(g.g) + np.abs(g.b)
    lam = np.abs(pt.lam)
    lbal = lam[g.f] + lam[g.t] + lam[B + g.f] + lam[B + g.t]
    hb = 2.2 * Y * lbal
    if pat.flow_limits:
        hb = hb + 61.0 * Y * Y * (lam[2 * B:2 * B + L] + lam[2 * B + L:])
    diag = pt.sigma + pt.delta_w
    diag = diag.copy()
    diag[2 * B:2 * B + G] += 2.0 * g.c2
    jb = [np.tile(3.2 * Y, 16), np.zeros(2 * G)]
    if pat.flow_limits:
        jb.append(np.tile(30.0 * Y * Y, 8))
    jb = np.concatenate(jb)
    w = np.concatenate([np.tile(hb, 16), np.abs(diag), jb, jb, np.full(pat.n_dual, pt.delta_c)])
    assert w.size == pat._inv.size
    return np.bincount(pat._inv, weights=w, minlength=pat.nnz)


def _assemble(m, pt, dev):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
    return m.assemble(t(pt.V), t(pt.theta), t(pt.lam), t(pt.sigma), pt.delta_w, pt.delta_c)


@pytest.mark.parametrize("args", [(1, 200, 300, 40), (3, 30, 40, 6), (7, 25_000, 32_000, 5_000)])
@pytest.mark.parametrize("flow", [True, False])
def test_assembled_values_match_generator(args, flow):
    dev = _dev()
    g = make_grid(*args)
    pat = KKTPattern(g, flow_limits=flow)
    m = K.KKTModel.from_grid(g, flow_limits=flow)
    assert np.array_equal(m.rowptr, pat.rowptr) and np.array_equal(m.colidx, pat.colidx)
    for step, mu in ((0, 1e-1), (5, 1e-6)):
        pt = pat.point(args[0], step, mu)
        ora = pat.values(pt)
        gpu = _assemble(m, pt, dev).cpu().numpy()
        tol = 64 * 2.0 ** -53 * _term_bounds(pat, pt)
        err = np.abs(gpu - ora)
        assert np.all(err <= tol), float((err / tol).max())
        again = _assemble(m, pt, dev).cpu().numpy()
        assert np.array_equal(gpu, again)                    # deterministic
    m.close()


def test_ipm_step_from_gpu_assembled_values():
    """Assemble on the GPU, refactor and refine: the solution meets the
    backward-error target on the generator's K (the oracle's matrix)."""
    dev = _dev()
    g = make_grid(1, 200, 300, 40)
    pat = KKTPattern(g)
    m = K.KKTModel.from_grid(g)
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal)
    for step, mu in enumerate((1e-1, 1e-4, 1e-8)):
        pt = pat.point(1, step, mu)
        vals = _assemble(m, pt, dev)
        s.refactor(vals)
        b = pat.rhs(1, step)
        x, info = s.refine(torch.from_numpy(b).to(dev), tol=1e-10)
        om = O.backward_error(pat.rowptr, pat.colidx, pat.values(pt), x.cpu().numpy(), b)
        assert om <= 1e-10, om
    s.close()
    m.close()


def test_assembled_values_with_the_slacks_term_match_generator():
    """The (2,2) diagonal with the eliminated slacks' term s/w on the flow rows
    (dual_diag): the generator's slack_inv assembly, within the same bound."""
    dev = _dev()
    g = make_grid(1, 200, 300, 40)
    pat = KKTPattern(g)
    m = K.KKTModel.from_grid(g)
    pt = pat.point(1, 3, 1e-3, slack_range=(1e-2, 1e2))
    ora = pat.values(pt)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)   # noqa: E731
    gpu = m.assemble(t(pt.V), t(pt.theta), t(pt.lam), t(pt.sigma), pt.delta_w, pt.delta_c,
                     dual_diag=t(pt.slack_inv)).cpu().numpy()
    tol = 64 * 2.0 ** -53 * (_term_bounds(pat, pt) + np.bincount(pat._inv[-pat.n_dual:], weights=pt.slack_inv,
                                                                  minlength=pat.nnz))
    assert np.all(np.abs(gpu - ora) <= tol)
    m.close()
