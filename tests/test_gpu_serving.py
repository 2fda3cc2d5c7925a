"""Serving on the GPU: a mix of sessions of different sizes under a small
memory budget (admission binds); every result must equal the same session's
result computed alone, and meet the backward-error tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import paper_2302_08656_gb300 as K
from paper_2302_08656_gb300.serve import GpuBackend, Server, SessionSpec, estimate_bytes, poisson_arrivals
from kktgen import KKTPattern, make_grid


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_results_alone_equal_results_in_the_mix():
    dev = _dev()
    rng = np.random.default_rng(3)
    sizes = [120, 300, 650, 200, 900, 450]
    reqs = 4
    arrivals = poisson_arrivals(rng, 3000.0, [reqs] * len(sizes))
    pats, sessions, host = [], [], {}
    for sid, B in enumerate(sizes):
        pat = KKTPattern(make_grid(50 + sid, B, int(1.28 * B), max(1, B // 5)))
        pats.append(pat)
        vals = [torch.from_numpy(pat.values(pat.point(sid, k, 10.0 ** -(1 + k)))).to(dev) for k in range(reqs)]
        rhs = [torch.from_numpy(pat.rhs(sid, k)).to(dev) for k in range(reqs)]
        host[sid] = (vals, rhs)
        sessions.append(SessionSpec(sid, pat.rowptr, pat.colidx, pat.n_primal, arrivals[sid],
                                    (lambda v, r: (lambda k: (v[k], r[k])))(vals, rhs),
                                    est_bytes=estimate_bytes(pat.nnz)))
    budget = sum(sorted(s.est_bytes for s in sessions)[-2:])     # roughly two sessions at a time
    be = GpuBackend(precision="fp32", tol=1e-10, streams=4, keep_results=True)
    rep = Server(be, budget_bytes=budget, max_inflight=4).run(sessions)
    assert rep.completed == reqs * len(sizes)
    assert rep.admission_waits > 0
    assert max(rep.omegas) <= 1e-10
    for sid, pat in enumerate(pats):
        solo = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, precision="fp32")
        omega = torch.empty(1, dtype=torch.float64).pin_memory()
        for k in range(reqs):
            v, b = host[sid][0][k], host[sid][1][k]
            x = torch.empty_like(b)
            solo.refactor(v)
            solo.solve_checked(b, x, omega)
            torch.cuda.synchronize()
            if not float(omega[0]) <= 1e-10:
                x, _ = solo.refine(b, out=x, tol=1e-10)
            xs = x.cpu().numpy()
            assert np.array_equal(xs, be.results[(sid, k)]), (sid, k)
            assert O.backward_error(pat.rowptr, pat.colidx, v.cpu().numpy(), xs, b.cpu().numpy()) <= 1e-10
        solo.close()
