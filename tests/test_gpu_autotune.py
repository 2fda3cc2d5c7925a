"""Schedule autotuner: times every (max_pivots, tree_min_fronts) candidate
with the fused refactor + refine call, keeps the fastest, caches it per
(pattern, precision, instance count), and the chosen schedule solves the
system like any other."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
import paper_2302_08656_gb300 as K
from paper_2302_08656_gb300 import autotune
from kktgen import KKTPattern, make_grid


def test_tuner_picks_a_candidate_and_caches_it(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    monkeypatch.setattr(autotune, "_CACHE_FILE", str(tmp_path / "tune.json"))
    pat = KKTPattern(make_grid(1, 200, 300, 40))
    count = 2
    vals = np.concatenate([pat.values(pat.point(60 + i, 1, 1e-3)) for i in range(count)])
    rhs = np.concatenate([pat.rhs(60 + i, 1) for i in range(count)])
    v, b = torch.from_numpy(vals).to(dev), torch.from_numpy(rhs).to(dev)
    best, times = autotune.tune(pat.rowptr, pat.colidx, pat.n_primal, v, b, precision="fp32", count=count,
                                candidates=(8, 16), tree_candidates=(0, 2432), reps=2)
    assert set(times) == {"8/0", "8/2432", "16/0", "16/2432"} and all(t > 0 for t in times.values())
    assert best["max_pivots"] in (8, 16) and best["tree_min_fronts"] in (0, 2432)
    assert times["%d/%d" % (best["max_pivots"], best["tree_min_fronts"])] == min(times.values())
    again, t2 = autotune.tune(pat.rowptr, pat.colidx, pat.n_primal, v, b, precision="fp32", count=count,
                              candidates=(8, 16), tree_candidates=(0, 2432))
    assert again == best and t2 == times                       # from the cache
    s = K.KKTSolver(pat.rowptr, pat.colidx, pat.n_primal, count=count, precision="fp32", **best)
    x, infos = s.refactor_refine(v, b, tol=1e-10)
    x = x.cpu().numpy()
    for i in range(count):
        om = O.backward_error(pat.rowptr, pat.colidx, vals[i * pat.nnz:(i + 1) * pat.nnz],
                              x[i * pat.n:(i + 1) * pat.n], rhs[i * pat.n:(i + 1) * pat.n])
        assert om <= 1e-10
    s.close()
