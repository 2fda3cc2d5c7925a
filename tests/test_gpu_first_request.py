"""The first request of a context created while other streams keep the GPU
busy. kkt_analyze uploads the plan; the caller then issues the first
refactorization and solve on a non-blocking stream of its own, which nothing
orders after copies made on another stream, so the uploads must have reached
the device before kkt_analyze returns. Contexts are created in worker threads
(as the serving layer's analysis workers do) while background contexts run
refactorizations on further streams; every first result must meet the
backward-error tolerance (FP64 factors: no refinement is needed).
The race this guards against is timing dependent; the test repeats the
pattern to make a regression likely to show."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2302_08656_gb300 as K
from kktgen import KKTPattern, make_grid


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_first_request_after_analyze_under_load():
    dev = _dev()
    pats = [KKTPattern(make_grid(700 + i, 3000, 3840, 600)) for i in range(4)]
    inputs = [(torch.from_numpy(p.values(p.point(i, 1, 1e-3))).to(dev), torch.from_numpy(p.rhs(i, 1)).to(dev))
              for i, p in enumerate(pats)]
    # background load: contexts refactoring in a loop on their own streams
    bg = [K.KKTSolver(p.rowptr, p.colidx, p.n_primal) for p in pats[:2]]
    bg_streams = [torch.cuda.Stream() for _ in bg]
    stop = threading.Event()

    def load(i):
        while not stop.is_set():
            bg[i].refactor(inputs[i][0], stream=bg_streams[i])
            bg_streams[i].synchronize()

    loaders = [threading.Thread(target=load, args=(i,)) for i in range(len(bg))]
    for t in loaders:
        t.start()
    omegas, errors = [], []

    def first_request(i):
        try:
            p = pats[i % len(pats)]
            v, b = inputs[i % len(pats)]
            st = torch.cuda.Stream()
            s = K.KKTSolver(p.rowptr, p.colidx, p.n_primal)          # analyze in this thread
            x = torch.empty_like(b)
            om = torch.empty(1, dtype=torch.float64).pin_memory()
            s.refactor(v, stream=st)
            s.solve_checked(b, x, om, stream=st)
            st.synchronize()
            omegas.append(float(om[0]))
            s.close()
        except Exception as e:                                        # reported below
            errors.append(repr(e))

    try:
        for _ in range(4):
            workers = [threading.Thread(target=first_request, args=(i,)) for i in range(8)]
            for t in workers:
                t.start()
            for t in workers:
                t.join()
    finally:
        stop.set()
        for t in loaders:
            t.join()
        for s in bg:
            s.close()
    assert not errors, errors
    assert len(omegas) == 32
    assert max(omegas) <= 1e-10, sorted(omegas)[-3:]
