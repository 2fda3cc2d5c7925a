"""Host-side scheduling of the serving loop with a fake backend (no GPU):
admission by memory budget, one request in flight per session, release after
the previous result, bounded in-flight window."""
import numpy as np

from paper_2302_08656_gb300.serve import Server, SessionSpec, poisson_arrivals


class FakeBackend:
    def __init__(self, service_s=0.002):
        self.service = service_s
        self.log = []
        self.open_now = 0
        self.max_open = 0
        self.inflight = 0
        self.max_inflight = 0

    def open(self, spec):
        self.open_now += 1
        self.max_open = max(self.max_open, self.open_now)
        return dict(spec=spec)

    def bytes_of(self, h, spec):
        return spec.est_bytes

    def issue(self, h, k):
        import time
        t = time.perf_counter()
        self.log.append((h["spec"].sid, k, t))
        self.inflight += 1
        self.max_inflight = max(self.max_inflight, self.inflight)
        return dict(h=h, k=k, done=t + self.service)

    def poll(self, t):
        import time
        return time.perf_counter() >= t["done"]

    def finish(self, t):
        self.inflight -= 1
        return 1e-14, False

    def close(self, h):
        self.open_now -= 1


def _sessions(n, reqs, rate, bytes_each, seed=0):
    rng = np.random.default_rng(seed)
    arr = poisson_arrivals(rng, rate, [reqs] * n)
    return [SessionSpec(i, None, None, 0, arr[i], None, est_bytes=bytes_each) for i in range(n)]


def test_all_requests_complete_in_order():
    be = FakeBackend()
    sess = _sessions(8, 5, 4000.0, 10)
    rep = Server(be, budget_bytes=10 ** 9, max_inflight=4).run(sess)
    assert rep.completed == 40
    for s in sess:
        ks = [k for sid, k, _ in be.log if sid == s.sid]
        assert ks == list(range(5))                      # one request at a time, in order
    assert min(rep.latencies_ms) >= 1.9                  # never faster than the service time
    assert max(rep.omegas) <= 1e-10


def test_budget_binds_admission():
    be = FakeBackend()
    sess = _sessions(6, 3, 10000.0, 100)
    rep = Server(be, budget_bytes=250, max_inflight=8).run(sess)
    assert rep.completed == 18
    assert rep.max_bytes <= 250
    assert be.max_open <= 2                              # at most two 100-byte sessions at once
    assert rep.admission_waits > 0


def test_inflight_window_is_respected():
    be = FakeBackend(service_s=0.003)
    sess = _sessions(10, 2, 1e6, 1)                       # everything arrives at once
    rep = Server(be, budget_bytes=10 ** 9, max_inflight=3).run(sess)
    assert rep.completed == 20
    assert be.max_inflight == 3
    assert rep.max_sessions <= 10
