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


class FailingBackend(FakeBackend):
    """Fails the analysis of one session and one request of two others."""

    def __init__(self, fail_open=(), fail_issue=(), fail_finish=()):
        super().__init__()
        self.fail_open, self.fail_issue, self.fail_finish = set(fail_open), set(fail_issue), set(fail_finish)
        self.closed = []

    def open(self, spec):
        if spec.sid in self.fail_open:
            raise RuntimeError("analysis failed")
        return super().open(spec)

    def issue(self, h, k):
        if (h["spec"].sid, k) in self.fail_issue:
            raise RuntimeError("launch failed")
        return super().issue(h, k)

    def finish(self, t):
        if (t["h"]["spec"].sid, t["k"]) in self.fail_finish:
            self.inflight -= 1
            raise RuntimeError("numeric failure")
        return super().finish(t)

    def close(self, h):
        self.closed.append(h["spec"].sid)
        super().close(h)


def test_a_failure_ends_only_its_session():
    be = FailingBackend(fail_open=[2], fail_issue=[(4, 1)], fail_finish=[(6, 2)])
    sess = _sessions(8, 4, 4000.0, 10)
    rep = Server(be, budget_bytes=10 ** 9, max_inflight=4).run(sess)
    assert sorted((sid, k) for sid, k, _ in rep.failed) == [(2, -1), (4, 1), (6, 2)]
    assert all(err.startswith("RuntimeError") for _, _, err in rep.failed)
    assert rep.completed == 32 - 4 - 3 - 2                 # session 4 finished 1 request, session 6 two
    assert be.open_now == 0 and sorted(be.closed) == [0, 1, 3, 4, 5, 6, 7]
    for s in sess:
        if s.sid in (2, 4, 6):
            continue
        assert [k for sid, k, _ in be.log if sid == s.sid] == [0, 1, 2, 3]


def test_a_failed_session_returns_its_memory():
    """With room for one session at a time, a session whose analysis fails and
    one whose first request fails must not hold the budget: the rest run."""
    be = FailingBackend(fail_open=[0], fail_issue=[(1, 0)])
    sess = _sessions(4, 2, 10000.0, 100)
    rep = Server(be, budget_bytes=150, max_inflight=4).run(sess)
    assert sorted((sid, k) for sid, k, _ in rep.failed) == [(0, -1), (1, 0)]
    assert rep.completed == 4
    assert rep.max_bytes <= 150 and be.max_open <= 1


def test_sessions_without_requests_are_done():
    be = FakeBackend()
    sess = _sessions(3, 2, 4000.0, 10)
    sess.append(SessionSpec(99, None, None, 0, [], None, est_bytes=10))
    rep = Server(be, budget_bytes=10 ** 9).run(sess)
    assert rep.completed == 6 and not rep.failed


def test_admission_estimate_bounds_the_device_memory():
    """Sessions are admitted on estimate_bytes(nnz) before their analysis
    exists; the estimate must not fall below the context's device memory,
    which the host-only plan reports exactly, over the serving sizes."""
    import paper_2302_08656_gb300 as K
    from paper_2302_08656_gb300.serve import estimate_bytes
    from kktgen import KKTPattern, make_grid
    for buses in (500, 3000, 25000):
        pat = KKTPattern(make_grid(9, buses, int(1.28 * buses), buses // 5))
        for prec in ("fp32", "fp64"):
            exact = K.plan(pat.rowptr, pat.colidx, precision=prec)["device_bytes"]
            assert exact <= estimate_bytes(pat.nnz, prec), (buses, prec, exact)
