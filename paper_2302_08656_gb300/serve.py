"""Serving loop: KKT solves of many concurrent ACOPF scenario sessions.

Every session is one interior-point run on its own grid: it issues one
refactor + solve request per IPM iteration, and its next request is released
no earlier than the result of the previous one. The server keeps each
session's analysis and factors resident on the device for the whole run
(Alg. 1 applied per session), admits sessions while their device memory fits
an HBM budget (the rest wait in arrival order), and batches continuously:
requests that arrive while others are on the GPU are issued at once on the
next free stream, so work of different sessions overlaps on the device.

The scheduler is plain Python over a backend with five operations (open,
issue, poll, finish, close); GpuBackend drives the library, and the tests
drive the same scheduler with a fake backend on the CPU. A failure is
confined to its session: when the analysis of a session, or the issue, poll
or finish of one of its requests, raises, that session ends (its handle is
closed, its memory returns to the budget, the error is recorded in
Report.failed) and every other session carries on.
"""
from __future__ import annotations

import heapq
import math
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class SessionSpec:
    sid: int
    rowptr: np.ndarray
    colidx: np.ndarray
    n_primal: int
    arrivals: list            # arrival time (s, from the start) of each request
    inputs: object            # inputs(k) -> (values, rhs) for request k
    est_bytes: int = 0        # device memory estimate used for admission


@dataclass
class Report:
    latencies_ms: list = field(default_factory=list)        # every request, arrival to result
    steady_latencies_ms: list = field(default_factory=list) # requests after a session's first
    omegas: list = field(default_factory=list)
    completed: int = 0
    wall_s: float = 0.0
    max_bytes: int = 0
    max_sessions: int = 0
    admission_waits: int = 0
    refined: int = 0
    failed: list = field(default_factory=list)              # (session, request or -1 for analysis, error)

    @property
    def solves_per_s(self):
        return self.completed / self.wall_s if self.wall_s > 0 else 0.0

    def percentile(self, q, steady=False):
        data = self.steady_latencies_ms if steady else self.latencies_ms
        return float(np.percentile(data, q)) if data else float("nan")


def estimate_bytes(nnz: int, precision: str = "fp32") -> int:
    """Upper estimate of a session's device memory from its nonzero count
    (measured: ~100 B per nonzero in FP32, ~125 B in FP64, plus workspace)."""
    return int((130 if precision == "fp32" else 160) * nnz + (8 << 20))


class Server:
    def __init__(self, backend, budget_bytes: int, max_inflight: int = 16, analysis_workers: int = 8,
                 poll_sleep_s: float = 20e-6):
        self.backend = backend
        self.budget = int(budget_bytes)
        self.max_inflight = int(max_inflight)
        self.workers = int(analysis_workers)
        self.poll_sleep_s = poll_sleep_s

    def run(self, sessions, clock=time.perf_counter) -> Report:
        rep = Report()
        sessions = [s for s in sessions if len(s.arrivals) > 0]   # a session without requests is done
        waiting = [(s.arrivals[0], s.sid) for s in sessions]
        heapq.heapify(waiting)
        spec = {s.sid: s for s in sessions}
        used = 0
        opening = {}                 # sid -> future
        active = {}                  # sid -> dict(handle, k, ticket, release, bytes)
        inflight = 0
        remaining = len(sessions)
        pool = ThreadPoolExecutor(max_workers=self.workers)

        def drop(sid, k, err):
            # end a failed session: close it, return its memory, record the error
            nonlocal used, remaining
            st = active.pop(sid)
            try:
                self.backend.close(st["handle"])
            except Exception:
                pass
            used -= st["bytes"]
            remaining -= 1
            rep.failed.append((sid, k, repr(err)))

        t0 = clock()
        try:
            while remaining:
                now = clock() - t0
                progressed = False
                # admission: sessions whose first request has arrived, in arrival order, while memory fits
                while waiting and waiting[0][0] <= now:
                    sid = waiting[0][1]
                    need = spec[sid].est_bytes
                    if used + need > self.budget and (active or opening):
                        rep.admission_waits += 1
                        break
                    heapq.heappop(waiting)
                    used += need
                    opening[sid] = pool.submit(self.backend.open, spec[sid])
                    progressed = True
                for sid in [s for s, f in opening.items() if f.done()]:
                    fut = opening.pop(sid)
                    progressed = True
                    if fut.exception() is not None:
                        used -= spec[sid].est_bytes
                        remaining -= 1
                        rep.failed.append((sid, -1, repr(fut.exception())))
                        continue
                    handle = fut.result()
                    real = self.backend.bytes_of(handle, spec[sid])
                    used += real - spec[sid].est_bytes
                    active[sid] = dict(handle=handle, k=0, ticket=None, release=spec[sid].arrivals[0],
                                       bytes=real)
                    progressed = True
                rep.max_bytes = max(rep.max_bytes, used)
                rep.max_sessions = max(rep.max_sessions, len(active))
                # completions
                for sid, st in list(active.items()):
                    t = st["ticket"]
                    if t is None:
                        continue
                    try:
                        if not self.backend.poll(t):
                            continue
                        omega, refined = self.backend.finish(t)
                    except Exception as e:
                        inflight -= 1
                        drop(sid, st["k"], e)
                        progressed = True
                        continue
                    done_t = clock() - t0
                    lat = 1000.0 * (done_t - st["release"])
                    rep.latencies_ms.append(lat)
                    if st["k"] > 0:
                        rep.steady_latencies_ms.append(lat)
                    rep.omegas.append(omega)
                    rep.completed += 1
                    rep.refined += int(refined)
                    inflight -= 1
                    st["ticket"] = None
                    st["k"] += 1
                    progressed = True
                    s = spec[sid]
                    if st["k"] == len(s.arrivals):
                        self.backend.close(st["handle"])
                        used -= st["bytes"]
                        del active[sid]
                        remaining -= 1
                    else:
                        st["release"] = max(s.arrivals[st["k"]], done_t)
                # issue every released request while the in-flight window has room
                failed_issue = []
                for sid, st in active.items():
                    if inflight >= self.max_inflight:
                        break
                    if st["ticket"] is None and st["release"] <= now:
                        try:
                            st["ticket"] = self.backend.issue(st["handle"], st["k"])
                        except Exception as e:
                            failed_issue.append((sid, st["k"], e))
                            continue
                        inflight += 1
                        progressed = True
                for sid, k, e in failed_issue:
                    drop(sid, k, e)
                    progressed = True
                if not progressed and self.poll_sleep_s:
                    time.sleep(self.poll_sleep_s)
        finally:
            pool.shutdown(wait=True)
        rep.wall_s = clock() - t0
        return rep


class GpuBackend:
    """Drives the library: one context per session, a pool of CUDA streams,
    refactor + asynchronous checked solve per request, FGMRES only when the
    device-side backward error is above tol."""

    def __init__(self, precision: str = "fp32", tol: float = 1e-10, streams: int = 16, keep_results=False,
                 **opts):
        import torch
        self.torch = torch
        self.precision = precision
        self.tol = tol
        self.opts = opts
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.next_stream = 0
        self.keep = keep_results
        self.results = {}

    def open(self, spec: SessionSpec):
        from . import KKTSolver
        torch = self.torch
        s = KKTSolver(spec.rowptr, spec.colidx, spec.n_primal, precision=self.precision, **self.opts)
        n = s.n
        st = self.streams[self.next_stream % len(self.streams)]
        self.next_stream += 1
        return dict(solver=s, spec=spec, stream=st, x=torch.empty(n, dtype=torch.float64, device="cuda"),
                    omega=torch.empty(1, dtype=torch.float64).pin_memory())

    def bytes_of(self, h, spec):
        return int(h["solver"].plan()["device_bytes"])

    def issue(self, h, k):
        torch = self.torch
        vals, rhs = h["spec"].inputs(k)
        s, st = h["solver"], h["stream"]
        s.refactor(vals, stream=st)
        s.solve_checked(rhs, h["x"], h["omega"], stream=st)
        ev = torch.cuda.Event()
        ev.record(st)
        return dict(h=h, k=k, ev=ev, rhs=rhs)

    def poll(self, t):
        return t["ev"].query()

    def finish(self, t):
        h = t["h"]
        omega = float(h["omega"][0])
        refined = False
        if not (omega <= self.tol):
            _, info = h["solver"].refine(t["rhs"], out=h["x"], tol=self.tol, stream=h["stream"],
                                         raise_on_noconv=False)
            omega = info.backward_err
            refined = True
        if self.keep:
            h["stream"].synchronize()
            self.results[(h["spec"].sid, t["k"])] = h["x"].cpu().numpy()
        return omega, refined

    def close(self, h):
        h["stream"].synchronize()
        h["solver"].close()


def poisson_arrivals(rng, rate_per_s: float, counts):
    """Merged Poisson stream of total rate `rate_per_s`, split over sessions with
    `counts[i]` requests each: returns per-session sorted arrival lists."""
    total = int(sum(counts))
    gaps = rng.exponential(1.0 / rate_per_s, size=total)
    times = np.cumsum(gaps)
    owners = np.repeat(np.arange(len(counts)), counts)
    rng.shuffle(owners)
    out = [[] for _ in counts]
    for t, o in zip(times, owners):
        out[o].append(float(t))
    return out


def log_uniform_sizes(rng, count, lo, hi):
    return [int(round(math.exp(x))) for x in rng.uniform(math.log(lo), math.log(hi), size=count)]
