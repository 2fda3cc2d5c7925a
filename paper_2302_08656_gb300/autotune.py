"""Per-pattern schedule autotuner.

The schedule depends on how many pivots a supernode may hold (few pivots:
short sequential pivot blocks but a taller assembly tree; many: the
opposite) and on how much of the narrow top of the tree the persistent tree
kernels take (tree_min_fronts). Which wins depends on the size of the
system, the precision (FP64 runs on the slow FP64 pipe) and the batch size.
The tuner times a short refactor + refine sequence (the fused call of an
interior-point iteration) for each candidate on the device and keeps the
fastest, cached per (pattern hash, precision, instance count).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

CANDIDATES = (8, 16, 24, 32)
TREE_CANDIDATES = (0, 2432, 9728)
_CACHE_FILE = os.environ.get("KKT_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                                "kkt_gb300_autotune.json"))


_BUILD_ID = None


def build_id() -> str:
    """Hash of the loaded library file: timings taken with other kernels are
    not reused."""
    global _BUILD_ID
    if _BUILD_ID is None:
        from ._native import LIB
        h = hashlib.sha1()
        try:
            with open(LIB, "rb") as f:
                for chunk in iter(lambda: f.read(1 << 20), b""):
                    h.update(chunk)
            _BUILD_ID = h.hexdigest()[:16]
        except OSError:
            _BUILD_ID = "unbuilt"
    return _BUILD_ID


def device_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except Exception:
        pass
    return "no-device"


def pattern_key(rowptr, colidx, precision: str, count: int, device: str | None = None,
                build: str | None = None) -> str:
    """Cache key: the pattern, precision and instance count, plus the device
    the times were taken on and the library build that was timed."""
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(rowptr, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(colidx, dtype=np.int32).tobytes())
    dev = device_name() if device is None else device
    bid = build_id() if build is None else build
    return "%s:%s:%d:%s:%s" % (h.hexdigest(), precision, int(count), dev, bid)


def _load_cache():
    try:
        with open(_CACHE_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(cache):
    try:
        os.makedirs(os.path.dirname(_CACHE_FILE), exist_ok=True)
        tmp = _CACHE_FILE + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, _CACHE_FILE)
    except Exception:
        pass


def cached_choice(entry, candidates=CANDIDATES, tree_candidates=TREE_CANDIDATES):
    """The fastest requested (max_pivots, tree_min_fronts) pair by the times of
    a cache entry, or None unless the entry timed every requested pair."""
    times = (entry or {}).get("times", {})
    want = ["%d/%d" % (mp, tmf) for mp in candidates for tmf in tree_candidates]
    if not want or any(k not in times for k in want):
        return None
    sub = {k: times[k] for k in want}
    mp, tmf = (int(x) for x in min(sub, key=sub.get).split("/"))
    return {"max_pivots": mp, "tree_min_fronts": tmf}, sub


def tune(rowptr, colidx, n_primal, vals, rhs, precision="fp64", count=1, candidates=CANDIDATES,
         tree_candidates=TREE_CANDIDATES, reps=3, use_cache=True):
    """Return (best options dict, {"max_pivots/tree_min_fronts": ms per refactor+refine}).

    vals / rhs: device tensors for `count` instances (instance-major)."""
    import torch

    from . import KKTSolver

    key = pattern_key(rowptr, colidx, precision, count)
    cache = _load_cache() if use_cache else {}
    hit = cached_choice(cache.get(key), candidates, tree_candidates)
    if hit is not None:
        return hit
    times = {}
    out = torch.empty_like(rhs)
    for mp in candidates:
        for tmf in tree_candidates:
            s = KKTSolver(rowptr, colidx, n_primal, count=count, precision=precision, max_pivots=mp,
                          tree_min_fronts=tmf)
            s.refactor_refine(vals, rhs, out=out, raise_on_noconv=False)     # captures the graphs
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for _ in range(reps):
                s.refactor_refine(vals, rhs, out=out, raise_on_noconv=False)
            ev1.record()
            torch.cuda.synchronize()
            times["%d/%d" % (mp, tmf)] = ev0.elapsed_time(ev1) / reps
            s.close()
    best = min(times, key=times.get)
    mp, tmf = (int(x) for x in best.split("/"))
    if use_cache:
        merged = dict(cache.get(key, {}).get("times", {}))      # keep pairs timed by earlier calls
        merged.update(times)
        cache[key] = {"max_pivots": mp, "tree_min_fronts": tmf, "times": merged}
        _store_cache(cache)
    return {"max_pivots": mp, "tree_min_fronts": tmf}, times
