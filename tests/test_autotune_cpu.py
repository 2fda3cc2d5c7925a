"""Host side of the schedule autotuner: cache keys and the reuse of cached
timings (no device work happens on a cache hit)."""
import json

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2302_08656_gb300 import autotune
from kktgen import KKTPattern, make_grid


def test_pattern_key_separates_pattern_precision_and_count():
    a = KKTPattern(make_grid(1, 20, 26, 4))
    b = KKTPattern(make_grid(2, 20, 26, 4))
    k = autotune.pattern_key(a.rowptr, a.colidx, "fp64", 1)
    assert k == autotune.pattern_key(a.rowptr.copy(), a.colidx.copy(), "fp64", 1)
    others = {autotune.pattern_key(b.rowptr, b.colidx, "fp64", 1), autotune.pattern_key(a.rowptr, a.colidx, "fp32", 1),
              autotune.pattern_key(a.rowptr, a.colidx, "fp64", 4)}
    assert k not in others and len(others) == 3


def test_pattern_key_separates_device_and_library_build():
    a = KKTPattern(make_grid(1, 20, 26, 4))
    k = autotune.pattern_key(a.rowptr, a.colidx, "fp64", 1, device="GPU A", build="b1")
    assert k == autotune.pattern_key(a.rowptr, a.colidx, "fp64", 1, device="GPU A", build="b1")
    assert k != autotune.pattern_key(a.rowptr, a.colidx, "fp64", 1, device="GPU B", build="b1")
    assert k != autotune.pattern_key(a.rowptr, a.colidx, "fp64", 1, device="GPU A", build="b2")
    # the defaults: this process's device and the loaded library file
    assert autotune.pattern_key(a.rowptr, a.colidx, "fp64", 1).endswith(
        ":%s:%s" % (autotune.device_name(), autotune.build_id()))


def test_cached_choice_needs_every_requested_pair():
    entry = {"times": {"8/0": 2.0, "8/2432": 1.5, "16/0": 1.2, "16/2432": 1.7}}
    best, times = autotune.cached_choice(entry, (8, 16), (0, 2432))
    assert best == {"max_pivots": 16, "tree_min_fronts": 0} and times["16/0"] == 1.2
    # a subset of the timed pairs: the fastest within the subset
    best, times = autotune.cached_choice(entry, (8,), (0, 2432))
    assert best == {"max_pivots": 8, "tree_min_fronts": 2432} and set(times) == {"8/0", "8/2432"}
    # a pair that was never timed: no reuse
    assert autotune.cached_choice(entry, (8, 24), (0,)) is None
    assert autotune.cached_choice(None, (8,), (0,)) is None
    assert autotune.cached_choice(entry, (), (0,)) is None


def test_tune_returns_a_cache_hit_without_device_work(tmp_path, monkeypatch):
    pat = KKTPattern(make_grid(1, 20, 26, 4))
    key = autotune.pattern_key(pat.rowptr, pat.colidx, "fp32", 2)
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: {"max_pivots": 8, "tree_min_fronts": 0,
                                      "times": {"8/0": 3.0, "16/0": 2.0, "24/0": 2.5}}}))
    monkeypatch.setattr(autotune, "_CACHE_FILE", str(path))
    # vals / rhs are never touched on a hit (None would fail any device work)
    best, times = autotune.tune(pat.rowptr, pat.colidx, pat.n_primal, None, None, precision="fp32", count=2,
                                candidates=(8, 16, 24), tree_candidates=(0,))
    assert best == {"max_pivots": 16, "tree_min_fronts": 0}
    assert times == {"8/0": 3.0, "16/0": 2.0, "24/0": 2.5}
