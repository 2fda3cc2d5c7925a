"""The pivot reciprocal that every factorization and back-substitution kernel
uses for 1 / u_pp (Newton-Raphson from the hardware approximation), against
the correctly rounded IEEE 1 / d: within one unit in the last place over a
log-uniform sweep of magnitudes and both signs inside the stated range, and
the IEEE division itself outside it (zeros, infinities, NaN, subnormals and
the magnitudes beyond the range ends)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2302_08656_gb300 as K

# (dtype, lowest and highest binary exponent served by the Newton step)
RANGES = [(np.float64, -1000, 1000), (np.float32, -100, 100)]


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _gpu_rcp(d):
    t = torch.from_numpy(d).to(_dev())
    out = K.debug_pivot_rcp(t)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dt,lo,hi", RANGES)
def test_pivot_reciprocal_within_one_ulp(dt, lo, hi):
    rng = np.random.default_rng(11)
    n = 1 << 22
    e = rng.integers(lo, hi + 1, n)
    m = rng.uniform(1.0, 2.0, n)
    d = (np.where(rng.random(n) < 0.5, -1.0, 1.0) * np.ldexp(m, e)).astype(dt)
    ad = np.abs(d)
    d = d[(ad >= np.ldexp(dt(1), lo)) & (ad < np.ldexp(dt(1), hi + 1))]
    ref = (dt(1) / d).astype(dt)
    got = _gpu_rcp(d)
    assert got.dtype == dt and np.all(np.isfinite(got))
    ulp = np.abs(got.astype(np.float64) - ref.astype(np.float64)) / np.spacing(np.abs(ref)).astype(np.float64)
    assert ulp.max() <= 1.0, (d[np.argmax(ulp)], got[np.argmax(ulp)], ref[np.argmax(ulp)])
    assert np.mean(got == ref) >= 0.99                     # almost always the correctly rounded value
    assert np.all(np.signbit(got) == np.signbit(d))


@pytest.mark.parametrize("dt,lo,hi", RANGES)
def test_pivot_reciprocal_is_the_ieee_division_outside_the_range(dt, lo, hi):
    fi = np.finfo(dt)
    one = dt(1)
    edge = [np.ldexp(one, lo - 1), np.nextafter(np.ldexp(one, lo), dt(0)), np.ldexp(one, hi + 1),
            np.ldexp(dt(1.5), hi + 2), fi.max, fi.tiny, fi.smallest_subnormal, dt(3) * fi.smallest_subnormal]
    vals = np.array(edge + [-v for v in edge] + [dt(0), -dt(0), dt(np.inf), -dt(np.inf), dt(np.nan)], dtype=dt)
    with np.errstate(divide="ignore", over="ignore"):
        ref = (one / vals).astype(dt)
    got = _gpu_rcp(vals)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])
    assert np.array_equal(np.signbit(got[~nan]), np.signbit(ref[~nan]))   # 1 / -0 = -inf


def test_pivot_reciprocal_argument_errors():
    dev = _dev()
    t = torch.ones(4, dtype=torch.float64, device=dev)
    lib = K.lib()
    assert lib.kkt_debug_pivot_rcp(None, None, 0, 0, None) == 0          # nothing to do
    assert lib.kkt_debug_pivot_rcp(t.data_ptr(), t.data_ptr(), -1, 0, None) != 0
    assert lib.kkt_debug_pivot_rcp(t.data_ptr(), None, 4, 0, None) != 0
    assert lib.kkt_debug_pivot_rcp(t.data_ptr(), t.data_ptr(), 4, 7, None) != 0
    # in place
    t.fill_(4.0)
    K.debug_pivot_rcp(t, out=t)
    torch.cuda.synchronize()
    assert torch.all(t == 0.25)
