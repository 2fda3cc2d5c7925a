"""Host-side checks of the model-evaluation ABI (no GPU): the library builds
the KKT pattern of a grid on its own (host-only mode), and it must equal the
pattern of the seeded generator bit for bit (integer work); bad inputs are
rejected."""
import ctypes as C

import numpy as np
import pytest

import paper_2302_08656_gb300 as K
from paper_2302_08656_gb300 import _native
from kktgen import KKTPattern, make_grid


@pytest.mark.parametrize("args", [(1, 200, 300, 40), (3, 30, 40, 6), (2, 2000, 2560, 400), (5, 2, 1, 1)])
@pytest.mark.parametrize("flow", [True, False])
def test_model_pattern_equals_generator_pattern(args, flow):
    g = make_grid(*args)
    pat = KKTPattern(g, flow_limits=flow)
    m = K.KKTModel.from_grid(g, flow_limits=flow, host_only=True)
    assert (m.n, m.n_primal, m.nnz) == (pat.n, pat.n_primal, pat.nnz)
    assert np.array_equal(m.rowptr, pat.rowptr)
    assert np.array_equal(m.colidx, pat.colidx)
    m.close()


def test_model_rejects_bad_grids():
    lib = _native.lib()
    f = np.array([0, 1], np.int32)
    t = np.array([1, 2], np.int32)
    r = np.array([0.01, 0.01])
    x = np.array([0.1, 0.1])
    gb = np.array([0], np.int32)
    c2 = np.array([0.05])
    h = C.c_void_p()

    def create(nb, f, t, r, x, gb, flags=3):
        return lib.kkt_model_create(nb, f.size, gb.size, f.ctypes.data, t.ctypes.data, r.ctypes.data,
                                    x.ctypes.data, gb.ctypes.data, c2.ctypes.data, flags, C.byref(h))

    assert create(3, f, t, r, x, gb) == 0
    lib.kkt_model_destroy(h)
    assert create(2, f, t, r, x, gb) == 1                                # bus index out of range
    assert create(3, f, np.array([1, 1], np.int32), r, x, gb) == 1       # line with equal ends
    assert create(3, f, t, np.zeros(2), np.zeros(2), gb) == 1            # zero impedance
    assert create(3, f, t, r, x, np.array([5], np.int32)) == 1           # generator bus out of range
    assert create(3, f, t, r, x, gb, flags=8) == 1                       # unknown flag
