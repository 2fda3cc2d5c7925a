"""Argument checks of the Python binding, run without a GPU: every tensor or
array the library would read or write is checked (type, float64, size,
contiguity, device) before any call reaches it, so a wrong argument raises
instead of reaching a kernel or a host copy."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2302_08656_gb300 as K


def _solver(n=10, nnz=28, count=2):
    s = object.__new__(K.KKTSolver)          # no analysis: the checks come first
    s.n, s.nnz, s.count, s._h = n, nnz, count, None
    return s


@pytest.mark.parametrize("call", ["refactor", "solve", "refine", "precondition", "refactor_refine"])
def test_device_arguments_are_checked(call):
    s = _solver()
    good_v, good_b = torch.zeros(56, dtype=torch.float64), torch.zeros(20, dtype=torch.float64)
    cases = {
        "float32": (torch.zeros(56, dtype=torch.float32), torch.zeros(20, dtype=torch.float32), "float64"),
        "int64": (torch.zeros(56, dtype=torch.int64), torch.zeros(20, dtype=torch.int64), "float64"),
        "size": (torch.zeros(55, dtype=torch.float64), torch.zeros(19, dtype=torch.float64), "elements"),
        "strided": (torch.zeros(112, dtype=torch.float64)[::2], torch.zeros(40, dtype=torch.float64)[::2],
                    "contiguous"),
        "host": (good_v, good_b, "CUDA device"),
    }
    for _, (v, b, msg) in cases.items():
        with pytest.raises(ValueError, match=msg):
            if call == "refactor":
                s.refactor(v)
            elif call == "refactor_refine":
                s.refactor_refine(v, good_b if msg == "CUDA device" else b)
            else:
                getattr(s, call)(b)
    with pytest.raises(TypeError):
        s.refactor(np.zeros(56))


def test_residual_and_checked_solve_arguments():
    s = _solver(count=1)
    b = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError, match="elements"):
        s.residual(torch.zeros(9, dtype=torch.float64), b)
    with pytest.raises(ValueError, match="CUDA device"):
        s.residual(b, b)
    with pytest.raises(ValueError, match="CUDA device"):
        s.solve_checked(b, b, torch.zeros(1, dtype=torch.float64))


def test_host_step_arguments_are_checked():
    s = _solver()
    v, b = np.zeros(56), np.zeros(20)
    with pytest.raises(ValueError, match="vals"):
        s.step_host(np.zeros(55), b)
    with pytest.raises(ValueError, match="rhs"):
        s.step_host(v, np.zeros(21))
    with pytest.raises(ValueError, match="out"):
        s.step_host(v, b, out=np.zeros(20, dtype=np.float32))
    with pytest.raises(ValueError, match="out"):
        s.step_host(v, b, out=np.zeros(40)[::2])
    ro = np.zeros(20)
    ro.flags.writeable = False
    with pytest.raises(ValueError, match="writeable"):
        s.step_host(v, b, out=ro)
    with pytest.raises(TypeError):
        s.step_host(v, b, out=[0.0] * 20)


def test_model_assemble_arguments_are_checked():
    from kktgen import make_grid
    g = make_grid(1, 20, 26, 4)
    m = K.KKTModel.from_grid(g, host_only=True)
    f64 = lambda k: torch.zeros(k, dtype=torch.float64)      # noqa: E731
    V, th, lam, sig = f64(m.n_bus), f64(m.n_bus), f64(m.n - m.n_primal), f64(m.n_primal)
    # arguments are checked in order, each completely (device last)
    with pytest.raises(ValueError, match="V must have"):
        m.assemble(f64(m.n_bus + 1), th, lam, sig)
    with pytest.raises(ValueError, match="V must be float64"):
        m.assemble(torch.zeros(m.n_bus, dtype=torch.float32), th, lam, sig)
    with pytest.raises(ValueError, match="V must be on a CUDA device"):
        m.assemble(V, th, lam, sig)
    m.close()


def test_batched_calls_check_every_solver_argument():
    a, b = _solver(count=2), _solver(n=12, nnz=34, count=1)
    f64 = lambda k: torch.zeros(k, dtype=torch.float64)      # noqa: E731
    with pytest.raises(ValueError, match="one vals"):
        K.refactor_batched([a, b], [f64(56)])
    with pytest.raises(ValueError, match=r"vals\[0\] must have 56"):
        K.refactor_batched([a, b], [f64(55), f64(34)])
    with pytest.raises(ValueError, match=r"vals\[0\] must be on a CUDA device"):
        K.refactor_batched([a, b], [f64(56), f64(34)])
    with pytest.raises(ValueError, match=r"rhs\[0\] must have 20"):
        K.solve_batched([a, b], [f64(19), f64(12)], [f64(20), f64(12)])
    with pytest.raises(ValueError, match="one rhs"):
        K.solve_batched([a, b], [f64(20)], [f64(20), f64(12)])


def test_model_grid_arrays_must_agree_in_length():
    from kktgen import make_grid
    g = make_grid(1, 20, 26, 4)
    with pytest.raises(ValueError, match="per branch"):
        K.KKTModel(g.n_bus, g.f, g.t[:-1], g.r, g.x, g.gen_bus, g.c2, host_only=True)
    with pytest.raises(ValueError, match="per branch"):
        K.KKTModel(g.n_bus, g.f, g.t, g.r, g.x[:-2], g.gen_bus, g.c2, host_only=True)
    with pytest.raises(ValueError, match="per generator"):
        K.KKTModel(g.n_bus, g.f, g.t, g.r, g.x, g.gen_bus, g.c2[:-1], host_only=True)
    K.KKTModel(g.n_bus, g.f, g.t, g.r, g.x, g.gen_bus, g.c2, host_only=True).close()


def test_pattern_arrays_are_checked_before_the_library_reads_them():
    from kktgen import KKTPattern, make_grid
    pat = KKTPattern(make_grid(1, 10, 12, 2))
    rp, ci = pat.rowptr, pat.colidx
    with pytest.raises(ValueError, match="rowptr"):
        K.plan(rp[1:], ci)                                   # does not start at 0
    with pytest.raises(ValueError, match="colidx must have"):
        K.plan(rp, ci[:-1])                                  # shorter than rowptr[-1]
    bad = rp.copy()
    bad[3], bad[4] = bad[4], bad[3]
    with pytest.raises(ValueError, match="non-decreasing"):
        K.plan(bad, ci)
    with pytest.raises(ValueError, match="one-dimensional"):
        K.plan(rp.reshape(1, -1), ci)
    with pytest.raises(ValueError, match="user_perm"):
        K.plan(rp, ci, user_perm=np.arange(pat.n - 1))
    with pytest.raises(ValueError, match="colidx must have"):
        K.KKTSolver(rp, ci[:-1])                             # before any device work
    assert K.plan(rp, ci)["n"] == pat.n


def test_allocation_free_backward_error_arguments():
    i32 = lambda k: torch.zeros(k, dtype=torch.int32)        # noqa: E731
    f64 = lambda k: torch.zeros(k, dtype=torch.float64)      # noqa: E731
    rp, ci = i32(11), i32(30)
    with pytest.raises(ValueError, match="rowptr must be int32"):
        K.backward_error_noalloc(torch.zeros(11, dtype=torch.int64), ci, f64(30), f64(10), f64(10), f64(10), f64(1))
    with pytest.raises(ValueError, match="rowptr must be on a CUDA device"):
        K.backward_error_noalloc(rp, ci, f64(30), f64(10), f64(10), f64(10), f64(1))


def test_pivot_reciprocal_hook_arguments():
    with pytest.raises(ValueError, match="float64 or float32"):
        K.debug_pivot_rcp(torch.zeros(4, dtype=torch.float16))
    with pytest.raises(ValueError, match="contiguous"):
        K.debug_pivot_rcp(torch.zeros(8, dtype=torch.float64)[::2])
    with pytest.raises(ValueError, match="CUDA device"):
        K.debug_pivot_rcp(torch.zeros(4, dtype=torch.float32))
