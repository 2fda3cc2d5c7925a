"""GB300-native refactorization of ACOPF KKT systems (arxiv 2302.08656).

Thin Python binding over the C ABI of ``include/kkt.h``: argument marshalling
only. Device memory and streams come from PyTorch; every step of the path
(equilibration, scatter, multifrontal LU, triangular solves, residual, FGMRES
vector work) runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._native import Info, KernelStat, Options, PlanInfo, build, lib

__all__ = ["KKTSolver", "KKTModel", "KKTGroup", "KKTError", "plan", "plan_fronts", "front_histogram",
           "refactor_batched",
           "solve_batched", "build",
           "FP64", "FP32_IR", "Options", "Info", "PlanInfo"]

FP64, FP32_IR = 0, 1
_ORDER = {"mindeg": 0, "user": 1, "natural": 2}
_STATUS = {0: "KKT_OK", 1: "KKT_E_ARG", 2: "KKT_E_CUDA", 3: "KKT_E_NOMEM", 4: "KKT_E_STATE",
           5: "KKT_E_STRUCT", 6: "KKT_E_NOCONV", 7: "KKT_E_TIMEOUT", 8: "KKT_E_NUMERIC"}


class KKTError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        msg = lib().kkt_status_string(self.status).decode()
        super().__init__("%s: %s (%s)" % (where, _STATUS.get(self.status, "?"), msg))


def _check(st: int, where: str):
    if st != 0:
        raise KKTError(st, where)


def _opts(precision="fp64", ordering="mindeg", user_perm=None, static_pivot_eps=0.0, ruiz_iters=10,
          restart=30, max_cycles=10, relax_pivots=16, relax_zeros=0.15, max_pivots=16, graphs=True,
          tree_min_fronts=None, spin_limit=None, precond="lu", jacobi_sweeps=4):
    o = Options()
    lib().kkt_default_options(C.byref(o))
    if precision in ("fp32", "fp32_ir", FP32_IR):
        o.precision = FP32_IR
    elif precision in ("fp64", FP64):
        o.precision = FP64
    else:
        raise ValueError("precision must be 'fp64' or 'fp32', got %r" % (precision,))
    o.ordering = _ORDER[ordering] if isinstance(ordering, str) else int(ordering)
    keep = None
    if user_perm is not None:
        keep = np.ascontiguousarray(user_perm, dtype=np.int32)
        o.user_perm = keep.ctypes.data
        o.ordering = 1
    o.static_pivot_eps = float(static_pivot_eps)
    o.ruiz_iters = int(ruiz_iters)
    o.restart = int(restart)
    o.max_cycles = int(max_cycles)
    o.relax_pivots = int(relax_pivots)
    o.relax_zeros = float(relax_zeros)
    o.max_pivots = int(max_pivots)
    o.no_graphs = 0 if graphs else 1
    if tree_min_fronts is not None:
        o.tree_min_fronts = int(tree_min_fronts)
    if spin_limit is not None:
        o.spin_limit = int(spin_limit)
    o.precond = {"lu": 0, "jacobi": 1, "block": 2}[precond] if isinstance(precond, str) else int(precond)
    o.jacobi_sweeps = int(jacobi_sweeps)
    return o, keep


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_tensor(t, numel, name, host=False, dtype=None):
    """Raise unless t is a contiguous torch tensor of `dtype` (float64 by
    default) with `numel` elements (None: any number) on a CUDA device
    (host=True: in host memory). Every pointer the library reads or writes is
    checked here first, so a wrong argument never reaches a kernel."""
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor, got %s" % (name, type(t).__name__))
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, str(dtype).replace("torch.", ""), t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if host and t.is_cuda:
        raise ValueError("%s must be in host memory" % name)
    if not host and not t.is_cuda:
        raise ValueError("%s must be on a CUDA device" % name)


def _check_array(a, numel, name, writeable=False):
    """Raise unless a is a contiguous float64 numpy array of `numel` elements."""
    if not isinstance(a, np.ndarray):
        raise TypeError("%s must be a numpy array, got %s" % (name, type(a).__name__))
    if a.dtype != np.float64 or a.size != numel or not a.flags.c_contiguous:
        raise ValueError("%s must be a contiguous float64 array of %d elements, got %s %s"
                         % (name, numel, a.dtype, a.shape))
    if writeable and not a.flags.writeable:
        raise ValueError("%s must be writeable" % name)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _pattern(rowptr, colidx, user_perm=None):
    """int32 copies of a CSR pattern, checked so that the library reads only
    inside them: rowptr one-dimensional, starting at 0, non-decreasing, and
    colidx holding exactly rowptr[-1] entries; a user permutation has one
    entry per row. (Column ranges, order, symmetry and the permutation's
    values are checked by the library.)"""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    if rp.ndim != 1 or ci.ndim != 1 or rp.size < 2:
        raise ValueError("rowptr and colidx must be one-dimensional, rowptr with at least 2 entries")
    if rp[0] != 0 or np.any(np.diff(rp) < 0):
        raise ValueError("rowptr must start at 0 and be non-decreasing")
    if ci.size != int(rp[-1]):
        raise ValueError("colidx must have rowptr[-1] = %d entries, got %d" % (int(rp[-1]), ci.size))
    if user_perm is not None and np.asarray(user_perm).size != rp.size - 1:
        raise ValueError("user_perm must have one entry per row")
    return rp, ci


def plan(rowptr, colidx, **opts) -> dict:
    """Host-only analysis sizes (no GPU needed)."""
    rp, ci = _pattern(rowptr, colidx, opts.get("user_perm"))
    o, keep = _opts(**opts)
    out = PlanInfo()
    _check(lib().kkt_plan(rp.size - 1, rp.ctypes.data, ci.ctypes.data, C.byref(o), C.byref(out)), "kkt_plan")
    return {f: getattr(out, f) for f, _ in PlanInfo._fields_}


def plan_fronts(rowptr, colidx, **opts):
    """Host-only: (front orders F, pivot counts w) of the supernodal fronts the
    analysis builds, in assembly-tree postorder (no GPU needed)."""
    rp, ci = _pattern(rowptr, colidx, opts.get("user_perm"))
    o, keep = _opts(**opts)
    cnt = C.c_int32(0)
    _check(lib().kkt_plan_fronts(rp.size - 1, rp.ctypes.data, ci.ctypes.data, C.byref(o), 0, None, None,
                                 C.byref(cnt)), "kkt_plan_fronts")
    F = np.empty(cnt.value, np.int32)
    w = np.empty(cnt.value, np.int32)
    _check(lib().kkt_plan_fronts(rp.size - 1, rp.ctypes.data, ci.ctypes.data, C.byref(o), cnt.value, F.ctypes.data,
                                 w.ctypes.data, C.byref(cnt)), "kkt_plan_fronts")
    return F, w


def front_histogram(rowptr, colidx, edges=(1, 9, 17, 33, 65, 129, 257, 513), **opts):
    """Dense work of the fronts by front order: per bucket of F the number of
    fronts and their flops (pivot block 2/3 w^3, panels 2 w^2 (F - w), Schur
    update 2 w (F - w)^2), and the Schur-update flops of the fronts with
    F - w >= 64 (those a tensor-core tile could take)."""
    F, w = plan_fronts(rowptr, colidx, **opts)
    F, w = F.astype(np.float64), w.astype(np.float64)
    m = F - w
    piv, pan, schur = 2.0 / 3.0 * w ** 3, 2.0 * w * w * m, 2.0 * w * m * m
    tot = piv + pan + schur
    rows = []
    for a, b in zip(edges[:-1], edges[1:]):
        sel = (F >= a) & (F < b)
        rows.append({"F": [int(a), int(b) - 1], "fronts": int(sel.sum()), "flops": float(tot[sel].sum()),
                     "schur_flops": float(schur[sel].sum())})
    big = m >= 64
    return {"fronts": int(F.size), "max_front": int(F.max()) if F.size else 0, "flops": float(tot.sum()),
            "schur_flops": float(schur.sum()), "buckets": rows,
            "tile_candidates": {"fronts": int(big.sum()), "schur_flops": float(schur[big].sum())}}


class KKTSolver:
    """One analysed KKT pattern with its device-resident factors."""

    def __init__(self, rowptr, colidx, n_primal: int = 0, count: int = 1, **opts):
        """count > 1: a batched context, `count` instances of this pattern
        (arrays are then instance-major: count x nnz values, count x n vectors)."""
        self._rp, self._ci = _pattern(rowptr, colidx, opts.get("user_perm"))
        self.n = self._rp.size - 1
        self.nnz = int(self._rp[-1])
        self.count = int(count)
        o, keep = _opts(**opts)
        self.precision = "fp32" if o.precision == FP32_IR else "fp64"
        h = C.c_void_p()
        if self.count == 1:
            st = lib().kkt_analyze(self.n, int(n_primal), self._rp.ctypes.data, self._ci.ctypes.data, None,
                                   C.byref(o), C.byref(h))
        else:
            st = lib().kkt_analyze_batch(self.n, int(n_primal), self._rp.ctypes.data, self._ci.ctypes.data,
                                         C.byref(o), self.count, C.byref(h))
        _check(st, "kkt_analyze")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kkt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- numeric stages ---------------------------------------------------
    def refactor(self, vals, stream=None):
        _check_tensor(vals, self.nnz * self.count, "vals")
        _check(lib().kkt_refactor(self._h, _ptr(vals), _stream(stream)), "kkt_refactor")

    def refactor_refine(self, vals, rhs, out=None, tol=1e-10, stream=None, raise_on_noconv=True):
        """refactor + refine in one call (the first solve's forward pass rides along the refactorization)."""
        import torch
        _check_tensor(vals, self.nnz * self.count, "vals")
        _check_tensor(rhs, self.n * self.count, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        _check_tensor(out, self.n * self.count, "out")
        infos = (Info * self.count)()
        st = lib().kkt_refactor_refine(self._h, _ptr(vals), _ptr(rhs), _ptr(out), float(tol), infos,
                                       _stream(stream))
        if st != 6 or raise_on_noconv:
            _check(st, "kkt_refactor_refine")
        return out, (infos[0] if self.count == 1 else list(infos))

    def solve(self, rhs, out=None, stream=None):
        import torch
        _check_tensor(rhs, self.n * self.count, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        _check_tensor(out, self.n * self.count, "out")
        _check(lib().kkt_solve(self._h, _ptr(rhs), _ptr(out), _stream(stream)), "kkt_solve")
        return out

    def refine(self, rhs, out=None, tol=1e-10, stream=None, raise_on_noconv=True):
        import torch
        _check_tensor(rhs, self.n * self.count, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        _check_tensor(out, self.n * self.count, "out")
        infos = (Info * self.count)()
        st = lib().kkt_refine(self._h, _ptr(rhs), _ptr(out), float(tol), infos, _stream(stream))
        if st != 6 or raise_on_noconv:
            _check(st, "kkt_refine")
        return out, (infos[0] if self.count == 1 else list(infos))

    def precondition(self, rhs, out=None, stream=None):
        """z = M^{-1} rhs with the context's preconditioner (exact solves, Jacobi or block-Jacobi sweeps)."""
        import torch
        _check_tensor(rhs, self.n * self.count, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        _check_tensor(out, self.n * self.count, "out")
        _check(lib().kkt_precondition(self._h, _ptr(rhs), _ptr(out), _stream(stream)), "kkt_precondition")
        return out

    def solve_checked(self, rhs, out, omega_host, stream=None):
        """Asynchronous solve + device-side backward error into omega_host
        (a pinned float64 tensor with `count` entries, valid after the stream work)."""
        _check_tensor(rhs, self.n * self.count, "rhs")
        _check_tensor(out, self.n * self.count, "out")
        _check_tensor(omega_host, self.count, "omega_host", host=True)
        _check(lib().kkt_solve_checked(self._h, _ptr(rhs), _ptr(out), C.c_void_p(omega_host.data_ptr()),
                                       _stream(stream)), "kkt_solve_checked")

    def step_host(self, vals, rhs, tol=1e-10, out=None, stream=None, raise_on_noconv=True):
        """Refactor + refine through host buffers (copies inside the call)."""
        v = np.ascontiguousarray(vals, dtype=np.float64).reshape(-1)
        b = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
        _check_array(v, self.nnz * self.count, "vals")
        _check_array(b, self.n * self.count, "rhs")
        x = np.empty(self.n * self.count) if out is None else out
        _check_array(x, self.n * self.count, "out", writeable=True)
        infos = (Info * self.count)()
        st = lib().kkt_step_host(self._h, v.ctypes.data, b.ctypes.data, x.ctypes.data, float(tol),
                                 infos, _stream(stream))
        if st != 6 or raise_on_noconv:
            _check(st, "kkt_step_host")
        return x, (infos[0] if self.count == 1 else list(infos))

    def residual(self, rhs, x, out=None, stream=None):
        """r = rhs - K x and the backward error of x, for one system of n rows
        (the first instance of a batched context)."""
        import torch
        _check_tensor(rhs, self.n, "rhs")
        _check_tensor(x, self.n, "x")
        if out is None:
            out = torch.empty_like(rhs)
        _check_tensor(out, self.n, "out")
        om = C.c_double(0.0)
        _check(lib().kkt_residual(self._h, _ptr(rhs), _ptr(x), _ptr(out), C.byref(om), _stream(stream)),
               "kkt_residual")
        return out, om.value

    # -- introspection ----------------------------------------------------
    def info(self) -> Info:
        i = Info()
        _check(lib().kkt_get_info(self._h, C.byref(i)), "kkt_get_info")
        return i

    def plan(self) -> dict:
        p = PlanInfo()
        _check(lib().kkt_get_plan(self._h, C.byref(p)), "kkt_get_plan")
        return {f: getattr(p, f) for f, _ in PlanInfo._fields_}

    def debug_stall(self):
        """Failure injection for tests: the next refactor's bounded device wait
        expires (KKT_E_TIMEOUT from info() / refine()); the context stays usable."""
        _check(lib().kkt_debug_stall(self._h), "kkt_debug_stall")

    def set_profiling(self, on: bool = True):
        _check(lib().kkt_set_profiling(self._h, 1 if on else 0), "kkt_set_profiling")

    def kernel_stats(self) -> dict:
        """{kernel name: (launches, ms)} since the last call (profiling mode)."""
        arr = (KernelStat * 32)()
        k = lib().kkt_kernel_stats(self._h, arr, 32)
        if k < 0:
            raise KKTError(2, "kkt_kernel_stats")
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].ms)) for i in range(k)}

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, dtype=np.int32)
        _check(lib().kkt_get_perm(self._h, p.ctypes.data), "kkt_get_perm")
        return p

    def scaling(self) -> np.ndarray:
        d = np.empty(self.n)
        _check(lib().kkt_get_scaling(self._h, d.ctypes.data), "kkt_get_scaling")
        return d

    def export_factors(self):
        """(L rows, L cols, L vals, U rows, U cols, U vals), original indices."""
        nl, nu = C.c_int64(0), C.c_int64(0)
        _check(lib().kkt_export_factors(self._h, C.byref(nl), None, None, None, C.byref(nu), None, None, None),
               "kkt_export_factors")
        lr, lc, lv = np.empty(nl.value, np.int32), np.empty(nl.value, np.int32), np.empty(nl.value)
        ur, uc, uv = np.empty(nu.value, np.int32), np.empty(nu.value, np.int32), np.empty(nu.value)
        _check(lib().kkt_export_factors(self._h, C.byref(nl), lr.ctypes.data, lc.ctypes.data, lv.ctypes.data,
                                        C.byref(nu), ur.ctypes.data, uc.ctypes.data, uv.ctypes.data),
               "kkt_export_factors")
        return lr, lc, lv, ur, uc, uv


class KKTModel:
    """GPU model evaluation of one grid: the KKT values of an interior-point
    iterate (Hessian of the Lagrangian, constraint Jacobian, barrier and
    regularization diagonals) in the model's own CSR pattern."""

    FLOW_LIMITS, HOST_ONLY = 1, 2

    def __init__(self, n_bus, f, t, r, x, gen_bus, c2, flow_limits=True, host_only=False):
        self._keep = [np.ascontiguousarray(a, dtype=dt) for a, dt in
                      ((f, np.int32), (t, np.int32), (r, np.float64), (x, np.float64), (gen_bus, np.int32),
                       (c2, np.float64))]
        ff, tt, rr, xx, gb, cc = self._keep
        if not ff.ndim == tt.ndim == rr.ndim == xx.ndim == gb.ndim == cc.ndim == 1:
            raise ValueError("grid arrays must be one-dimensional")
        if not ff.size == tt.size == rr.size == xx.size:
            raise ValueError("f, t, r and x must have one entry per branch")
        if gb.size != cc.size:
            raise ValueError("gen_bus and c2 must have one entry per generator")
        flags = (self.FLOW_LIMITS if flow_limits else 0) | (self.HOST_ONLY if host_only else 0)
        h = C.c_void_p()
        _check(lib().kkt_model_create(int(n_bus), ff.size, gb.size, ff.ctypes.data, tt.ctypes.data, rr.ctypes.data,
                                      xx.ctypes.data, gb.ctypes.data, cc.ctypes.data, flags, C.byref(h)),
               "kkt_model_create")
        self._h = h
        self.n_bus = int(n_bus)
        self.n_gen = int(gb.size)
        self.n_branch = int(ff.size)
        n, npr, nnz = C.c_int32(0), C.c_int32(0), C.c_int64(0)
        _check(lib().kkt_model_pattern(h, C.byref(n), C.byref(npr), C.byref(nnz), None, None), "kkt_model_pattern")
        self.n, self.n_primal, self.nnz = n.value, npr.value, nnz.value
        self.rowptr = np.empty(self.n + 1, np.int32)
        self.colidx = np.empty(self.nnz, np.int32)
        _check(lib().kkt_model_pattern(h, C.byref(n), C.byref(npr), C.byref(nnz), self.rowptr.ctypes.data,
                                       self.colidx.ctypes.data), "kkt_model_pattern")

    @classmethod
    def from_grid(cls, grid, flow_limits=True, host_only=False):
        """From any object with n_bus, f, t, r, x, gen_bus, c2 attributes."""
        return cls(grid.n_bus, grid.f, grid.t, grid.r, grid.x, grid.gen_bus, grid.c2, flow_limits, host_only)

    def assemble(self, V, theta, lam, sigma, delta_w=1e-8, delta_c=1e-10, out=None, stream=None, dual_diag=None):
        """K values (device float64, nnz) from device float64 V, theta (n_bus),
        lam (constraint rows) and sigma (n_primal); dual_diag (constraint rows,
        optional) is added to delta_c on the (2,2) diagonal."""
        import torch
        _check_tensor(V, self.n_bus, "V")
        _check_tensor(theta, self.n_bus, "theta")
        _check_tensor(lam, self.n - self.n_primal, "lam")
        _check_tensor(sigma, self.n_primal, "sigma")
        if dual_diag is not None:
            _check_tensor(dual_diag, self.n - self.n_primal, "dual_diag")
        if out is None:
            out = torch.empty(self.nnz, dtype=torch.float64, device=V.device)
        _check_tensor(out, self.nnz, "out")
        _check(lib().kkt_model_assemble(self._h, _ptr(V), _ptr(theta), _ptr(lam), _ptr(sigma),
                                        _ptr(dual_diag) if dual_diag is not None else None, float(delta_w),
                                        float(delta_c), _ptr(out), _stream(stream)), "kkt_model_assemble")
        return out

    def set_limits(self, data):
        """Loads and limits (an object with Pd, Qd, Vmin, Vmax (buses), Pmin,
        Pmax, Qmin, Qmax (generators), Smax (lines)); allocates the
        interior-point loop's workspace."""
        arrs = []
        for name, size in (("Pd", self.n_bus), ("Qd", self.n_bus), ("Vmin", self.n_bus), ("Vmax", self.n_bus),
                           ("Pmin", self.n_gen), ("Pmax", self.n_gen), ("Qmin", self.n_gen), ("Qmax", self.n_gen),
                           ("Smax", self.n_branch)):
            a = np.ascontiguousarray(getattr(data, name), dtype=np.float64).reshape(-1)
            _check_array(a, size, name)
            arrs.append(a)
        self._limits = arrs
        _check(lib().kkt_model_set_limits(self._h, *[a.ctypes.data for a in arrs]), "kkt_model_set_limits")

    def ipm_solve(self, solver, x0, stream=None, **opts):
        """The interior-point loop from the starting point x0 (device float64,
        n_primal; overwritten with the last iterate). Returns (x, lam, info)."""
        import torch
        from ._native import IpmInfo, IpmOptions
        if solver.n != self.n or solver.nnz != self.nnz or solver.count != 1:
            raise ValueError("the solver must be a single-instance context of the model's pattern")
        _check_tensor(x0, self.n_primal, "x0")
        o = IpmOptions()
        lib().kkt_ipm_default_options(C.byref(o))
        for k, v in opts.items():
            if not hasattr(o, k):
                raise ValueError("unknown interior-point option %r" % k)
            setattr(o, k, type(getattr(o, k))(v))
        lam = torch.empty(self.n - self.n_primal, dtype=torch.float64, device=x0.device)
        info = IpmInfo()
        st = lib().kkt_ipm_solve(self._h, solver.handle, C.byref(o), _ptr(x0), _ptr(lam), C.byref(info),
                                 _stream(stream))
        if st not in (0, 6):
            _check(st, "kkt_ipm_solve")
        return x0, lam, info

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kkt_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def backward_error_noalloc(rowptr, colidx, vals, x, rhs, r, omega, stream=None):
    """r = b - K x and omega into caller-provided device tensors, allocating
    nothing (rowptr / colidx int32 and vals float64, all seven tensors on one
    CUDA device; the call is made with that device current). The library
    checks the pattern as it reads it: rows out of range or column indices
    outside [0, n) give NaN in r and omega, never a read outside the arrays."""
    import torch
    _check_tensor(rowptr, None, "rowptr", dtype=torch.int32)
    n = rowptr.numel() - 1
    if n < 1:
        raise ValueError("rowptr must have at least 2 entries")
    _check_tensor(colidx, None, "colidx", dtype=torch.int32)
    _check_tensor(vals, colidx.numel(), "vals")
    for t, name in ((x, "x"), (rhs, "rhs"), (r, "r")):
        _check_tensor(t, n, name)
    _check_tensor(omega, 1, "omega")
    dev = rowptr.device
    for t, name in ((colidx, "colidx"), (vals, "vals"), (x, "x"), (rhs, "rhs"), (r, "r"), (omega, "omega")):
        if t.device != dev:
            raise ValueError("%s is on %s, rowptr on %s: all tensors must be on one device" % (name, t.device, dev))
    with torch.cuda.device(dev):
        _check(lib().kkt_backward_error_noalloc(n, colidx.numel(), _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(x),
                                                _ptr(rhs), _ptr(r), _ptr(omega), _stream(stream)),
               "kkt_backward_error_noalloc")


def debug_pivot_rcp(d, out=None, stream=None):
    """The pivot reciprocal the factorization and backward kernels use for
    1 / d, elementwise over a float64 or float32 device tensor."""
    import torch
    if not isinstance(d, torch.Tensor) or d.dtype not in (torch.float64, torch.float32):
        raise ValueError("d must be a float64 or float32 tensor")
    _check_tensor(d, d.numel(), "d", dtype=d.dtype)
    out = torch.empty_like(d) if out is None else out
    _check_tensor(out, d.numel(), "out", dtype=d.dtype)
    prec = 0 if d.dtype == torch.float64 else 1
    _check(lib().kkt_debug_pivot_rcp(_ptr(d), _ptr(out), d.numel(), prec, _stream(stream)), "kkt_debug_pivot_rcp")
    return out


def _ptr_array(items):
    arr = (C.c_void_p * len(items))(*[C.c_void_p(x) for x in items])
    return arr


def refactor_batched(solvers, vals, stream=None):
    if len(vals) != len(solvers):
        raise ValueError("one vals tensor per solver")
    for i, (s, v) in enumerate(zip(solvers, vals)):
        _check_tensor(v, s.nnz * s.count, "vals[%d]" % i)
    hs = _ptr_array([s.handle.value for s in solvers])
    vs = _ptr_array([v.data_ptr() for v in vals])
    _check(lib().kkt_refactor_batched(hs, vs, len(solvers), _stream(stream)), "kkt_refactor_batched")


class KKTGroup:
    """Solvers (patterns of any size, each possibly batched, one precision)
    refactored together: level parts concurrently, the tops of all their
    assembly trees in one launch."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        if not self.solvers:
            raise ValueError("a group needs at least one solver")
        if len({id(s) for s in self.solvers}) != len(self.solvers):
            raise ValueError("a solver appears twice in the group")
        if len({s.precision for s in self.solvers}) != 1:
            raise ValueError("the solvers of a group share one precision")
        hs = _ptr_array([s.handle.value for s in self.solvers])
        h = C.c_void_p()
        _check(lib().kkt_group_create(hs, len(self.solvers), C.byref(h)), "kkt_group_create")
        self._h = h

    def refactor(self, vals, stream=None):
        if len(vals) != len(self.solvers):
            raise ValueError("one vals tensor per solver")
        for i, (s, v) in enumerate(zip(self.solvers, vals)):
            _check_tensor(v, s.nnz * s.count, "vals[%d]" % i)
        vs = _ptr_array([v.data_ptr() for v in vals])
        _check(lib().kkt_refactor_group(self._h, vs, _stream(stream)), "kkt_refactor_group")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kkt_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BorrowedContext:
    """A context owned by another object: introspection only, never destroyed here."""

    def __init__(self, handle, owner):
        self._h = handle
        self._owner = owner          # keeps the owner (and so the context) alive

    info = KKTSolver.info
    plan = KKTSolver.plan
    set_profiling = KKTSolver.set_profiling
    kernel_stats = KKTSolver.kernel_stats


class SaddlePointSolver:
    """Saddle-point specialised solve of K (kkt_hykkt_*; Sec. V): inequality
    rows condensed, equality rows augmented by gamma J_E^T J_E, conjugate
    gradients on the reduced symmetric operator, one factorization of H_g by
    the library per call. Unknowns ordered (primal, m_eq equality duals,
    inequality duals); the (2,2) block diagonal. gamma must keep
    gamma * d_E < 1; the default suits the literal regularization (d_E =
    1e-10): larger gamma, fewer iterations (8 to 12 at 1e8 on the 25,000- and
    70,000-bus systems) at an unchanged backward error."""

    def __init__(self, rowptr, colidx, n_primal, m_eq, gamma=1e8):
        rp, ci = _pattern(rowptr, colidx)
        self.n = len(rp) - 1
        self.nnz = int(rp[-1])
        if not (0 < int(n_primal) and 0 < int(m_eq) and int(n_primal) + int(m_eq) <= self.n):
            raise ValueError("need 0 < n_primal, 0 < m_eq, n_primal + m_eq <= n")
        if not (gamma >= 0 and np.isfinite(gamma)):
            raise ValueError("gamma must be finite and >= 0")
        h = C.c_void_p()
        _check(lib().kkt_hykkt_analyze(self.n, int(n_primal), int(m_eq), rp.ctypes.data, ci.ctypes.data,
                                       float(gamma), C.byref(h)), "kkt_hykkt_analyze")
        self._h = h
        self.n_primal, self.m_eq, self.gamma = int(n_primal), int(m_eq), float(gamma)

    def solve(self, vals, rhs, tol=1e-12, max_iter=500, out=None, stream=None, raise_on_noconv=True):
        import torch
        _check_tensor(vals, self.nnz, "vals")
        _check_tensor(rhs, self.n, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        _check_tensor(out, self.n, "out")
        if not (vals.device == rhs.device == out.device):
            raise ValueError("vals, rhs and out must be on one device")
        if out.data_ptr() == rhs.data_ptr():
            raise ValueError("out must not be rhs")
        from ._native import HykktInfo
        info = HykktInfo()
        with torch.cuda.device(rhs.device):
            st = lib().kkt_hykkt_solve(self._h, _ptr(vals), _ptr(rhs), _ptr(out), float(tol), int(max_iter),
                                       C.byref(info), _stream(stream))
        if st != 6 or raise_on_noconv:
            _check(st, "kkt_hykkt_solve")
        return out, info

    def inner(self):
        """The context factoring H_g (borrowed, valid while this solver is
        open): plan(), info(), set_profiling(), kernel_stats()."""
        h = C.c_void_p()
        _check(lib().kkt_hykkt_inner(self._h, C.byref(h)), "kkt_hykkt_inner")
        return _BorrowedContext(h, self)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kkt_hykkt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(solvers, rhs, outs, stream=None):
    if not len(rhs) == len(outs) == len(solvers):
        raise ValueError("one rhs and one out tensor per solver")
    for i, (s, b, x) in enumerate(zip(solvers, rhs, outs)):
        _check_tensor(b, s.n * s.count, "rhs[%d]" % i)
        _check_tensor(x, s.n * s.count, "outs[%d]" % i)
    hs = _ptr_array([s.handle.value for s in solvers])
    bs = _ptr_array([b.data_ptr() for b in rhs])
    xs = _ptr_array([x.data_ptr() for x in outs])
    _check(lib().kkt_solve_batched(hs, bs, xs, len(solvers), _stream(stream)), "kkt_solve_batched")
