"""Build and load the native library (libkkt_gb300.so) and declare its C ABI.

The library is compiled in-tree for sm_103a only. Nothing here falls back to
another implementation: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libkkt_gb300.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["analysis.cpp", "tree_plan.cpp", "kernels.cu", "kkt_capi.cu", "noalloc.cu", "tree.cu", "model.cu", "jacobi.cu",
           "ipm.cu", "hykkt.cu", "hykkt_plan.cpp"]
HEADERS = ["analysis.hpp", "kernels.cuh", "tree_plan.hpp", "model.hpp", "hykkt_plan.hpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "kkt.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units in parallel and link the shared library."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


# ------------------------------------------------------------- ABI structs

class IpmOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("mu0", C.c_double), ("kappa_eps", C.c_double),
                ("kappa_mu", C.c_double), ("theta_mu", C.c_double), ("tau_min", C.c_double),
                ("delta_w", C.c_double), ("delta_c", C.c_double), ("push", C.c_double), ("lin_tol", C.c_double),
                ("angle_ref", C.c_int), ("angle_pin", C.c_double)]


class IpmInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("objective", C.c_double), ("err", C.c_double),
                ("mu", C.c_double), ("lin_iters", C.c_int), ("lin_omega_max", C.c_double),
                ("lin_noconv", C.c_int)]


class HykktInfo(C.Structure):
    _fields_ = [("cg_iters", C.c_int), ("status", C.c_int), ("n_perturbed", C.c_int), ("launches", C.c_int),
                ("cg_resid", C.c_double), ("backward_err", C.c_double)]


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("ordering", C.c_int),
        ("user_perm", C.c_void_p),
        ("static_pivot_eps", C.c_double),
        ("ruiz_iters", C.c_int),
        ("restart", C.c_int),
        ("max_cycles", C.c_int),
        ("relax_pivots", C.c_int),
        ("relax_zeros", C.c_double),
        ("max_pivots", C.c_int),
        ("no_graphs", C.c_int),
        ("tree_min_fronts", C.c_int),
        ("spin_limit", C.c_longlong),
        ("precond", C.c_int),
        ("jacobi_sweeps", C.c_int),
    ]


class Info(C.Structure):
    _fields_ = [
        ("n_perturbed", C.c_int),
        ("iters", C.c_int),
        ("backward_err", C.c_double),
        ("rel_resid2", C.c_double),
        ("refactor_count", C.c_int),
        ("status", C.c_int),
        ("launches", C.c_longlong),
        ("batch", C.c_int),
    ]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_longlong), ("ms", C.c_double)]


class PlanInfo(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("nnz", C.c_int64),
        ("nnz_lu", C.c_int64),
        ("stored_factor", C.c_int64),
        ("n_fronts", C.c_int),
        ("n_levels", C.c_int),
        ("max_front", C.c_int),
        ("max_pivots", C.c_int),
        ("flops", C.c_double),
        ("flops_exact", C.c_double),
        ("device_bytes", C.c_int64),
        ("batch", C.c_int),
        ("tree_levels", C.c_int),
        ("tree_units", C.c_int),
        ("tree_bytes", C.c_int64),
        ("tree_nnz_k", C.c_int64),
        ("tree_nnz_lu", C.c_int64),
        ("tree_pivots", C.c_int),
    ]


# every exported symbol and its signature (the C ABI of include/kkt.h)
_P = C.c_void_p
SIGNATURES = {
    "kkt_default_options": (None, [C.POINTER(Options)]),
    "kkt_plan": (C.c_int, [C.c_int32, _P, _P, C.POINTER(Options), C.POINTER(PlanInfo)]),
    "kkt_analyze": (C.c_int, [C.c_int32, C.c_int32, _P, _P, _P, C.POINTER(Options), C.POINTER(_P)]),
    "kkt_analyze_batch": (C.c_int, [C.c_int32, C.c_int32, _P, _P, C.POINTER(Options), C.c_int32, C.POINTER(_P)]),
    "kkt_refactor": (C.c_int, [_P, _P, _P]),
    "kkt_solve": (C.c_int, [_P, _P, _P, _P]),
    "kkt_refine": (C.c_int, [_P, _P, _P, C.c_double, _P, _P]),
    "kkt_step_host": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, _P]),
    "kkt_solve_checked": (C.c_int, [_P, _P, _P, _P, _P]),
    "kkt_refactor_batched": (C.c_int, [_P, _P, C.c_int, _P]),
    "kkt_solve_batched": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "kkt_residual": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_double), _P]),
    "kkt_get_info": (C.c_int, [_P, C.POINTER(Info)]),
    "kkt_get_plan": (C.c_int, [_P, C.POINTER(PlanInfo)]),
    "kkt_set_profiling": (C.c_int, [_P, C.c_int]),
    "kkt_kernel_stats": (C.c_int, [_P, C.POINTER(KernelStat), C.c_int]),
    "kkt_get_perm": (C.c_int, [_P, _P]),
    "kkt_get_scaling": (C.c_int, [_P, _P]),
    "kkt_export_factors": (C.c_int, [_P, C.POINTER(C.c_int64), _P, _P, _P, C.POINTER(C.c_int64), _P, _P, _P]),
    "kkt_debug_stall": (C.c_int, [_P]),
    "kkt_debug_pivot_rcp": (C.c_int, [_P, _P, C.c_int64, C.c_int, _P]),
    "kkt_precondition": (C.c_int, [_P, _P, _P, _P]),
    "kkt_refactor_refine": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, _P]),
    "kkt_model_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P, C.c_int,
                                   C.POINTER(_P)]),
    "kkt_model_pattern": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64), _P, _P]),
    "kkt_model_assemble": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_double, C.c_double, _P, _P]),
    "kkt_model_set_limits": (C.c_int, [_P] + [_P] * 9),
    "kkt_ipm_default_options": (None, [C.POINTER(IpmOptions)]),
    "kkt_ipm_solve": (C.c_int, [_P, _P, C.POINTER(IpmOptions), _P, _P, C.POINTER(IpmInfo), _P]),
    "kkt_model_destroy": (C.c_int, [_P]),
    "kkt_group_create": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "kkt_refactor_group": (C.c_int, [_P, _P, _P]),
    "kkt_group_destroy": (C.c_int, [_P]),
    "kkt_plan_fronts": (C.c_int, [C.c_int32, _P, _P, C.POINTER(Options), C.c_int32, _P, _P,
                                  C.POINTER(C.c_int32)]),
    "kkt_backward_error_noalloc": (C.c_int, [C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "kkt_destroy": (C.c_int, [_P]),
    "kkt_status_string": (C.c_char_p, [C.c_int]),
    "kkt_hykkt_analyze": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_double, C.POINTER(_P)]),
    "kkt_hykkt_solve": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int32, C.POINTER(HykktInfo), _P]),
    "kkt_hykkt_inner": (C.c_int, [_P, C.POINTER(_P)]),
    "kkt_hykkt_destroy": (None, [_P]),
}

_lib = None


def lib():
    """Load libkkt_gb300.so (building it first if sources are newer)."""
    global _lib
    if _lib is None:
        if _stale():
            build()
        if not os.path.exists(LIB):
            raise RuntimeError("libkkt_gb300.so is missing; run paper_2302_08656_gb300.build()")
        L = C.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
