"""ctypes declarations of libpf (the C ABI in include/pf.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpf.so")

PF_OK, PF_EINVAL, PF_ESINGULAR_PATTERN, PF_ENOMEM, PF_ECUDA, PF_ESTATE, PF_ENOTSUP = range(7)
PF_CONVERGED, PF_MAXITER, PF_DIVERGED, PF_SINGULAR = range(4)
PF_FP64, PF_MIXED = 0, 1
PF_NOALLOC_SCRATCH_BYTES = 16 << 20

# every function and its (restype, argtypes); the CPU tests check this list against pf.h
_p = C.c_void_p
_i = C.c_int
_d = C.c_double
_sz = C.c_size_t
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)


class PlanInfo(C.Structure):
    _fields_ = [("n_bus", C.c_int), ("n_slack", C.c_int), ("n_pv", C.c_int), ("n_pq", C.c_int),
                ("n_unknowns", C.c_int), ("n_block", C.c_int), ("nnz_ybus", C.c_int),
                ("nnz_j1", C.c_int), ("nnzb_lu", C.c_int), ("n_levels", C.c_int),
                ("schur_block_ops", C.c_longlong), ("plan_bytes", C.c_longlong),
                ("top_pivots", C.c_int), ("top_levels", C.c_int), ("top_blocks", C.c_int),
                ("top_arena_bytes", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("ir_steps", C.c_int), ("ir_rtol", C.c_double),
                ("group_threads", C.c_int), ("keep_factors", C.c_int), ("placement", C.c_int),
                ("instances_per_cta", C.c_int), ("ir_gate", C.c_double), ("pack", C.c_int),
                ("cluster", C.c_int)]


class PlanOpts(C.Structure):
    _fields_ = [("order_slack", C.c_int), ("top_rows", C.c_int), ("top_blocks", C.c_int),
                ("top_min_pivots", C.c_int), ("split_len", C.c_int), ("split_rows", C.c_int)]


class TuneResult(C.Structure):
    _fields_ = [("group_threads", C.c_int), ("placement", C.c_int),
                ("instances_per_cta", C.c_int), ("ms", C.c_float), ("pack", C.c_int),
                ("cluster", C.c_int)]


(PF_PLACE_AUTO, PF_PLACE_ONCHIP, PF_PLACE_VECTORS, PF_PLACE_GLOBAL, PF_PLACE_FACTOR,
 PF_PLACE_INTERLEAVED) = range(6)
PF_MAX_JOBS = 8


class Job(C.Structure):
    _fields_ = [("h", C.c_void_p), ("batch", C.c_int),
                ("Pd", C.c_void_p), ("Qd", C.c_void_p), ("Pg", C.c_void_p), ("Vset", C.c_void_p),
                ("Vm", C.c_void_p), ("Va", C.c_void_p), ("Pg_out", C.c_void_p), ("Qg_out", C.c_void_p),
                ("iters", C.c_void_p), ("status", C.c_void_p), ("final_mismatch", C.c_void_p)]


SIGNATURES = {
    "pf_build_ybus": (_i, [_i, _i, _ip, _ip, _dp, _dp, _dp, _dp, _ip, _ip, _dp, _dp, _ip]),
    "pf_create": (_i, [_i, _ip, _ip, _dp, _dp, _ip, C.POINTER(_p)]),
    "pf_create_ex": (_i, [_i, _ip, _ip, _dp, _dp, _ip, C.POINTER(PlanOpts), C.POINTER(_p)]),
    "pf_plan_opts_default": (None, [C.POINTER(PlanOpts)]),
    "pf_analyze": (_i, [_i, _ip, _ip, _dp, _dp, _ip, C.POINTER(PlanInfo), _ip, _ip, _ip, _ip,
                        _ip, _ip]),
    "pf_analyze_ex": (_i, [_i, _ip, _ip, _dp, _dp, _ip, C.POINTER(PlanOpts), C.POINTER(PlanInfo),
                           _ip, _ip, _ip, _ip, _ip, _ip]),
    "pf_jacobian_pattern": (_i, [_p, _ip, _ip]),
    "pf_bde_pattern": (_i, [_p, _i, _p, _p, _p]),
    "pf_export_jacobian": (_i, [_p, _i, _p, _p, _p, _p]),
    "pf_get_plan_info": (_i, [_p, C.POINTER(PlanInfo)]),
    "pf_workspace_size": (_i, [_p, _i, C.POINTER(SolveOpts), C.POINTER(_sz)]),
    "pf_solve": (_i, [_p, _i, _p, _p, _p, _p, _d, _i, C.POINTER(SolveOpts),
                      _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "pf_solve_host": (_i, [_p, _i, _p, _p, _p, _p, _d, _i, C.POINTER(SolveOpts),
                           _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "pf_addressable": (_i, [_p, _p, _sz, _ip]),
    "pf_autotune": (_i, [_p, _i, _p, _p, _p, _p, _d, _i, C.POINTER(SolveOpts), _p, _sz, _p,
                         C.POINTER(TuneResult)]),
    "pf_adjoint": (_i, [_p, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "pf_solve_noalloc": (_i, [_p, _i, _p, _p, _p, _p, _d, _i, C.POINTER(SolveOpts),
                              _p, _p, _p, _p, _p, _p, _p, _p]),
    "pf_multi_workspace_size": (_i, [_i, C.POINTER(Job), C.POINTER(SolveOpts), C.POINTER(_sz),
                                     C.POINTER(_sz)]),
    "pf_solve_multi": (_i, [_i, C.POINTER(Job), _d, _i, C.POINTER(SolveOpts), _p, _sz, _p]),
    "pf_autotune_multi": (_i, [_i, C.POINTER(Job), _d, _i, C.POINTER(SolveOpts), _p, _sz, _p,
                               C.POINTER(TuneResult)]),
    "pf_qlim_workspace_size": (_i, [_p, _i, C.POINTER(SolveOpts), C.POINTER(_sz)]),
    "pf_solve_qlim": (_i, [_p, _i, _p, _p, _p, _p, _p, _p, _d, _i, _i, C.POINTER(SolveOpts),
                           _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "pf_adjoint_qlim": (_i, [_p, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _sz,
                             _p]),
    "pf_bde_workspace_size": (_i, [_p, _i, C.POINTER(_sz)]),
    "pf_solve_bde": (_i, [_p, _i, _p, _p, _p, _p, _d, _i, _p, _p, _p, _p, _p, _p, _p, _p, _sz, _p]),
    "pf_measure_fma_peak": (_i, [_i, _i, C.POINTER(_d), _p]),
    "pf_destroy": (None, [_p]),
    "pf_error_string": (C.c_char_p, [_i]),
}

_lib = None


class PFError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (code {code})")


def load() -> C.CDLL:
    """Load libpf.so from the package directory; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpf.so is not built ({LIB_PATH}); run "
                          "`python -m paper_2606_07099_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def error_string(code: int) -> str:
    try:
        return load().pf_error_string(code).decode()
    except Exception:
        return "error"


def check(code: int, where: str) -> None:
    if code != PF_OK:
        raise PFError(code, where)


def measure_fma_peak(fp64: bool, iters: int = 1 << 16, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (pf_measure_fma_peak)."""
    out = C.c_double(0.0)
    check(load().pf_measure_fma_peak(1 if fp64 else 0, int(iters), C.byref(out), stream),
          "pf_measure_fma_peak")
    return out.value
