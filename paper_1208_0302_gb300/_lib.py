"""ctypes binding of libgenesis.so (include/genesis.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

ME_OK = 0
ME_EINVAL = -1
ME_ENOMEM = -2
ME_ECUDA = -3
ME_EAGAIN = -4
ME_EPENDING = -5
ME_ETIMEOUT = -6
ME_ENOTFOUND = -7

ME_NPAR = 9
ME_NPAR_MAX = 10
ME_MAX_LINES = 4
ME_MAX_LAMBDA = 512
ME_F32 = 0
ME_F64 = 1
ME_W_INVMAX = 0
ME_W_USER = 1


ME_MAX_COMP = 9


class MeLine(C.Structure):
    _fields_ = [("lambda0_A", C.c_double), ("g_eff", C.c_double), ("eta_ratio", C.c_double),
                ("pattern", C.c_int), ("j_lower", C.c_int), ("j_upper", C.c_int),
                ("g_lower", C.c_double), ("g_upper", C.c_double)]


class MeProblem(C.Structure):
    _fields_ = [("n_lines", C.c_int), ("line", MeLine * ME_MAX_LINES), ("n_lambda", C.c_int),
                ("lambda_A", C.POINTER(C.c_double)), ("lambda_dop_A", C.c_double),
                ("mu", C.c_double), ("dtype", C.c_int), ("fill_fraction", C.c_int)]


class MeBounds(C.Structure):
    _fields_ = [("lo", C.c_double * ME_NPAR_MAX), ("hi", C.c_double * ME_NPAR_MAX)]


class GaConfig(C.Structure):
    _fields_ = [("npop", C.c_int), ("ngen", C.c_int), ("nsamp", C.c_int), ("pc", C.c_double),
                ("pmut_lsb", C.c_double), ("pmut_ratio", C.c_double), ("seed", C.c_uint64),
                ("weight_mode", C.c_int)]


class ServeConfig(C.Structure):
    _fields_ = [("arena_bytes", C.c_size_t), ("max_inflight", C.c_int), ("max_queue", C.c_int),
                ("small_pixels", C.c_int), ("fail_next_admissions", C.c_int)]


class ServeRequest(C.Structure):
    _fields_ = [("obs", C.c_void_p), ("w", C.c_void_p), ("mu_px", C.c_void_p), ("npix", C.c_int),
                ("pixel_id0", C.c_uint64), ("ga", GaConfig), ("bounds", MeBounds),
                ("polish_iters", C.c_int), ("lambda0", C.c_double), ("polish_w", C.c_void_p)]


class ServeResult(C.Structure):
    _fields_ = [("best", C.c_void_p), ("chi2", C.c_void_p), ("status", C.c_int),
                ("queue_ns", C.c_uint64), ("latency_ns", C.c_uint64)]


class ServeStats(C.Structure):
    _fields_ = [("queued", C.c_int), ("running", C.c_int), ("arena_used", C.c_size_t),
                ("arena_bytes", C.c_size_t)]


class GenesisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"genesis error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_VP = C.c_void_p
_P = C.POINTER(MeProblem)

_SIGNATURES = {
    "me_last_error": ([], C.c_char_p),
    "me_zeeman_components": ([C.POINTER(MeLine), _VP, _VP, _VP], C.c_int),
    "me_version": ([], C.c_int),
    "me_synth": ([_P, _VP, _VP, C.c_int, _VP, _VP], C.c_int),
    "me_synth_jac": ([_P, _VP, _VP, C.c_int, _VP, _VP, _VP], C.c_int),
    "me_synth_vjp": ([_P, _VP, _VP, C.c_int, _VP, _VP, _VP], C.c_int),
    "me_chi2": ([_P, _VP, _VP, _VP, C.c_int, _VP, _VP, _VP], C.c_int),
    "ga_invert_batch": ([_P, _VP, _VP, _VP, C.c_int, C.c_uint64, C.POINTER(MeBounds),
                         C.POINTER(GaConfig), _VP, _VP, _VP, _VP], C.c_int),
    "ga_count_evaluations": ([_P, _VP, _VP, _VP, C.c_int, C.c_uint64, C.POINTER(MeBounds),
                              C.POINTER(GaConfig), _VP, _VP, _VP], C.c_int),
    "ga_fitness": ([_P, _VP, _VP, _VP, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, _VP], C.c_int),
    "me_faddeeva_pairs": ([_VP, _VP, _VP, C.c_int, C.c_int, _VP, _VP], C.c_int),
    "me_fp32_peak": ([C.c_int, C.c_int, C.c_int, _VP, _VP, _VP], C.c_int),
    "lm_polish": ([_P, _VP, _VP, _VP, C.c_int, C.POINTER(MeBounds), C.c_int, C.c_double, _VP,
                   _VP, _VP], C.c_int),
    "lm_uncertainty": ([_P, _VP, _VP, _VP, C.c_int, _VP, _VP, _VP], C.c_int),
    "me_line_centre": ([_P, _VP, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP, _VP], C.c_int),
    "me_classify": ([_P, _VP, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _VP, _VP,
                     _VP, _VP, _VP, _VP, _VP], C.c_int),
    "me_select_scratch_bytes": ([C.c_int], C.c_size_t),
    "me_select": ([_VP, C.c_int, C.c_int, _VP, _VP, _VP, C.c_size_t, _VP], C.c_int),
    "me_select_static": ([_VP, C.c_int, C.c_int, _VP, _VP, _VP], C.c_int),
    "ga_invert_subset": ([_P, _VP, _VP, _VP, C.c_int, C.c_uint64, C.POINTER(MeBounds), C.POINTER(GaConfig),
                          _VP, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], C.c_int),
    "lm_fit": ([_P, _VP, _VP, _VP, C.c_int, C.POINTER(MeBounds), C.c_int, C.c_double, C.c_uint, _VP, _VP,
                _VP, _VP, _VP], C.c_int),
    "me_prefit_bounds": ([_VP, C.c_int, C.c_int, C.POINTER(MeBounds), _VP, _VP, _VP, _VP], C.c_int),
    "ga_breed": ([_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.POINTER(GaConfig), _VP,
                  _VP, _VP], C.c_int),
    "ga_restart": ([_VP, _VP, C.c_int, C.c_int, C.c_int, C.c_uint64, _VP], C.c_int),
    "serve_create": ([_P, C.POINTER(ServeConfig), C.POINTER(C.c_void_p)], C.c_int),
    "serve_submit": ([_VP, C.POINTER(ServeRequest), C.POINTER(C.c_uint64)], C.c_int),
    "serve_poll": ([_VP, C.c_uint64, C.POINTER(ServeResult), C.c_int], C.c_int),
    "serve_stats": ([_VP, C.POINTER(ServeStats)], C.c_int),
    "serve_destroy": ([_VP], C.c_int),
    "me_philox": ([_VP, C.c_int, C.c_uint64, _VP, _VP], C.c_int),
    "me_sobol": ([C.c_uint64, C.c_int, C.c_int, _VP, _VP], C.c_int),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgenesis.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libgenesis.so is not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(rc: int):
    if rc != ME_OK:
        msg = load().me_last_error().decode()
        raise GenesisError(rc, msg)
