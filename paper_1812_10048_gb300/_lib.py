"""ctypes binding of libdpmm.so (include/dpmm.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only
converts Python / numpy / torch arguments to pointers and sizes.  If the
shared library is missing the first call raises: there is no fallback.
"""

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdpmm.so")

DPMM_OK = 0
ERRORS = {-1: "DPMM_EINVAL", -2: "DPMM_ENOMEM", -3: "DPMM_ECUDA", -4: "DPMM_ECAPACITY",
          -5: "DPMM_EOVERFLOW", -6: "DPMM_ETIMEOUT", -7: "DPMM_ESTATE"}

ENGINE_AUTO, ENGINE_CSR_FP32, ENGINE_TILE_BF16 = 0, 1, 2


class DpmmError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{ERRORS.get(code, code)}: {message}")
        self.code = code


class dpmm_opts(ctypes.Structure):
    _fields_ = [("kmax", ctypes.c_int32), ("engine", ctypes.c_int32), ("split_q", ctypes.c_int32),
                ("chain_id", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("hastings", ctypes.c_int32), ("open_new_cluster", ctypes.c_int32),
                ("local_iters", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class dpmm_tuning(ctypes.Structure):
    _fields_ = [("stats_blocks_per_sm", ctypes.c_int32), ("tile_stages", ctypes.c_int32),
                ("tile_scatter", ctypes.c_int32), ("draw_blocks_per_sm", ctypes.c_int32),
                ("local_lanes", ctypes.c_int32), ("local_stream", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


_P = ctypes.c_void_p
_I32, _I64, _U64, _F64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double

# name: (restype, argtypes)
SIGNATURES = {
    "dpmm_default_opts": (None, [ctypes.POINTER(dpmm_opts)]),
    "dpmm_init": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, _P, _I64, _I32, _F64, _F64,
                                 ctypes.POINTER(dpmm_opts), _P]),
    "dpmm_free": (None, [_P]),
    "dpmm_sweep": (ctypes.c_int, [_P, _I32]),
    "dpmm_split_merge": (ctypes.c_int, [_P, _I32, _P]),
    "dpmm_step": (ctypes.c_int, [_P, _I32]),
    "dpmm_labels": (ctypes.c_int, [_P, _P, _P]),
    "dpmm_sync": (ctypes.c_int, [_P]),
    "dpmm_plans_applied": (ctypes.c_int, [_P, _P]),
    "dpmm_debug_engine": (ctypes.c_int, [_P, _P]),
    "dpmm_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(dpmm_tuning)]),
    "dpmm_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(dpmm_tuning)]),
    "dpmm_init_batch": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _I32, _P, _P, _P, _P]),
    "dpmm_chain": (ctypes.c_int, [_P, _I32, _P]),
    "dpmm_logml_grad": (ctypes.c_int, [_P, _P, _I32, ctypes.c_double, _P, _P, _P, _P]),
    "dpmm_set_hyper": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double]),
    "dpmm_eb_step": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, _P, _P,
                                    _P]),
    "dpmm_profile": (ctypes.c_int, [_P, _I32]),
    "dpmm_phase_times": (ctypes.c_int, [_P, _P, _I32]),
    "dpmm_stream": (_P, [_P]),
    "dpmm_last_error": (ctypes.c_char_p, []),
    "dpmm_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "dpmm_set_state": (ctypes.c_int, [_P, _P, _P, _I32, _I64, _I64, _P]),
    "dpmm_get_stats": (ctypes.c_int, [_P, _P, _P, _P]),
    "dpmm_draw_params": (ctypes.c_int, [_P]),
    "dpmm_debug_tile_layout": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "dpmm_local_gibbs": (ctypes.c_int, [_P, ctypes.c_int32]),
    "dpmm_assign": (ctypes.c_int, [_P]),
    "dpmm_get_params": (ctypes.c_int, [_P, _P, _P]),
    "dpmm_set_params": (ctypes.c_int, [_P, _P, _P]),
    "dpmm_debug_scores": (ctypes.c_int, [_P, _P, _I32, _P]),
    "dpmm_debug_moves": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "dpmm_debug_tile_scores": (ctypes.c_int, [_P, _P]),
    "dpmm_logml_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, _P, _I64, _I32, _P, _I32,
                                         _P]),
    "dpmm_logml_free": (None, [_P]),
    "dpmm_logml_forward": (ctypes.c_int, [_P, _F64, _P, _P]),
    "dpmm_logml_backward": (ctypes.c_int, [_P, _F64, _P, _P, _P]),
    "dpmm_logml_grad_noalloc": (ctypes.c_int, [_P, _P, _P, _I64, _I32, _P, _I32, _F64, _P, _P,
                                               _P, _P, _P]),
    "dpmm_debug_philox": (ctypes.c_int, [_P, _U64, _P, _I64]),
    "dpmm_debug_curand_philox": (ctypes.c_int, [_U64, _I64, _P]),
    "dpmm_debug_tc_gemm": (ctypes.c_int, [_P, _P, _I32, _I32, _P]),
}

_lib = None


def lib():
    """Load libdpmm.so (built in-tree by ``build.build()``); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1812_10048_gb300.build.build() (no CPU fallback exists)")
        l = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(l, name)
            fn.restype = res
            fn.argtypes = args
        _lib = l
    return _lib


def check(rc):
    if rc != DPMM_OK:
        msg = lib().dpmm_last_error()
        raise DpmmError(rc, msg.decode() if msg else "")
    return rc


def ptr(a):
    """Data pointer of a numpy array or torch tensor (must be C-contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")
