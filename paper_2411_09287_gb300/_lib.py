"""ctypes declarations of the C-ABI in include/mpc3.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_LIB = None

c_u64p = C.POINTER(C.c_uint64)


class MpcConfig(C.Structure):
    _fields_ = [("seed", C.c_uint8 * 32), ("device", C.c_int), ("reduce_mode", C.c_int),
                ("gemm_path", C.c_int), ("stream", C.c_void_p)]


class MpcTuning(C.Structure):
    _fields_ = [("trunc_block", C.c_int64), ("trunc_chunk", C.c_int64), ("row_split", C.c_int64),
                ("tc_combine_min", C.c_int32), ("gemm_split_min", C.c_int32),
                ("gram_split", C.c_int32), ("fold_batch_max", C.c_int32),
                ("gr_producers", C.c_int32), ("gr_drain_warps", C.c_int32)]


_SIGS = {
    "mpc_create": (C.c_int, [C.POINTER(MpcConfig), C.POINTER(C.c_void_p)]),
    "mpc_destroy": (None, [C.c_void_p]),
    "mpc_last_error": (C.c_char_p, [C.c_void_p]),
    "mpc_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mpc_h2d_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "mpc_h2d_wait": (C.c_int, [C.c_void_p, C.c_int]),
    "mpc_d2h_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "mpc_sync": (C.c_int, [C.c_void_p]),
    "mpc_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(MpcTuning)]),
    "mpc_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(MpcTuning)]),
    "mpc_trace_words": (C.c_int64, [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_int64,
                                    C.c_int, C.c_int, C.c_int]),
    "mpc_status": (C.c_int, [C.c_void_p]),
    "mpc_workspace_size": (C.c_int64, [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_int64,
                                       C.c_int, C.c_int, C.c_int]),
    "mpc_share_input": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int, C.c_int64,
                                  C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_share_input_from": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_int,
                                       C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_mult": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64,
                           C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_matmul": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64,
                             C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_size_t]),
    "mpc_verify_mult": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int64, C.c_uint64, C.c_int, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "mpc_verify_mult_calls": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_uint64), C.c_int,
                                        C.c_void_p, C.c_size_t, C.c_void_p]),
    "mpc_verify_matmul": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int,
                                    C.c_uint64, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                    C.c_void_p]),
    "mpc_reconstruct": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int,
                                  C.c_void_p, C.c_size_t]),
    "mpc_ledger": (C.c_int, [C.c_void_p, c_u64p, c_u64p]),
    "mpc_ledger_reset": (None, [C.c_void_p]),
    "mpc_inject_fault": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64]),
    "mpc_reconstruct_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mpc_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "mpc_gather": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "mpc_hash_u64": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "mpc_relu": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p,
                           C.c_void_p, C.c_size_t, C.c_void_p]),
    "mpc_maxpool2": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p, C.c_int64, C.c_int64,
                               C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "mpc_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), c_u64p,
                                   C.POINTER(C.c_double)]),
    "mpc_launch_count": (C.c_uint64, []),
    "mpc_test_wait_expires": (C.c_int, [C.c_void_p, C.c_int64]),
    "mpc_matmul_keyed": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64,
                                   C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_verify_matmul_keyed": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                          C.c_int, C.c_void_p, C.c_uint64, C.c_int, C.c_int,
                                          C.c_void_p, C.c_size_t, C.c_void_p]),
    "mpc_share_fixed": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.c_void_p, C.c_int, C.c_int64,
                                  C.c_int, C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_reconstruct_fixed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                                        C.c_int, C.c_void_p, C.c_size_t]),
    "mpc_conv2d": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p,
                             C.POINTER(C.c_int32), C.c_int64, C.c_int, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_trunc": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64, C.c_int, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_size_t]),
    "mpc_verify_trunc": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64, C.c_int,
                                   C.c_uint64, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load libmpc3.so; raises if it is missing (there is no fallback implementation)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libmpc3 is not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = C.CDLL(path, mode=C.RTLD_GLOBAL)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def declared_symbols() -> list:
    return list(_SIGS)
