"""ctypes declarations of the C ABI in include/sv.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsv.so")

SV_OK, SV_ERR_ARG, SV_ERR_OOM, SV_ERR_CUDA, SV_ERR_PLAN, SV_ERR_TIMEOUT, SV_ERR_UNSUPPORTED = range(7)
SV_C64, SV_C128 = 1, 2
SV_GATE_SWAP, SV_GATE_DIAG = 1, 2
(SV_K_UNITARY1, SV_K_UNITARY2, SV_K_U3, SV_K_CX, SV_K_H, SV_K_X, SV_K_Y, SV_K_Z, SV_K_RY, SV_K_RZ,
 SV_K_CP, SV_K_CZ, SV_K_SWAP) = range(13)

STATUS_NAMES = {0: "SV_OK", 1: "SV_ERR_ARG", 2: "SV_ERR_OOM", 3: "SV_ERR_CUDA", 4: "SV_ERR_PLAN",
                5: "SV_ERR_TIMEOUT", 6: "SV_ERR_UNSUPPORTED"}

GATE_DTYPE = np.dtype([("nq", np.int32), ("q", np.int32, (2,)), ("flags", np.int32), ("m", np.float64, (32,))],
                      align=True)
assert GATE_DTYPE.itemsize == 272


class sv_options(ctypes.Structure):
    _fields_ = [("chunk_bits", ctypes.c_int32), ("reserve", ctypes.c_int32), ("restore_layout", ctypes.c_int32),
                ("seg_bits", ctypes.c_int32), ("use_tc", ctypes.c_int32), ("use_model", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("gather_pinned", ctypes.c_int32), ("diag_outside", ctypes.c_int32),
                ("lookahead", ctypes.c_int32), ("tc_no_renorm", ctypes.c_int32), ("wait_limit_ms", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class sv_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("chunk_bits", ctypes.c_int32), ("reserve", ctypes.c_int32),
                ("restore_layout", ctypes.c_int32), ("n_blocks", ctypes.c_int32), ("n_swap_rounds", ctypes.c_int32),
                ("n_unpermute_rounds", ctypes.c_int32), ("n_segments", ctypes.c_int32),
                ("n_gates_emitted", ctypes.c_int64), ("final_map", ctypes.c_int32 * 64)]


class sv_apply_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("sweeps_block", ctypes.c_int64),
                ("sweeps_permute", ctypes.c_int64), ("sweeps_gate", ctypes.c_int64),
                ("algorithmic_bytes", ctypes.c_double), ("ms_block", ctypes.c_double),
                ("ms_permute", ctypes.c_double), ("ms_gate", ctypes.c_double)]


class SVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
SV_BATCH_GRAPH = 1
SV_BATCH_FROM_ZERO = 2
SV_BATCH_TEST_STALL = 4
SV_COSTMODEL_FEATURES = 16
SV_COSTMODEL_PARAMS = 5313
_VP = ctypes.c_void_p
_SIGS = {
    "sv_gate_make": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), _VP]),
    "sv_gates_make": (ctypes.c_int, [ctypes.c_int64, _VP, _VP, _VP, ctypes.c_int32, _VP]),
    "sv_options_default": (None, [ctypes.POINTER(sv_options)]),
    "sv_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "sv_destroy": (ctypes.c_int, [_VP]),
    "sv_init_basis": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "sv_get_state": (ctypes.c_int, [_VP, _VP]),
    "sv_get_state_async": (ctypes.c_int, [_VP, _VP]),
    "sv_set_state_async": (ctypes.c_int, [_VP, _VP]),
    "sv_set_state": (ctypes.c_int, [_VP, _VP]),
    "sv_device_ptr": (ctypes.c_int, [_VP, ctypes.POINTER(_VP)]),
    "sv_synchronize": (ctypes.c_int, [_VP]),
    "sv_plan_blocking": (ctypes.c_int, [ctypes.c_int32, _VP, ctypes.c_int64, ctypes.POINTER(sv_options), ctypes.POINTER(_VP)]),
    "sv_plan_free": (ctypes.c_int, [_VP]),
    "sv_plan_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(sv_plan_info)]),
    "sv_plan_get_widths": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "sv_plan_serialize": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "sv_apply_circuit": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "sv_apply_plan_ops": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_int32]),
    "sv_shard_pack": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP]),
    "sv_shard_unpack": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP]),
    "sv_apply_circuit_host": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _VP, _VP, ctypes.c_int64, _VP, _VP,
                                             ctypes.c_size_t, _VP, _VP]),
    "sv_get_apply_stats": (ctypes.c_int, [_VP, ctypes.POINTER(sv_apply_stats)]),
    "sv_probabilities": (ctypes.c_int, [_VP, _VP, ctypes.c_int32]),
    "sv_norm2": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "sv_sample": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_uint64, _VP]),
    "sv_expval_pauli": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "sv_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "sv_expval_pauli_noalloc": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "sv_batch_create": (ctypes.c_int, [ctypes.c_int32, _VP, _VP, _VP, ctypes.POINTER(sv_options), ctypes.POINTER(_VP)]),
    "sv_batch_run": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "sv_batch_sync": (ctypes.c_int, [_VP]),
    "sv_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_double)]),
    "sv_batch_tune": (ctypes.c_int, [ctypes.c_int32, _VP, _VP, _VP, ctypes.POINTER(sv_options),
                                     ctypes.POINTER(sv_options), ctypes.POINTER(ctypes.c_double)]),
    "sv_batch_free": (ctypes.c_int, [_VP]),
    "sv_autotune": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _VP, ctypes.c_int64, ctypes.POINTER(sv_options),
                                   ctypes.POINTER(sv_options), ctypes.POINTER(ctypes.c_double)]),
    "sv_costmodel_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(_VP)]),
    "sv_costmodel_free": (ctypes.c_int, [_VP]),
    "sv_costmodel_get_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "sv_costmodel_set_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "sv_costmodel_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "sv_costmodel_gradient": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.POINTER(ctypes.c_double)]),
    "sv_costmodel_adam_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_float,
                                              ctypes.POINTER(ctypes.c_double)]),
    "sv_costmodel_add_samples": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64]),
    "sv_costmodel_num_samples": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "sv_costmodel_collect": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_uint64,
                                            ctypes.POINTER(ctypes.c_int64)]),
    "sv_costmodel_train": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_double)]),
    "sv_costmodel_predict_us": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP]),
    "sv_costmodel_features": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_int64)]),
    "sv_plan_blocking_steered": (ctypes.c_int, [ctypes.c_int32, _VP, ctypes.c_int64, ctypes.POINTER(sv_options),
                                                ctypes.c_int32, _VP, ctypes.POINTER(_VP)]),
    "sv_get_launch_times": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "sv_last_error": (ctypes.c_char_p, []),
}


def exported_names():
    return list(_SIGS)


def lib():
    """Load libsv.so (built by paper_2102_02957_gb300.build). Raises if it is missing: there is
    no fallback implementation."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run paper_2102_02957_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int):
    if status != SV_OK:
        msg = lib().sv_last_error()
        raise SVError(status, msg.decode() if msg else "")
