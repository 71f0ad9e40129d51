"""ctypes binding of libmickey.so (the C ABI of include/mickey.h).

Argument marshalling only: every step of the keystream path runs in the
library's CUDA kernels.  If the library has not been built this module
raises; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmickey.so")

OK = 0
E_ARG, E_IVLEN, E_LIMIT, E_LAYOUT, E_OOM, E_CUDA, E_TIMEOUT, E_STATE = range(-1, -9, -1)
LAYOUT_BITSLICED_U32, LAYOUT_BYTES, LAYOUT_U32, LAYOUT_U32_F32 = 0, 1, 2, 3
MEM_HOST, MEM_DEVICE = 0, 1
MODE_AUTO, MODE_GRID, MODE_PERSISTENT, MODE_PERSISTENT2 = 0, 1, 2, 3
BATCH_SPLIT_SHARED, BATCH_SPLIT_OWN = 0, 1


class TuneResult(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("unroll", ctypes.c_int), ("stage", ctypes.c_int),
                ("ms", ctypes.c_float)]
MAX_STREAM_BITS = 1 << 40

_lock = threading.Lock()
_lib = None

c_void_p, c_size_t, c_uint64, c_int, c_char_p = (ctypes.c_void_p, ctypes.c_size_t,
                                                 ctypes.c_uint64, ctypes.c_int,
                                                 ctypes.c_char_p)
c_uint8 = ctypes.c_uint8

# name: (restype, argtypes)
SIGNATURES = {
    "mickey_lfsr_generate": (c_int, [c_void_p, c_size_t, c_int, c_uint64, c_uint64, c_void_p, c_int,
                                     c_void_p]),
    "mickey_crc8": (c_int, [c_void_p, c_size_t, c_size_t, c_uint8, c_uint8, c_uint8, c_void_p, c_int,
                            c_void_p]),
    "mickey_init_streams": (c_void_p, [c_void_p, c_void_p, c_void_p, c_size_t]),
    "mickey_init_streams_ex": (c_void_p, [c_void_p, c_void_p, c_void_p, c_size_t, c_int,
                                          c_void_p]),
    "mickey_reset_streams": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "mickey_set_stream": (c_int, [c_void_p, c_void_p]),
    "mickey_generate": (c_int, [c_void_p, c_uint64, c_void_p, c_int]),
    "mickey_output_bytes": (c_size_t, [c_size_t, c_uint64, c_int]),
    "mickey_generate_ragged": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "mickey_ragged_output_bytes": (c_size_t, [c_size_t, c_void_p, c_int]),
    "mickey_generate_host": (c_int, [c_void_p, c_uint64, c_void_p, c_int]),
    "mickey_sync": (c_int, [c_void_p]),
    "mickey_num_streams": (c_size_t, [c_void_p]),
    "mickey_position": (c_uint64, [c_void_p, c_size_t]),
    "mickey_export_state": (c_int, [c_void_p, c_void_p, c_void_p]),
    "mickey_import_state": (c_void_p, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "mickey_free": (None, [c_void_p]),
    "mickey_last_error": (c_int, []),
    "mickey_last_error_message": (c_char_p, []),
    "mickey_error_string": (c_char_p, [c_int]),
    "mickey_tables": (None, [c_void_p]),
    "mickey_ops_per_clock": (c_int, [c_int]),
    "mickey_version": (c_char_p, []),
    "mickey_probe_lop3": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "mickey_probe_clock": (c_int, [c_int, c_int, c_void_p, c_void_p]),
    "mickey_set_config": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
    "mickey_get_config": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "mickey_tune": (c_int, [c_void_p, c_uint64, c_int, c_void_p, c_int, c_void_p]),
    "mickey_batch_create": (c_void_p, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "mickey_batch_output_bytes": (c_size_t, [c_void_p]),
    "mickey_batch_offsets": (c_int, [c_void_p, c_void_p]),
    "mickey_batch_clocks": (c_int, [c_void_p, c_void_p, c_void_p]),
    "mickey_batch_run": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "mickey_batch_set_config": (c_int, [c_void_p, c_int, c_int, c_uint64]),
    "mickey_batch_get_config": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "mickey_batch_set_split_mode": (c_int, [c_void_p, c_int]),
    "mickey_batch_get_split_mode": (c_int, [c_void_p]),
    "mickey_batch_sync": (c_int, [c_void_p]),
    "mickey_batch_free": (None, [c_void_p]),
    "mickey_server_create": (c_void_p, [c_size_t, ctypes.c_uint32, c_void_p]),
    "mickey_server_init_streams": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                           c_size_t]),
    "mickey_server_step": (c_int, [c_void_p, ctypes.c_uint32, ctypes.c_uint32, c_void_p,
                                   c_void_p, c_void_p]),
    "mickey_server_read_states": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p]),
    "mickey_server_set_config": (c_int, [c_void_p, c_int, c_int]),
    "mickey_server_sync": (c_int, [c_void_p]),
    "mickey_server_free": (None, [c_void_p]),
    "mickey_init_state_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, c_void_p,
                                          c_void_p]),
    "grain_init_streams": (c_void_p, [c_void_p, c_void_p, c_size_t, c_int, c_void_p]),
    "grain_reset_streams": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "grain_generate": (c_int, [c_void_p, c_uint64, c_void_p, c_int]),
    "grain_output_bytes": (c_size_t, [c_size_t, c_uint64, c_int]),
    "grain_set_stream": (c_int, [c_void_p, c_void_p]),
    "grain_sync": (c_int, [c_void_p]),
    "grain_position": (c_uint64, [c_void_p]),
    "grain_export_state": (c_int, [c_void_p, c_void_p]),
    "grain_ops_per_clock": (c_int, [c_int]),
    "grain_free": (None, [c_void_p]),
    "grain_probe_clock": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p]),
}


class MickeyError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("mickey error %d: %s" % (code, message))
        self.code = code
        self.message = message


def lib():
    """Load libmickey.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libmickey.so is not built (%s); run `python -m "
                    "paper_1909_04750_gb300.build` or __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> MickeyError:
    L = lib()
    code = L.mickey_last_error()
    msg = L.mickey_last_error_message()
    return MickeyError(code, msg.decode() if msg else "")


def check(rc: int) -> int:
    if rc != OK:
        raise last_error()
    return rc


def check_ptr(p):
    if not p:
        raise last_error()
    return p
