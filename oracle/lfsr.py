"""Scalar LFSR and CRC-8 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and ``__graft_entry__`` may import this module; the product
shares no code with it.  ``lfsr_oracle.c`` (plain C, built here with gcc)
follows the paper's LFSR (Sec. II-B and IV-C, Eq. 1 and 2: output x_0,
feedback XOR of a_i x_i into x_{n-1}, shift down) and its CRC-8 example
(Sec. IV-B, Figs. CRC1 and CRC2: MSB first, register preset, polynomial
with implicit x^8, final XOR), one bit per byte.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfsr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblfsr_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lfsr_oracle.c with gcc into oracle/_build (if stale)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC,
                        "-lpthread"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.lfsr_oracle_generate.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.c_void_p]
            L.lfsr_oracle_generate.restype = ctypes.c_int
            L.crc8_oracle.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.c_uint8,
                                      ctypes.c_uint8, ctypes.c_uint8]
            L.crc8_oracle.restype = ctypes.c_uint8
            L.crc8_oracle_batch.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                            ctypes.c_uint8, ctypes.c_uint8, ctypes.c_uint8,
                                            ctypes.c_void_p, ctypes.c_int]
            L.crc8_oracle_batch.restype = ctypes.c_int
            _lib = L
    return _lib


def lfsr_bits(seed: int, degree: int, taps: int, n_bits: int) -> np.ndarray:
    """Output bits x_0(t), t = 0 .. n_bits-1, of one LFSR (uint8 0/1)."""
    out = np.zeros(n_bits, np.uint8)
    if lib().lfsr_oracle_generate(seed, degree, taps, n_bits, out.ctypes.data) != 0:
        raise ValueError("degree must be 2..64")
    return out


def crc8(msg: bytes, poly: int, init: int = 0, xorout: int = 0) -> int:
    return int(lib().crc8_oracle(bytes(msg), len(msg), poly, init, xorout))


def crc8_batch(data: np.ndarray, poly: int, init: int = 0, xorout: int = 0,
               threads: int = 1) -> np.ndarray:
    """CRC of every row of a uint8 [n, len] array."""
    d = np.ascontiguousarray(data, np.uint8)
    n, ln = d.shape
    out = np.zeros(n, np.uint8)
    if lib().crc8_oracle_batch(d.ctypes.data, n, ln, poly, init, xorout, out.ctypes.data,
                               int(threads)) != 0:
        raise MemoryError("oracle batch")
    return out
