"""Scalar Grain oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and ``bench.py``'s CPU legs may import this module; the
product shares no code with it.  ``grain_oracle.c`` (plain C, built here
with gcc) states Grain v1, the paper's second stream cipher (Sec. II-C-3:
80-bit LFSR and NFSR, 80-bit key, 64-bit IV, 160 initialisation clocks),
one bit per byte, in the specification's order; the bit order (least
significant bit first, for key, IV and keystream bytes) is the one the
specification's test vectors fix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "grain_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgrain_oracle.so")
_lock = threading.Lock()
_lib = None

REG = 80
KEY_BYTES = 10
IV_BYTES = 8
INIT_CLOCKS = 160


class State(ctypes.Structure):
    """One Grain state: s[0..79] (LFSR), b[0..79] (NFSR), one bit per byte."""
    _fields_ = [("s", ctypes.c_uint8 * REG), ("b", ctypes.c_uint8 * REG)]

    def bits(self):
        return (np.frombuffer(bytes(self.s), np.uint8).copy(),
                np.frombuffer(bytes(self.b), np.uint8).copy())

    @classmethod
    def from_bits(cls, s, b):
        st = cls()
        for i in range(REG):
            st.s[i] = int(s[i]) & 1
            st.b[i] = int(b[i]) & 1
        return st


def build(force: bool = False) -> str:
    """Compile grain_oracle.c with gcc into oracle/_build (if stale)."""
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
            sp = ctypes.POINTER(State)
            L.grain_oracle_output.argtypes = [sp]
            L.grain_oracle_output.restype = ctypes.c_uint8
            L.grain_oracle_clock.argtypes = [sp, ctypes.c_int]
            L.grain_oracle_init.argtypes = [sp, ctypes.c_char_p, ctypes.c_char_p]
            L.grain_oracle_keystream.argtypes = [sp, ctypes.c_uint64, ctypes.c_void_p,
                                                 ctypes.c_uint64]
            L.grain_oracle_stream.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_uint64,
                                              ctypes.c_void_p]
            L.grain_oracle_batch.argtypes = [ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
            L.grain_oracle_batch.restype = ctypes.c_int
            L.grain_oracle_state_size.restype = ctypes.c_size_t
            assert L.grain_oracle_state_size() == ctypes.sizeof(State)
            _lib = L
    return _lib


def output(st: State) -> int:
    return int(lib().grain_oracle_output(ctypes.byref(st)))


def clock(st: State, extra: int = 0) -> None:
    lib().grain_oracle_clock(ctypes.byref(st), int(extra))


def init(key: bytes, iv: bytes) -> State:
    st = State()
    lib().grain_oracle_init(ctypes.byref(st), bytes(key), bytes(iv))
    return st


def keystream_from(st: State, n_bits: int) -> bytes:
    """Continue `st` for n_bits; ceil(n_bits/8) bytes, least significant bit first."""
    out = (ctypes.c_uint8 * ((n_bits + 7) // 8))()
    lib().grain_oracle_keystream(ctypes.byref(st), n_bits, out, 0)
    return bytes(out)


def stream(key: bytes, iv: bytes, n_bits: int) -> bytes:
    out = (ctypes.c_uint8 * ((n_bits + 7) // 8))()
    lib().grain_oracle_stream(bytes(key), bytes(iv), n_bits, out)
    return bytes(out)


def batch_bytes(keys, ivs, n_bits: int, threads: int = 1) -> np.ndarray:
    """Keystreams of many streams: uint8 [n, ceil(n_bits/8)], row i from
    keys[i] (10 bytes) and ivs[i] (8 bytes)."""
    k = np.ascontiguousarray(keys, np.uint8).reshape(-1, KEY_BYTES)
    v = np.ascontiguousarray(ivs, np.uint8).reshape(-1, IV_BYTES)
    n = k.shape[0]
    out = np.zeros((n, (n_bits + 7) // 8), np.uint8)
    if lib().grain_oracle_batch(n, k.ctypes.data, v.ctypes.data, n_bits, out.ctypes.data,
                                int(threads)) != 0:
        raise MemoryError("oracle batch")
    return out


def to_bitsliced(rows: np.ndarray, n_bits: int) -> np.ndarray:
    """Column-major layout of Sec. IV-A: out[g, t] has bit l = z_t of
    instance 32g + l (rows: least-significant-bit-first bytes)."""
    n = rows.shape[0]
    G = (n + 31) // 32
    bits = np.unpackbits(np.asarray(rows, np.uint8), axis=1, bitorder="little")[:, :n_bits]
    pad = np.zeros((G * 32, n_bits), np.uint8)
    pad[:n] = bits
    w = pad.reshape(G, 32, n_bits).astype(np.uint64)
    out = np.zeros((G, n_bits), np.uint64)
    for l in range(32):
        out |= w[:, l, :] << np.uint64(l)
    return out.astype(np.uint32)
