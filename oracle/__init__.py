"""Scalar MICKEY 2.0 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1909_04750_gb300``)
never imports it and shares no code with it.

Contents
--------
* A ctypes binding to ``mickey_oracle.c`` (plain C, built here with gcc):
  the cipher's procedures CLOCK_R, CLOCK_S, CLOCK_KG, key/IV loading and
  keystream generation, one bit per byte, following the MICKEY 2.0
  specification that the paper cites for the cipher (Sec. II-C-1) and
  bitslices (Sec. IV-D).
* Plain numpy statements of the output layouts the GPU path produces:
  row-major bytes, the column-major "bitsliced" layout of Sec. IV-A (word t
  of group g holds bit t of 32 instances, lane l = instance 32g+l), row-major
  big-endian u32 words, and FP32 uniforms from the top 24 bits of each word.

Every function here is slow on purpose and is written to be checked by eye.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mickey_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmickey_oracle.so")
_lock = threading.Lock()
_lib = None

REG = 100
KEY_BITS = 80
MAX_IV_BITS = 80
PRECLOCKS = 100


class State(ctypes.Structure):
    """One MICKEY 2.0 state: r[0..99], s[0..99], one bit per byte."""

    _fields_ = [("r", ctypes.c_uint8 * REG), ("s", ctypes.c_uint8 * REG)]

    def bits(self):
        return np.frombuffer(bytes(self.r), np.uint8).copy(), np.frombuffer(
            bytes(self.s), np.uint8).copy()

    @classmethod
    def from_bits(cls, r, s):
        st = cls()
        for i in range(REG):
            st.r[i] = int(r[i]) & 1
            st.s[i] = int(s[i]) & 1
        return st


def build(force: bool = False) -> str:
    """Compile mickey_oracle.c with gcc into oracle/_build (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                        "-Wall", "-o", tmp, _SRC, "-lpthread"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            sp = ctypes.POINTER(State)
            L.mickey_oracle_tables.argtypes = [u8p] * 5
            L.mickey_oracle_clock_r.argtypes = [sp, ctypes.c_int, ctypes.c_int]
            L.mickey_oracle_clock_s.argtypes = [sp, ctypes.c_int, ctypes.c_int]
            L.mickey_oracle_clock_kg.argtypes = [sp, ctypes.c_int, ctypes.c_int]
            L.mickey_oracle_init.argtypes = [sp, ctypes.c_char_p,
                                             ctypes.c_char_p, ctypes.c_uint32]
            L.mickey_oracle_init.restype = ctypes.c_int
            L.mickey_oracle_keystream.argtypes = [sp, ctypes.c_uint64,
                                                  ctypes.c_void_p,
                                                  ctypes.c_uint64]
            L.mickey_oracle_stream.argtypes = [ctypes.c_char_p, ctypes.c_char_p,
                                               ctypes.c_uint32, ctypes.c_uint64,
                                               ctypes.c_void_p]
            L.mickey_oracle_stream.restype = ctypes.c_int
            L.mickey_oracle_batch.argtypes = [
                ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_int]
            L.mickey_oracle_batch.restype = ctypes.c_int
            L.mickey_oracle_state_size.restype = ctypes.c_size_t
            assert L.mickey_oracle_state_size() == ctypes.sizeof(State)
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# cipher procedures
# --------------------------------------------------------------------------

def tables():
    """The five constant tables as uint8 arrays of length 100 (0/1)."""
    bufs = [(ctypes.c_uint8 * REG)() for _ in range(5)]
    lib().mickey_oracle_tables(*bufs)
    names = ("rtaps", "comp0", "comp1", "fb0", "fb1")
    return {n: np.frombuffer(bytes(b), np.uint8).copy() for n, b in zip(names, bufs)}


def clock_r(st: State, input_bit_r: int, control_bit_r: int) -> None:
    lib().mickey_oracle_clock_r(ctypes.byref(st), input_bit_r, control_bit_r)


def clock_s(st: State, input_bit_s: int, control_bit_s: int) -> None:
    lib().mickey_oracle_clock_s(ctypes.byref(st), input_bit_s, control_bit_s)


def clock_kg(st: State, mixing: int, input_bit: int) -> None:
    lib().mickey_oracle_clock_kg(ctypes.byref(st), mixing, input_bit)


def init(key: bytes, iv: bytes, iv_len: int) -> State:
    st = State()
    rc = lib().mickey_oracle_init(ctypes.byref(st), bytes(key),
                                  bytes(iv) if iv is not None else None, iv_len)
    if rc != 0:
        raise ValueError("iv_len %d exceeds 80 bits" % iv_len)
    return st


def keystream_from(st: State, n_bits: int) -> bytes:
    """Continue `st` for n_bits; returns ceil(n_bits/8) bytes, MSB first."""
    out = (ctypes.c_uint8 * ((n_bits + 7) // 8))()
    lib().mickey_oracle_keystream(ctypes.byref(st), n_bits, out, 0)
    return bytes(out)


def stream(key: bytes, iv: bytes, iv_len: int, n_bits: int) -> bytes:
    out = (ctypes.c_uint8 * ((n_bits + 7) // 8))()
    rc = lib().mickey_oracle_stream(bytes(key), bytes(iv), iv_len, n_bits, out)
    if rc != 0:
        raise ValueError("iv_len %d exceeds 80 bits" % iv_len)
    return bytes(out)


def batch_bytes(keys, ivs, iv_lens, n_bits, threads: int = 1):
    """Keystreams of many streams, row-major bytes.

    keys, ivs: uint8 [n, 10]; iv_lens: [n]; n_bits: scalar or [n].
    Returns a list of per-stream byte arrays when lengths differ, else a
    uint8 array [n, ceil(n_bits/8)].
    """
    keys = np.ascontiguousarray(keys, np.uint8).reshape(-1, 10)
    ivs = np.ascontiguousarray(ivs, np.uint8).reshape(-1, 10)
    n = keys.shape[0]
    lens = np.ascontiguousarray(np.broadcast_to(np.asarray(iv_lens, np.uint32), (n,)))
    nb = np.ascontiguousarray(np.broadcast_to(np.asarray(n_bits, np.uint64), (n,)))
    nbytes = (nb + 7) // 8
    offs = np.zeros(n, np.uint64)
    if n > 1:
        offs[1:] = np.cumsum(nbytes[:-1])
    out = np.zeros(int(nbytes.sum()), np.uint8)
    rc = lib().mickey_oracle_batch(
        n, keys.ctypes.data, ivs.ctypes.data, lens.ctypes.data, nb.ctypes.data,
        out.ctypes.data, offs.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("oracle batch failed (iv_len > 80?)")
    if n and np.all(nb == nb[0]):
        return out.reshape(n, int(nbytes[0]))
    return [out[int(o):int(o) + int(c)] for o, c in zip(offs, nbytes)]


# --------------------------------------------------------------------------
# output layouts (plain numpy, from the row-major bytes)
# --------------------------------------------------------------------------

def bits_of(rows: np.ndarray, n_bits: int) -> np.ndarray:
    """[n, nbytes] MSB-first bytes -> [n, n_bits] array of 0/1."""
    return np.unpackbits(np.asarray(rows, np.uint8), axis=1, bitorder="big")[:, :n_bits]


def bytes_of(bits: np.ndarray) -> np.ndarray:
    """[n, n_bits] 0/1 -> [n, ceil(n_bits/8)] MSB-first bytes."""
    return np.packbits(np.asarray(bits, np.uint8), axis=1, bitorder="big")


def to_bitsliced(rows: np.ndarray, n_bits: int) -> np.ndarray:
    """Column-major layout of Sec. IV-A: out[g, t] has bit l = z_t of
    instance 32*g + l.  Lanes past the last instance read as zero."""
    bits = bits_of(rows, n_bits).astype(np.uint32)
    n = bits.shape[0]
    groups = (n + 31) // 32
    padded = np.zeros((groups * 32, n_bits), np.uint32)
    padded[:n] = bits
    padded = padded.reshape(groups, 32, n_bits)
    out = np.zeros((groups, n_bits), np.uint32)
    for lane in range(32):
        out |= padded[:, lane, :] << np.uint32(lane)
    return out


def from_bitsliced(words: np.ndarray, n: int) -> np.ndarray:
    """Inverse of to_bitsliced: [G, n_bits] words -> [n, ceil(n_bits/8)] bytes."""
    words = np.asarray(words, np.uint32)
    groups, n_bits = words.shape
    bits = np.zeros((groups, 32, n_bits), np.uint8)
    for lane in range(32):
        bits[:, lane, :] = (words >> np.uint32(lane)) & 1
    return bytes_of(bits.reshape(groups * 32, n_bits)[:n])


def to_u32(rows: np.ndarray, n_bits: int) -> np.ndarray:
    """Row-major words: out[i, k] holds z_{32k..32k+31} with z_{32k} as the
    most significant bit (big-endian read of 4 keystream bytes)."""
    if n_bits % 32:
        raise ValueError("u32 layout needs n_bits % 32 == 0")
    b = np.asarray(rows, np.uint8)[:, : n_bits // 8].astype(np.uint32)
    b = b.reshape(b.shape[0], -1, 4)
    return (b[:, :, 0] << 24) | (b[:, :, 1] << 16) | (b[:, :, 2] << 8) | b[:, :, 3]


def to_f32(words: np.ndarray) -> np.ndarray:
    """FP32 uniform in [0, 1) from the top 24 bits of each word:
    (w >> 8) * 2**-24, formed in float64 (exact) and rounded to float32
    (exact too, since the value has at most 24 significant bits)."""
    w = np.asarray(words, np.uint64)
    return ((w >> np.uint64(8)).astype(np.float64) * 2.0 ** -24).astype(np.float32)
