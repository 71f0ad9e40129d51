"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/mickey.h declares, carries the same constant tables as the oracle,
and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return N.lib()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"MICKEY_API[^;{]*?\b(mickey_\w+)\s*\(", text, re.S))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 19
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_declarations():
    assert set(declared_symbols()) <= set(N.SIGNATURES)


def test_kernel_tables_match_oracle(L):
    m = (ctypes.c_uint32 * 20)()
    L.mickey_tables(m)
    words = np.frombuffer(bytes(m), np.uint32).reshape(5, 4)
    ref = oracle.tables()
    for row, name in enumerate(("rtaps", "comp0", "comp1", "fb0", "fb1")):
        bits = np.array([(words[row, i // 32] >> (i % 32)) & 1 for i in range(100)], np.uint8)
        if name in ("comp0", "comp1"):
            # defined for positions 1..98 only
            assert np.array_equal(bits[1:99], ref[name][1:99]), name
        else:
            assert np.array_equal(bits, ref[name]), name


def test_ops_per_clock_counts(L):
    t = oracle.tables()
    fb = (t["fb0"] | t["fb1"])[1:99]
    taps = int(t["rtaps"].sum())
    # CONTROL_BIT_R, R: one op per bit + one per tap except bit 0 (folded),
    # f0/f1, S: one op per bit 1..98 + one per feedback position, S'_99, z.
    expect = 1 + (100 + taps - 1) + 2 + (98 + int(fb.sum())) + 1 + 1
    assert L.mickey_ops_per_clock(0) == expect
    assert L.mickey_ops_per_clock(1) == expect + 2


def test_output_bytes(L):
    assert L.mickey_output_bytes(33, 64, N.LAYOUT_BITSLICED_U32) == 2 * 64 * 4
    assert L.mickey_output_bytes(33, 65, N.LAYOUT_BYTES) == 33 * 9
    assert L.mickey_output_bytes(33, 64, N.LAYOUT_U32) == 33 * 8
    assert L.mickey_output_bytes(33, 64, N.LAYOUT_U32_F32) == 33 * 16
    assert L.mickey_output_bytes(33, 65, N.LAYOUT_U32) == 0
    assert L.mickey_output_bytes(33, 64, 9) == 0


def test_invalid_arguments_rejected_on_host(L):
    keys = np.zeros((4, 10), np.uint8)
    assert not L.mickey_init_streams(None, keys.ctypes.data, None, 4)
    assert L.mickey_last_error() == N.E_ARG
    assert not L.mickey_init_streams(keys.ctypes.data, keys.ctypes.data, None, 0)
    assert L.mickey_last_error() == N.E_ARG
    lens = np.array([80, 81, 0, 5], np.uint32)
    assert not L.mickey_init_streams(keys.ctypes.data, keys.ctypes.data, lens.ctypes.data, 4)
    assert L.mickey_last_error() == N.E_IVLEN
    assert b"81" in L.mickey_last_error_message()
    assert L.mickey_generate(None, 32, None, 0) == N.E_ARG
    assert L.mickey_sync(None) == N.E_ARG
    L.mickey_free(None)
    assert L.mickey_error_string(N.E_LIMIT) == b"more than 2^40 keystream bits for one key/IV"
    assert L.mickey_version().startswith(b"mickey-gb300")
