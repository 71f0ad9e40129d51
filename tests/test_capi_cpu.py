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
            names |= set(re.findall(r"MICKEY_API[^;{]*?\b((?:mickey|grain)_\w+)\s*\(", text,
                                    re.S))
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


def test_first_long_iv_length_is_named(L):
    # host IV lengths are checked block by block; the error names the first
    # length above 80, wherever it lies
    n = 10000
    keys = np.zeros((n, 10), np.uint8)
    for bad in ((5000, 81), (9999, 200), (0, 81), (4095, 81), (4096, 255)):
        lens = np.full(n, 80, np.uint32)
        lens[bad[0]] = bad[1]
        lens[min(n - 1, bad[0] + 3000)] = max(lens[min(n - 1, bad[0] + 3000)], 90)
        assert not L.mickey_init_streams(keys.ctypes.data, keys.ctypes.data, lens.ctypes.data, n)
        assert L.mickey_last_error() == N.E_IVLEN
        assert ("iv_lens[%d] = %d" % bad).encode() in L.mickey_last_error_message(), bad


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
    # the bare-clock probe checks its arguments before touching a device
    for bps, clocks in ((0, 64), (3, 64), (1, 0), (1, 6)):
        assert L.mickey_probe_clock(bps, clocks, None, None) == N.E_ARG


def _plan_only(**kw):
    # the scheduler's planning step is host logic: build the object without
    # a device (no handle), with the attributes _plan reads
    from paper_1909_04750_gb300.serve import Server
    srv = Server.__new__(Server)
    srv.quantum, srv.split_quantum = kw.get("quantum", 256), kw.get("split_quantum", 1024)
    srv.split_min_bits = kw.get("split_min_bits", 0)
    srv.max_split_groups = kw.get("max_split_groups", 1 << 20)
    srv.max_groups = kw.get("max_groups", 1 << 16)
    return srv


@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000])
def test_server_plan_groups_never_overrun(n):
    rng = np.random.default_rng(n)
    rem = (rng.integers(1, 5000, n) * 8).astype(np.int64)
    srv = _plan_only(split_min_bits=8 * 3000, max_split_groups=5)
    order, k_g, ns = srv._plan(rem)
    G = k_g.size
    assert G == (n + 31) // 32 and sorted(order.tolist()) == list(range(n))
    # longest first, every lane of a group gets the same clocks, never more
    # than its remaining bits, and at most the group's quantum
    assert np.all(np.diff(rem[order]) <= 0)
    for g in range(G):
        lanes = rem[order[32 * g:32 * g + 32]]
        assert k_g[g] == min(1024 if g < ns else 256, lanes.min())
    assert ns == min(5, (int((rem >= 8 * 3000).sum()) + 31) // 32)


def test_server_plan_caps_groups_and_splits_all_by_default():
    rem = np.full(100, 4096, np.int64)
    order, k_g, ns = _plan_only(max_groups=2)._plan(rem)
    assert k_g.size == 2 and order.size == 64 and ns == 2      # split_min_bits 0: all split
    assert np.all(k_g == 1024)


def test_served_trace_shape():
    from paper_1909_04750_gb300 import workloads
    reqs, keys = workloads.served_trace(seed=4, duration_s=2.0)
    arr = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(arr) >= 0) and arr[-1] < 2.0
    assert abs(len(reqs) / 2.0 - 1e4) < 500                    # Poisson 10^4/s
    ids = np.array([r.stream_id for r in reqs])
    new = np.r_[True, ids[1:] > np.maximum.accumulate(ids)[:-1]]
    assert abs(1 - new.mean() - 0.7) < 0.02                     # 70 % continue
    nb = np.array([r.n_bytes for r in reqs])
    assert nb.min() >= 1024 and nb.max() <= 1 << 26
    # log-uniform: median near 2^18 bytes
    assert 2 ** 17.5 < np.median(nb) < 2 ** 18.5
    # a stream's key/IV never changes
    seen = {}
    for r in reqs:
        assert seen.setdefault(r.stream_id, (r.key, r.iv)) == (r.key, r.iv)


def test_lfsr_and_crc_reject_bad_arguments_on_the_host(L):
    seeds = np.ones(4, np.uint64)
    out = np.zeros(16, np.uint32)      # never written: every call below fails first
    p, o = seeds.ctypes.data, out.ctypes.data
    assert L.mickey_lfsr_generate(p, 4, 1, 1, 8, o, N.MEM_HOST, None) == N.E_ARG      # degree
    assert L.mickey_lfsr_generate(p, 4, 65, 1, 8, o, N.MEM_HOST, None) == N.E_ARG
    assert L.mickey_lfsr_generate(p, 4, 8, 0b10, 8, o, N.MEM_HOST, None) == N.E_ARG   # no a_0
    assert L.mickey_lfsr_generate(p, 4, 8, 1 << 8, 8, o, N.MEM_HOST, None) == N.E_ARG  # tap >= degree
    assert L.mickey_lfsr_generate(p, 0, 8, 1, 8, o, N.MEM_HOST, None) == N.E_ARG      # empty
    assert L.mickey_lfsr_generate(None, 4, 8, 1, 8, o, N.MEM_HOST, None) == N.E_ARG
    assert L.mickey_crc8(None, 4, 4, 7, 0, 0, o, N.MEM_HOST, None) == N.E_ARG   # data, len > 0
    assert L.mickey_crc8(p, 4, 4, 7, 0, 0, None, N.MEM_HOST, None) == N.E_ARG   # crc
    assert L.mickey_crc8(p, 4, 4, 7, 0, 0, o, 5, None) == N.E_ARG                     # mem kind
    assert L.mickey_crc8(p, 0, 4, 7, 0, 0, o, N.MEM_HOST, None) == N.OK               # nothing to do


def test_plain_c_program_compiles_and_links(L, tmp_path):
    # include/mickey.h is valid C11 and the library resolves every symbol a C
    # user needs (the program runs in the GPU tests)
    import subprocess
    exe = str(tmp_path / "generate_c")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi", "generate_c.c"), "-o", exe,
                    "-L", os.path.dirname(B.LIB), "-lmickey",
                    "-Wl,-rpath," + os.path.dirname(B.LIB)], check=True)
    assert os.path.exists(exe)


def test_ragged_host_side_errors_and_sizes(L):
    nb = np.array([0, 1, 7, 33, 8191] + [64] * 30, np.uint64)
    # no handle: rejected before any device work
    assert L.mickey_generate_ragged(None, nb.ctypes.data, ctypes.c_void_p(16), None,
                                    N.LAYOUT_BYTES) == N.E_ARG
    assert L.mickey_last_error() == N.E_ARG
    # packed sizes: rows back to back, or the groups' word arrays
    assert L.mickey_ragged_output_bytes(nb.size, nb.ctypes.data, N.LAYOUT_BYTES) == \
        int(((nb + 7) // 8).sum())
    assert L.mickey_ragged_output_bytes(nb.size, nb.ctypes.data, N.LAYOUT_BITSLICED_U32) == \
        4 * (8191 + 64)
    assert L.mickey_ragged_output_bytes(nb.size, nb.ctypes.data, N.LAYOUT_U32) == 0
    w = np.array([32, 0, 64], np.uint64)
    assert L.mickey_ragged_output_bytes(3, w.ctypes.data, N.LAYOUT_U32) == 12
    assert L.mickey_ragged_output_bytes(3, w.ctypes.data, N.LAYOUT_U32_F32) == 0
    assert L.mickey_ragged_output_bytes(3, None, N.LAYOUT_BYTES) == 0
    # a length above the per-call limit (e.g. a negative length cast to
    # uint64) is refused rather than wrapping the sum
    big = np.array([1 << 34, (1 << 34) + 1, 2**64 - 4096], np.uint64)
    assert L.mickey_ragged_output_bytes(1, big.ctypes.data, N.LAYOUT_BYTES) == (1 << 31)
    for lay in (N.LAYOUT_BYTES, N.LAYOUT_BITSLICED_U32, N.LAYOUT_U32):
        assert L.mickey_ragged_output_bytes(3, big.ctypes.data, lay) == 0


def test_packed_offsets_match_library_sizes(L):
    from paper_1909_04750_gb300.streams import packed_offsets
    rng = np.random.default_rng(4)
    nb = rng.integers(0, 5000, 77).astype(np.uint64)
    for lay in (N.LAYOUT_BYTES, N.LAYOUT_BITSLICED_U32):
        offs = packed_offsets(nb, lay)
        total = L.mickey_ragged_output_bytes(nb.size, nb.ctypes.data, lay)
        if lay == N.LAYOUT_BYTES:
            assert offs[-1] + (nb[-1] + 7) // 8 == total
        else:
            last = 4 * int(nb[64:].max())
            assert int(offs[-1]) + last == total


def test_grain_ops_per_clock(L):
    # output 10 (the 5-input filter as H0 + b63 H1 with H0, H1 of LFSR bits:
    # 5, then b63 H1 and the 7 NFSR taps: 5), LFSR 3 (6 taps), NFSR 23 (12
    # linear terms, 11 products); an init clock adds z once more
    assert L.grain_ops_per_clock(0) == 36
    assert L.grain_ops_per_clock(1) == 37
    assert not L.grain_init_streams(None, None, 4, N.MEM_HOST, None)
    assert L.mickey_last_error() == N.E_ARG
