"""mickey_generate_ragged through the C ABI against the scalar oracle.

Every stream of a handle continues by its own number of bits in one call;
afterwards each stream's state and position must be those after exactly its
own bits, so that a following call continues it.  Lengths that end inside
the same 32-lane group at different clocks (0, 1, 7, 33, 8191, ...) are the
case the per-lane end-point snapshots exist for.  Comparisons are exact.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04750_gb300 import build as B
    B.build()
    N.lib()


def _streams(s):
    from paper_1909_04750_gb300.streams import Streams
    return Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda(),
                   torch.from_numpy(s.iv_lens.astype(np.int32)).cuda())


def _bits(s, total):
    """[n] lists of the first total[i] keystream bits (0/1 arrays)."""
    rows = oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, np.asarray(total, np.uint64),
                              threads=THREADS)
    if isinstance(rows, np.ndarray):
        rows = list(rows)
    return [np.unpackbits(np.asarray(r, np.uint8))[:int(t)] for r, t in zip(rows, total)]


def _pack(bits):
    return np.packbits(bits) if bits.size else np.zeros(0, np.uint8)


def _mixed_lengths(n, seed=3):
    """Lengths with every group holding several distinct end points: the
    first group gets 0, 1, 7, 33, 8191 and a few repeats; the rest random
    in [0, 3000] with some zeros and repeats."""
    rng = np.random.default_rng(seed)
    nb = rng.integers(0, 3000, n).astype(np.uint64)
    head = np.array([0, 1, 7, 33, 8191, 8191, 1, 0, 32, 31, 64, 65, 95, 96, 97, 8190],
                    np.uint64)
    nb[: min(n, head.size)] = head[: min(n, head.size)]
    nb[rng.integers(0, n, n // 8)] = 0
    return nb


def _rows_from(out, offs, nb):
    host = out.cpu().numpy().view(np.uint8).reshape(-1)
    return [host[int(o):int(o) + (int(b) + 7) // 8] for o, b in zip(offs, nb)]


@pytest.mark.parametrize("n", [32, 100, 161])
def test_ragged_bytes_every_stream_then_continue(n):
    s = workloads.batched(n)                 # IV lengths 0..80 mixed inside groups
    nb = _mixed_lengths(n)
    st = _streams(s)
    out, offs = st.generate_ragged(nb, "bytes")
    K = 256
    cont = st.generate(K, "bytes").cpu().numpy()
    st.sync()
    ref = _bits(s, nb + np.uint64(K))
    for i, row in enumerate(_rows_from(out, offs, nb)):
        assert np.array_equal(row, _pack(ref[i][: int(nb[i])])), i
        assert np.array_equal(cont[i], _pack(ref[i][int(nb[i]):])), i
        assert st.position(i) == int(nb[i]) + K


@pytest.mark.parametrize("layout", ["bytes", "bitsliced"])
def test_ragged_several_blocks_uneven_warp_groups(layout):
    # 386 groups in several blocks, the last one partly empty; groups whose
    # longest lanes differ widely inside a warp, every stream compared, then
    # a plain continuation
    n = 386 * 32 - 19
    s = workloads.batched(n)
    rng = np.random.default_rng(9)
    nb = rng.integers(0, 700, n).astype(np.uint64)
    nb[::97] = 2500
    nb[5 * 32:6 * 32] = 0                     # a group with nothing to do
    st = _streams(s)
    out, offs = st.generate_ragged(nb, layout)
    cont = st.generate(64, "bytes").cpu().numpy()
    host = out.cpu().numpy().view(np.uint8).reshape(-1)
    st.sync()
    ref = _bits(s, nb + np.uint64(64))
    if layout == "bytes":
        for i, row in enumerate(_rows_from(out, offs, nb)):
            assert np.array_equal(row, _pack(ref[i][: int(nb[i])])), i
    else:
        words_all = host.view(np.uint32)
        for g in range((n + 31) // 32):
            lanes = range(32 * g, min(n, 32 * g + 32))
            C = max(int(nb[i]) for i in lanes)
            words = words_all[int(offs[g]) // 4: int(offs[g]) // 4 + C]
            for i in lanes:
                got = ((words >> np.uint32(i - 32 * g)) & 1).astype(np.uint8)
                want = np.zeros(C, np.uint8)
                want[: int(nb[i])] = ref[i][: int(nb[i])]
                assert np.array_equal(got, want), (g, i)
    for i in range(n):
        assert np.array_equal(cont[i], _pack(ref[i][int(nb[i]):])), i


def test_ragged_bitsliced_every_stream():
    n = 70
    s = workloads.batched(n)
    nb = _mixed_lengths(n, seed=5)
    st = _streams(s)
    out, offs = st.generate_ragged(nb, "bitsliced")
    host = out.cpu().numpy().view(np.uint32)
    st.sync()
    ref = _bits(s, nb)
    G = (n + 31) // 32
    for g in range(G):
        lanes = range(32 * g, min(n, 32 * g + 32))
        C = max(int(nb[i]) for i in lanes)
        words = host[int(offs[g]) // 4: int(offs[g]) // 4 + C]
        for i in lanes:
            l = i - 32 * g
            got = ((words >> np.uint32(l)) & 1).astype(np.uint8)
            want = np.zeros(C, np.uint8)
            want[: int(nb[i])] = ref[i]
            assert np.array_equal(got, want), (g, l)
        for l in range(len(lanes), 32):       # padding lanes stay zero
            assert not np.any((words >> np.uint32(l)) & 1)


def test_ragged_u32_rows():
    n = 45
    s = workloads.batched(n)
    rng = np.random.default_rng(9)
    nb = (32 * rng.integers(0, 90, n)).astype(np.uint64)
    nb[:6] = [0, 32, 64, 2048, 32, 0]
    st = _streams(s)
    out, offs = st.generate_ragged(nb, "u32")
    host = out.cpu().numpy().view(np.uint8)
    st.sync()
    ref = _bits(s, nb)
    for i in range(n):
        o = int(offs[i])
        words = host[o:o + int(nb[i]) // 8].view(np.uint32)   # native words
        # word k holds z_{32k..32k+31} with z_{32k} in bit 31
        want = (np.packbits(ref[i]).view(">u4").astype(np.uint32) if nb[i]
                else np.zeros(0, np.uint32))
        assert np.array_equal(words, want), i


def test_ragged_explicit_offsets_leave_gaps_untouched():
    n = 64
    s = workloads.batched(n)
    nb = _mixed_lengths(n, seed=8)
    sizes = (nb + np.uint64(7)) // np.uint64(8)
    # unaligned rows with 3-byte gaps of a sentinel between them
    offs = np.concatenate(([1], 1 + np.cumsum(sizes[:-1] + np.uint64(3)))).astype(np.uint64)
    total = int(offs[-1] + sizes[-1] + 5)
    out = torch.full((total,), 0xA5, dtype=torch.uint8, device="cuda")
    st = _streams(s)
    st.generate_ragged(nb, "bytes", out=out, offsets=offs)
    host = out.cpu().numpy()
    st.sync()
    ref = _bits(s, nb)
    mask = np.ones(total, bool)
    for i in range(n):
        o, c = int(offs[i]), int(sizes[i])
        assert np.array_equal(host[o:o + c], _pack(ref[i])), i
        mask[o:o + c] = False
    assert np.all(host[mask] == 0xA5)


@pytest.mark.parametrize("layout,b", [("bytes", 1001), ("u32", 1024), ("bitsliced", 1001)])
@pytest.mark.parametrize("offsets", ["none", "packed", "gapped"])
def test_ragged_equal_lengths(layout, b, offsets):
    """Equal lengths: at the packed offsets the call is one keystream launch
    (the plain generate's layout); at other offsets the ragged kernel's
    all-lanes-end-together write-back.  Both against the oracle, then a
    continuation."""
    n = 100
    s = workloads.batched(n)
    nb = np.full(n, b, np.uint64)
    st = _streams(s)
    G = (n + 31) // 32
    if layout == "bitsliced":
        step, n_off = 4 * b, G
    else:
        step, n_off = (b // 8 if layout == "u32" else (b + 7) // 8), n
    gap = 16 if offsets == "gapped" else 0
    offs = np.arange(n_off, dtype=np.uint64) * np.uint64(step + gap)
    total = int(offs[-1]) + step + 16
    out = torch.full((total,), 0xA5, dtype=torch.uint8, device="cuda")
    st.generate_ragged(nb, layout, out=out, offsets=None if offsets == "none" else offs)
    K = 96
    cont = st.generate(K, "bytes").cpu().numpy()
    host = out.cpu().numpy()
    st.sync()
    ref = _bits(s, np.full(n, b + K, np.uint64))
    if layout == "bitsliced":
        for g in range(G):
            words = host[int(offs[g]):int(offs[g]) + 4 * b].view(np.uint32)
            for i in range(32 * g, min(n, 32 * g + 32)):
                got = ((words >> np.uint32(i - 32 * g)) & 1).astype(np.uint8)
                assert np.array_equal(got, ref[i][:b]), (g, i)
    else:
        for i in range(n):
            row = host[int(offs[i]):int(offs[i]) + step]
            want = _pack(ref[i][:b])
            if layout == "u32":
                want = want.view(">u4").astype(np.uint32).view(np.uint8)
            assert np.array_equal(row, want), i
    for i in range(n):
        assert np.array_equal(cont[i], _pack(ref[i][b:])), i
        assert st.position(i) == b + K
    if offsets == "gapped":                    # the gaps keep their sentinel
        mask = np.ones(total, bool)
        for k in range(n_off):
            mask[int(offs[k]):int(offs[k]) + step] = False
        assert np.all(host[mask] == 0xA5)


def test_ragged_twice_and_export_state():
    n = 96
    s = workloads.batched(n)
    a = _mixed_lengths(n, seed=1)
    b = _mixed_lengths(n, seed=2)
    st = _streams(s)
    out1, o1 = st.generate_ragged(a, "bytes")
    out2, o2 = st.generate_ragged(b, "bytes")
    states, pos = st.export_state()
    st.sync()
    ref = _bits(s, a + b)
    r1, r2 = _rows_from(out1, o1, a), _rows_from(out2, o2, b)
    for i in range(n):
        assert np.array_equal(r1[i], _pack(ref[i][: int(a[i])])), i
        assert np.array_equal(r2[i], _pack(ref[i][int(a[i]):])), i
        assert pos[i] == a[i] + b[i]
    # the exported state is the oracle's state after a[i] + b[i] bits
    for i in range(0, n, 7):
        o = oracle.init(s.keys[i].tobytes(), s.ivs[i].tobytes(), int(s.iv_lens[i]))
        oracle.keystream_from(o, int(a[i] + b[i]))
        r, s_ = o.bits()
        rec = np.unpackbits(states[i])
        assert np.array_equal(rec[:100], r) and np.array_equal(rec[104:204], s_), i


def test_ragged_all_zero_is_a_no_op():
    s = workloads.plain_scale(40)
    st = _streams(s)
    st.generate(64, "bytes")
    out = torch.full((64,), 0x5A, dtype=torch.uint8, device="cuda")
    st.generate_ragged(np.zeros(40, np.uint64), "bytes", out=out)
    cont = st.generate(64, "bytes").cpu().numpy()
    st.sync()
    assert np.all(out.cpu().numpy() == 0x5A)
    ref = oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, 128, threads=THREADS)
    assert np.array_equal(cont, ref[:, 8:])
    assert st.position(0) == 128


def test_ragged_rejections_leave_streams_untouched():
    from paper_1909_04750_gb300.streams import Streams
    import ctypes
    s = workloads.plain_scale(33)
    st = Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    L = N.lib()
    out = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(out.data_ptr())
    nb = np.full(33, 64, np.uint64)
    assert L.mickey_generate_ragged(st._h, nb.ctypes.data, p, None, N.LAYOUT_U32_F32) == \
        N.E_LAYOUT
    odd = nb.copy()
    odd[5] = 40
    assert L.mickey_generate_ragged(st._h, odd.ctypes.data, p, None, N.LAYOUT_U32) == N.E_LAYOUT
    big = nb.copy()
    big[3] = (1 << 34) + 1
    assert L.mickey_generate_ragged(st._h, big.ctypes.data, p, None, N.LAYOUT_BYTES) == N.E_ARG
    mis = ctypes.c_void_p(out.data_ptr() + 2)
    assert L.mickey_generate_ragged(st._h, nb.ctypes.data, mis, None, N.LAYOUT_U32) == N.E_ARG
    assert L.mickey_last_error() == N.E_ARG
    for i in range(33):
        assert st.position(i) == 0
    got = st.generate(96, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, 96, threads=THREADS))


def test_ragged_limit_2_pow_40():
    from paper_1909_04750_gb300.streams import Streams
    import ctypes
    s = workloads.plain_scale(32)
    st = Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    states, _ = st.export_state()
    pos = np.zeros(32, np.uint64)
    pos[4] = (1 << 40) - 10
    h = Streams.import_state(states, pos)
    out = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    nb = np.zeros(32, np.uint64)
    nb[4] = 11
    assert N.lib().mickey_generate_ragged(h._h, nb.ctypes.data, ctypes.c_void_p(out.data_ptr()),
                                          None, N.LAYOUT_BYTES) == N.E_LIMIT
    nb[4] = 10
    h.generate_ragged(nb, "bytes", out=out)
    h.sync()
    assert h.position(4) == 1 << 40
