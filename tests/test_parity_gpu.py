"""GPU parity: the CUDA path through the C ABI against the scalar oracle.

The cipher is deterministic, so every comparison is exact (tolerance 0).
Small cases are compared on every instance and bit; the full-size workloads
(2^20 x 2^14 and 2^24 x 2^12 bits) are compared on sampled instances that
always include the first and the last group, plus properties checked on the
whole output.
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


def _ref(s, n_bits):
    return oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, n_bits, threads=THREADS)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _first_diff(a, b):
    rows = np.nonzero(np.any(a != b, axis=tuple(range(1, a.ndim))))[0]
    return None if rows.size == 0 else int(rows[0])


# -------------------------------------------------------------- plain, small

def test_plain_small_bitsliced_full():
    s = workloads.plain_small()
    ref = _ref(s, 65536)
    st = _streams(s)
    got = _u32(st.generate(65536, "bitsliced"))
    st.sync()
    assert _first_diff(got, oracle.to_bitsliced(ref, 65536)) is None


def test_plain_small_bytes_full():
    s = workloads.plain_small()
    ref = _ref(s, 65536)
    st = _streams(s)
    got = st.generate(65536, "bytes").cpu().numpy()
    st.sync()
    assert _first_diff(got, ref) is None


@pytest.mark.parametrize("n,n_bits", [(1, 8), (1, 40), (33, 96), (45, 77), (64, 1000),
                                      (100, 4096), (31, 33)])
def test_ragged_sizes_all_layouts(n, n_bits):
    s = workloads.plain_scale(n)
    ref = _ref(s, n_bits)
    st = _streams(s)
    got = _u32(st.generate(n_bits, "bitsliced"))
    assert _first_diff(got, oracle.to_bitsliced(ref, n_bits)) is None
    st.reset(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    got = st.generate(n_bits, "bytes").cpu().numpy()
    assert _first_diff(got, ref) is None
    if n_bits % 32 == 0:
        st.reset(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
        u = _u32(st.generate(n_bits, "u32"))
        assert _first_diff(u, oracle.to_u32(ref, n_bits)) is None
        st.reset(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
        both = st.generate(n_bits, "u32_f32").cpu().numpy()
        assert _first_diff(both[0].view(np.uint32), oracle.to_u32(ref, n_bits)) is None
        f = both[1].view(np.float32)
        assert np.array_equal(f, oracle.to_f32(oracle.to_u32(ref, n_bits)))
    st.sync()


def test_mixed_iv_lengths_in_one_group():
    # every IV length 0..80 appears, many inside the same 32-lane groups
    s = workloads.batched(162)
    s.iv_lens[:] = np.arange(162) % 81
    ref = _ref(s, 512)
    st = _streams(s)
    got = st.generate(512, "bytes").cpu().numpy()
    st.sync()
    assert _first_diff(got, ref) is None


def test_batched_workload_iv_lengths_sampled():
    s = workloads.batched(4096)
    ref = _ref(s, 256)
    st = _streams(s)
    got = st.generate(256, "bytes").cpu().numpy()
    st.sync()
    assert _first_diff(got, ref) is None


def test_host_input_path():
    from paper_1909_04750_gb300.streams import Streams
    s = workloads.batched(70)
    st = Streams(s.keys, s.ivs, s.iv_lens)   # numpy: host-memory inputs
    got = st.generate(200, "bytes").cpu().numpy()
    st.sync()
    assert _first_diff(got, _ref(s, 200)) is None


# -------------------------------------------------------------- continuation

def test_resume_split_equals_contiguous():
    s = workloads.plain_scale(70)
    st = _streams(s)
    a = _u32(st.generate(137, "bitsliced"))
    b = _u32(st.generate(1000, "bitsliced"))
    c = _u32(st.generate(32, "bitsliced"))
    st.sync()
    assert st.position(0) == 1169
    whole = oracle.to_bitsliced(_ref(s, 1169), 1169)
    assert np.array_equal(np.concatenate([a, b, c], axis=1), whole)


def test_export_import_resume():
    from paper_1909_04750_gb300.streams import Streams
    s = workloads.plain_scale(50)
    st = _streams(s)
    first = st.generate(64, "bytes").cpu().numpy()
    states, pos = st.export_state()
    assert np.all(pos == 64)
    st2 = Streams.import_state(states, pos)
    rest = st2.generate(192, "bytes").cpu().numpy()
    st2.sync()
    assert st2.position(49) == 256
    assert np.array_equal(np.concatenate([first, rest], axis=1), _ref(s, 256))


def test_export_state_matches_oracle_state():
    s = workloads.plain_scale(40)
    st = _streams(s)
    st.generate(77, "bitsliced")
    states, _ = st.export_state()
    for i in (0, 17, 39):
        ost = oracle.init(s.keys[i].tobytes(), s.ivs[i].tobytes(), int(s.iv_lens[i]))
        oracle.keystream_from(ost, 77)
        r, sb = ost.bits()
        rec = np.concatenate([np.packbits(r), np.packbits(sb)])
        assert np.array_equal(states[i], rec)


def test_generate_host_matches_device():
    s = workloads.plain_scale(96)
    st = _streams(s)
    dev = _u32(st.generate(2048, "bitsliced"))
    host = st.generate_host(4096, "bytes").numpy()
    host_u = st.generate_host(1024, "u32_f32").numpy()
    st.sync()
    ref = _ref(s, 2048 + 4096 + 1024)
    assert np.array_equal(dev, oracle.to_bitsliced(ref, 2048 + 4096 + 1024)[:, :2048])
    assert np.array_equal(host, ref[:, 256:768])
    u = oracle.to_u32(ref[:, 768:], 1024)
    assert np.array_equal(host_u[0].view(np.uint32), u)
    assert np.array_equal(host_u[1].view(np.float32), oracle.to_f32(u))


# -------------------------------------------------------------- lanes

def test_lane_independence():
    s = workloads.plain_scale(64)
    base = _streams(s).generate(512, "bytes").cpu().numpy()
    k2 = s.keys.copy()
    k2[37, 3] ^= 0x10
    s2 = workloads.StreamSet("x", 0, k2, s.ivs, s.iv_lens, s.n_bits)
    other = _streams(s2).generate(512, "bytes").cpu().numpy()
    changed = np.nonzero(np.any(base != other, axis=1))[0]
    assert changed.tolist() == [37]


def test_rejected_calls_leave_the_streams_untouched():
    # host-side argument errors (no bits, a 32-bit layout that cannot hold
    # n_bits, an unknown layout) return before any launch: positions stay,
    # and the next call continues exactly where the streams stood
    import ctypes
    s = workloads.plain_scale(40)
    st = _streams(s)
    first = st.generate(64, "bytes").cpu().numpy()
    L = N.lib()
    buf = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert L.mickey_generate(st._h, 0, p, N.LAYOUT_BYTES) == N.E_ARG
    assert L.mickey_generate(st._h, 40, p, N.LAYOUT_U32) == N.E_LAYOUT
    assert L.mickey_generate(st._h, 64, p, 7) == N.E_LAYOUT
    assert st.position(0) == 64
    rest = st.generate(64, "bytes").cpu().numpy()
    st.sync()
    ref = _ref(s, 128)
    assert np.array_equal(first, ref[:, :8]) and np.array_equal(rest, ref[:, 8:16])


def test_device_iv_len_above_80_reported():
    from paper_1909_04750_gb300.streams import Streams
    s = workloads.plain_scale(40)
    lens = torch.full((40,), 80, dtype=torch.int32, device="cuda")
    lens[5] = 81
    st = Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda(), lens)
    with pytest.raises(N.MickeyError) as ei:
        st.sync()
    assert ei.value.code == N.E_IVLEN
    st.sync()  # the flag is cleared once reported


def test_limit_2_pow_40_enforced():
    from paper_1909_04750_gb300.streams import Streams
    s = workloads.plain_scale(32)
    st = _streams(s)
    states, _ = st.export_state()
    near = Streams.import_state(states, np.full(32, (1 << 40) - 64, np.uint64))
    near.generate(64, "bitsliced")
    with pytest.raises(N.MickeyError) as ei:
        near.generate(32, "bitsliced")
    assert ei.value.code == N.E_LIMIT


def test_positions_after_uniform_and_ragged_calls():
    # a call that continues every stream by the same count moves one common
    # position; ragged calls and imports move single streams; the limit
    # check and every report see their sum
    import ctypes
    from paper_1909_04750_gb300.streams import Streams
    s = workloads.plain_scale(70)
    st = _streams(s)
    st.generate(64, "bytes")
    lens = np.arange(70, dtype=np.uint64) * 3
    st.generate_ragged(lens, "bytes")
    last = st.generate(32, "bytes").cpu().numpy()
    st.sync()
    assert [st.position(i) for i in (0, 1, 69)] == [96, 99, 96 + 207]
    states, pos = st.export_state()
    assert np.array_equal(pos, 96 + lens)
    ref = oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, 96 + lens,
                                                threads=THREADS)
    for i in (0, 1, 33, 69):
        bits = np.unpackbits(np.asarray(ref[i], np.uint8))[64 + int(lens[i]):96 + int(lens[i])]
        assert np.array_equal(np.packbits(bits), last[i]), i
    # near the 2^40 limit, with stream 5 furthest: a uniform call that only
    # stream 5 cannot take is refused and names it; one that fits goes
    far = np.full(70, (1 << 40) - 1000, np.uint64)
    far[5] = (1 << 40) - 40
    near = Streams.import_state(states, far)
    with pytest.raises(N.MickeyError) as ei:
        near.generate(64, "bitsliced")
    assert ei.value.code == N.E_LIMIT and "stream 5 " in ei.value.message
    near.generate(32, "bitsliced")
    near.sync()
    assert near.position(5) == (1 << 40) - 8 and near.position(0) == (1 << 40) - 968
    L = N.lib()
    buf = torch.empty(1 << 12, dtype=torch.uint8, device="cuda")
    rc = L.mickey_generate(near._h, (1 << 64) - 1, ctypes.c_void_p(buf.data_ptr()),
                           N.LAYOUT_BYTES)
    assert rc == N.E_LIMIT and near.position(5) == (1 << 40) - 8
    # a re-key starts every stream at 0 again
    st.reset(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda(),
             torch.from_numpy(s.iv_lens.astype(np.int32)).cuda())
    assert all(st.position(i) == 0 for i in (0, 5, 69))
    again = st.generate(64, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(again, _ref(s, 64))


# -------------------------------------------------------------- full size

def _sample_rows(n, k, seed):
    rng = np.random.default_rng(seed)
    pick = set(range(32)) | set(range(n - 32, n)) | set(rng.integers(0, n, k).tolist())
    return np.array(sorted(pick))


def test_plain_scale_full_size_sampled():
    # in the launch configurations bench.py times: the autotuner's choice
    # for this shape, per layout
    from paper_1909_04750_gb300 import autotune
    s = workloads.plain_scale()
    n_bits = int(s.n_bits[0])
    st = _streams(s)
    autotune.tune(st, n_bits, N.LAYOUT_BYTES)
    autotune.tune(st, n_bits, N.LAYOUT_BITSLICED_U32)
    assert st.position(0) == 0
    out = st.generate(n_bits, "bytes")
    st.reset(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    bs = st.generate(n_bits, "bitsliced")
    st.sync()
    rows = _sample_rows(s.n, 4096, 11)
    sub = s.subset(rows)
    ref = _ref(sub, n_bits)
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert _first_diff(got, ref) is None
    # bitsliced layout: the sampled instances' lanes of their groups
    groups = np.unique(rows // 32)
    gbs = _u32(bs[torch.from_numpy(groups).cuda()])
    for r in rows[:: max(1, len(rows) // 64)]:
        gi = int(np.searchsorted(groups, r // 32))
        lane = ((gbs[gi] >> np.uint32(r % 32)) & 1).astype(np.uint8)
        assert np.array_equal(np.packbits(lane), ref[np.searchsorted(rows, r)])
    # whole-output property: both layouts hold the same number of ones
    ones_bytes = int(torch.bitwise_count(out.view(torch.int32)).sum()) if hasattr(
        torch, "bitwise_count") else None
    if ones_bytes is not None:
        assert ones_bytes == int(torch.bitwise_count(bs).sum())
    del out, bs
    torch.cuda.empty_cache()


def test_fused_full_size_sampled():
    from paper_1909_04750_gb300 import autotune
    s = workloads.fused()
    n_bits = int(s.n_bits[0])
    st = _streams(s)
    autotune.tune(st, n_bits, N.LAYOUT_U32_F32)     # the launch bench_fused times
    both = st.generate(n_bits, "u32_f32")
    st.sync()
    u = both[0]
    f = both[1].view(torch.float32)
    # property on every output word: f == (u >> 8) * 2^-24, exactly
    chk = (u.view(torch.int32) >> 8) & 0xFFFFFF
    assert bool(torch.equal(chk.to(torch.float32) * (2.0 ** -24), f))
    rows = _sample_rows(s.n, 4096, 13)
    ref = oracle.to_u32(_ref(s.subset(rows), n_bits), n_bits)
    got = u[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint32)
    assert _first_diff(got, ref) is None
    del both, u, f, chk
    torch.cuda.empty_cache()


# -------------------------------------------------------------- persistent mode

@pytest.mark.parametrize("mode", ["persistent", "persistent2"])
@pytest.mark.parametrize("stage", ["0", "1"])
@pytest.mark.parametrize("n,n_bits,blocks", [(10 * 1024, 1000, 1), (7 * 1024 + 5, 4096, 1),
                                             (41 * 1024 - 3, 776, 2), (20 * 1024, 64, 3),
                                             (10 * 1024, 4096, 3), (41 * 1024 - 3, 1024, 2)])
def test_persistent_mode_matches_grid_and_oracle(monkeypatch, n, n_bits, blocks, stage, mode):
    # The work line is cut into 4*blocks (persistent2: 8*blocks) equal
    # segments, so warp-groups are split into head and tail pieces run by
    # different warps.
    s = workloads.plain_scale(n)
    monkeypatch.setenv("MICKEY_STAGE", stage)
    monkeypatch.setenv("MICKEY_MODE", "grid")
    st_g = _streams(s)
    monkeypatch.setenv("MICKEY_MODE", mode)
    monkeypatch.setenv("MICKEY_PERSIST_BLOCKS", str(blocks))
    st_p = _streams(s)
    got = {}
    for layout in ("bytes", "bitsliced", "u32_f32"):
        if layout == "u32_f32" and n_bits % 32:
            continue
        a = st_g.generate(n_bits, layout).cpu().numpy()
        b = st_p.generate(n_bits, layout).cpu().numpy()
        st_p.sync()
        assert np.array_equal(a, b), layout
        got[layout] = b
    # the second call continued every stream: check sampled rows bit-exactly
    rows = _sample_rows(n, 64, 5)
    ref = _ref(s.subset(rows), 3 * n_bits)
    bits = oracle.bits_of(ref, 3 * n_bits)[:, n_bits:2 * n_bits]
    bs = got["bitsliced"]
    for k, r in enumerate(rows):
        lane = ((bs[r // 32].view(np.uint32) >> np.uint32(r % 32)) & 1).astype(np.uint8)
        assert np.array_equal(lane, bits[k]), int(r)
    assert np.array_equal(got["bytes"][rows], ref[:, : (n_bits + 7) // 8]) or n_bits % 8
    if "u32_f32" in got:
        u = oracle.to_u32(ref[:, 2 * n_bits // 8:], n_bits)
        assert np.array_equal(got["u32_f32"][0][rows].view(np.uint32), u)
        assert np.array_equal(got["u32_f32"][1][rows].view(np.float32), oracle.to_f32(u))


@pytest.mark.parametrize("n,n_bits", [(5 * 1024 - 7, 1000), (33, 4096), (300 * 1024, 256)])
def test_paired_kernel_with_few_warp_groups_matches_grid(monkeypatch, n, n_bits):
    # fewer warp-groups than clock warps: each clock/emission pair takes a
    # whole warp-group (no segments, no hand-off); compared with the grid
    # kernel word for word and with the oracle on sampled rows
    s = workloads.plain_scale(n)
    monkeypatch.setenv("MICKEY_MODE", "grid")
    st_g = _streams(s)
    monkeypatch.setenv("MICKEY_MODE", "persistent")
    st_p = _streams(s)
    for layout in ("bytes", "bitsliced", "u32_f32"):
        if layout == "u32_f32" and n_bits % 32:
            continue
        a = st_g.generate(n_bits, layout).cpu().numpy()
        b = st_p.generate(n_bits, layout).cpu().numpy()
        st_p.sync()
        assert np.array_equal(a, b), layout
    calls = 2 + (n_bits % 32 == 0)             # generate calls made so far
    rows = _sample_rows(n, 48, 17)
    ref = _ref(s.subset(rows), (calls + 1) * n_bits)
    last = st_p.generate(n_bits, "bytes").cpu().numpy()
    st_p.sync()
    assert np.array_equal(last[rows], ref[:, calls * n_bits // 8:])


def test_autotune_keeps_positions_and_output():
    from paper_1909_04750_gb300 import autotune
    s = workloads.plain_scale(24 * 1024)
    st = _streams(s)
    first = st.generate(256, "bytes").cpu().numpy()
    entry = autotune.tune(st, 1024, N.LAYOUT_BYTES, refresh=True)
    assert entry["candidates"] and entry["unroll"] in (2, 4)
    assert st.position(0) == 256          # tuning restored the state
    rest = st.generate(1024, "bytes").cpu().numpy()
    st.sync()
    rows = _sample_rows(s.n, 64, 3)
    ref = _ref(s.subset(rows), 1280)
    assert np.array_equal(first[rows], ref[:, :32])
    assert np.array_equal(rest[rows], ref[:, 32:])


def test_persistent_wait_runs_out_without_a_fault(monkeypatch):
    # the hand-off wait of a tail piece is bounded: with the test hook no
    # head publishes the value the tails wait for, so every tail gives up
    # after MICKEY_SPIN_LIMIT polls, the call still returns, mickey_sync
    # reports the timeout, and the context keeps working
    s = workloads.plain_scale(10 * 1024)
    monkeypatch.setenv("MICKEY_MODE", "persistent")
    monkeypatch.setenv("MICKEY_PERSIST_BLOCKS", "1")
    monkeypatch.setenv("MICKEY_SPIN_LIMIT", "2000")
    monkeypatch.setenv("MICKEY_TEST_UNPUBLISHED", "1")
    st = _streams(s)
    st.generate(1000, "bytes")
    with pytest.raises(N.MickeyError) as ei:
        st.sync()
    assert ei.value.code == N.E_TIMEOUT
    st.free()
    monkeypatch.delenv("MICKEY_TEST_UNPUBLISHED")
    ok = _streams(s)
    got = ok.generate(1000, "bytes").cpu().numpy()
    ok.sync()
    rows = _sample_rows(s.n, 48, 6)
    assert np.array_equal(got[rows], _ref(s.subset(rows), 1000)[:, :125])


def test_plain_c_program_through_the_abi(tmp_path):
    # a C user of include/mickey.h, built with gcc against the in-tree
    # library, generates the 32-instance workload into host memory
    import subprocess
    from paper_1909_04750_gb300 import build as B
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "generate_c")
    subprocess.run(["gcc", "-std=c11", "-O1", "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "c_abi", "generate_c.c"), "-o", exe,
                    "-L", os.path.dirname(B.LIB), "-lmickey",
                    "-Wl,-rpath," + os.path.dirname(B.LIB)], check=True)
    s = workloads.plain_small()
    (tmp_path / "in.bin").write_bytes(s.keys.tobytes() + s.ivs.tobytes())
    n_bits = 4096 + 13                                   # ragged last byte
    subprocess.run([exe, str(tmp_path / "in.bin"), str(s.n), str(n_bits),
                    str(tmp_path / "out.bin")], check=True)
    got = np.frombuffer((tmp_path / "out.bin").read_bytes(), np.uint8).reshape(s.n, -1)
    assert np.array_equal(got, _ref(s, n_bits))


# -------------------------------------------------------------- roofline probes

def test_roofline_probes_stay_below_the_lop3_rate():
    # the LOP3 probe measures the denominator (64 per SM per clock); the bare
    # keystream clock (327 algorithmic ops per group-clock) can come close to
    # it but not above, else the op count or the probe would be wrong
    import ctypes
    L = N.lib()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    N.check(L.mickey_probe_lop3(1, 128, 2000, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    assert 56.0 < a.value <= 64.5, a.value
    for bps in (1, 2):
        x, mhz = ctypes.c_double(), ctypes.c_double()
        N.check(L.mickey_probe_clock(bps, 1024, ctypes.byref(x), ctypes.byref(mhz)))
        assert 40.0 < x.value <= 64.5, (bps, x.value)
        assert 500.0 < mhz.value < 2200.0, mhz.value


@pytest.mark.parametrize("mode,depth", [("grid", 2), ("grid", 4), ("persistent", 2),
                                        ("persistent", 4), ("persistent", 8),
                                        ("persistent2", 4)])
@pytest.mark.parametrize("n,n_bits", [(10 * 1024 + 7, 1024), (41 * 1024 - 3, 2048),
                                      (3000, 768)])
def test_output_tile_depths_match_direct_and_oracle(n, n_bits, mode, depth):
    # rows staged `depth` tiles deep (the autotuner's output-tile axis) give
    # the same bytes as direct row stores, and the oracle's on sampled rows
    modes = {"grid": N.MODE_GRID, "persistent": N.MODE_PERSISTENT,
             "persistent2": N.MODE_PERSISTENT2}
    s = workloads.plain_scale(n)
    L = N.lib()
    st_d, st_s = _streams(s), _streams(s)
    for layout in (N.LAYOUT_BYTES, N.LAYOUT_U32_F32):
        N.check(L.mickey_set_config(st_d._h, layout, N.MODE_GRID, 4, 0))
        N.check(L.mickey_set_config(st_s._h, layout, modes[mode], 4, depth))
    a = st_d.generate(n_bits, "bytes").cpu().numpy()
    b = st_s.generate(n_bits, "bytes").cpu().numpy()
    c = st_d.generate(n_bits, "u32_f32").cpu().numpy()
    d = st_s.generate(n_bits, "u32_f32").cpu().numpy()
    st_s.sync()
    assert np.array_equal(a, b) and np.array_equal(c, d)
    rows = _sample_rows(n, 64, 9)
    ref = _ref(s.subset(rows), 2 * n_bits)
    assert np.array_equal(b[rows], ref[:, : n_bits // 8])
    assert np.array_equal(d[0][rows].view(np.uint32), oracle.to_u32(ref[:, n_bits // 8:], n_bits))
