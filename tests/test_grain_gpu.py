"""Bitsliced Grain through the C ABI against the scalar Grain oracle
(exact comparison: the cipher is deterministic)."""
import os

import numpy as np
import pytest

from oracle import grain as og
from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04750_gb300 import build as B
    B.build()
    N.lib()


def _gs(s):
    from paper_1909_04750_gb300.grain import GrainStreams
    return GrainStreams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())


@pytest.mark.parametrize("n,n_bits", [(1000, 3000), (3 * 1024 + 17, 2560), (2100, 1281),
                                      (64, 6000)])
def test_queue_fed_launch_every_instance(monkeypatch, n, n_bits):
    # the persistent launch with (warp-group, chunk) items, forced for a few
    # warp-groups: every chunk after the first waits for its predecessor
    monkeypatch.setenv("MICKEY_GRAIN_QUEUE", "1")
    s = workloads.grain_streams(n, seed=16)
    ref = og.batch_bytes(s.keys, s.ivs, n_bits, threads=THREADS)
    st = _gs(s)
    got = st.generate(n_bits, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, ref)
    st2 = _gs(s)
    words = st2.generate(n_bits, "bitsliced").cpu().numpy().view(np.uint32)
    st2.sync()
    assert np.array_equal(words, og.to_bitsliced(ref, n_bits))


@pytest.mark.parametrize("n,n_bits", [(1000, 3000), (9000, 1281), (64, 6000)])
def test_grid_launch_every_instance(monkeypatch, n, n_bits):
    # one warp per warp-group for the whole call (the default whenever the
    # warp-groups fit), also with the override set to it
    monkeypatch.setenv("MICKEY_GRAIN_QUEUE", "0")
    s = workloads.grain_streams(n, seed=17)
    ref = og.batch_bytes(s.keys, s.ivs, n_bits, threads=THREADS)
    st = _gs(s)
    got = st.generate(n_bits, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, ref)
    st2 = _gs(s)
    words = st2.generate(n_bits, "bitsliced").cpu().numpy().view(np.uint32)
    st2.sync()
    assert np.array_equal(words, og.to_bitsliced(ref, n_bits))


@pytest.mark.parametrize("layout", ["bytes", "bitsliced"])
def test_queue_wait_runs_out_without_a_fault(monkeypatch, layout):
    # the wait of a chunk for its predecessor is bounded: with one poll of
    # about 256 ns allowed, every chunk after the first gives up long before
    # its predecessor (about 1280 clocks) has published, the call still
    # returns, grain_sync reports the timeout, and the context keeps working
    # (the bytes layout's blocks also free their tensor memory)
    monkeypatch.setenv("MICKEY_GRAIN_QUEUE", "1")
    monkeypatch.setenv("MICKEY_SPIN_LIMIT", "1")
    s = workloads.grain_streams(3 * 1024 + 17, seed=18)
    st = _gs(s)
    st.generate(6000, layout)
    with pytest.raises(N.MickeyError) as ei:
        st.sync()
    assert ei.value.code == N.E_TIMEOUT
    monkeypatch.delenv("MICKEY_SPIN_LIMIT")
    ok = _gs(s)
    got = ok.generate(6000, "bytes").cpu().numpy()
    ok.sync()
    assert np.array_equal(got, og.batch_bytes(s.keys, s.ivs, 6000, threads=THREADS))


def test_known_answer_vectors_on_the_gpu():
    from paper_1909_04750_gb300.grain import GrainStreams
    rows = [l.split() for l in open(os.path.join(GOLDEN, "grain_kat.txt"))
            if l.strip() and not l.startswith("#")]
    keys = np.array([list(bytes.fromhex(k)) for k, _, _ in rows], np.uint8)
    ivs = np.array([list(bytes.fromhex(v)) for _, v, _ in rows], np.uint8)
    st = GrainStreams(keys, ivs)                     # host inputs
    got = st.generate(80, "bytes").cpu().numpy()
    st.sync()
    for i, (_, _, z) in enumerate(rows):
        assert got[i].tobytes() == bytes.fromhex(z)


@pytest.mark.parametrize("n,n_bits", [(32, 4096), (70, 1000), (33, 161), (5, 1), (64, 7),
                                      (96, 80), (40, 159), (31, 320), (1000, 3000),
                                      (3 * 1024 + 17, 2560), (2100, 1281)])
def test_every_instance_both_layouts(n, n_bits):
    s = workloads.grain_streams(n, seed=11)
    ref = og.batch_bytes(s.keys, s.ivs, n_bits, threads=THREADS)
    st = _gs(s)
    got = st.generate(n_bits, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, ref)
    st2 = _gs(s)
    words = st2.generate(n_bits, "bitsliced").cpu().numpy().view(np.uint32)
    st2.sync()
    assert np.array_equal(words, og.to_bitsliced(ref, n_bits))


def test_continuation_and_state():
    s = workloads.grain_streams(100, seed=12)
    st = _gs(s)
    parts = [st.generate(k, "bytes").cpu().numpy() for k in (160, 37, 243, 80)]
    st.sync()
    total = 160 + 37 + 243 + 80
    ref = og.batch_bytes(s.keys, s.ivs, total, threads=THREADS)
    bits = np.concatenate([np.unpackbits(p, axis=1, bitorder="little")[:, :k]
                           for p, k in zip(parts, (160, 37, 243, 80))], axis=1)
    assert np.array_equal(np.packbits(bits, axis=1, bitorder="little"), ref)
    assert st.position() == total
    rec = st.export_state()
    for i in (0, 31, 32, 99):
        o = og.init(s.keys[i].tobytes(), s.ivs[i].tobytes())
        og.keystream_from(o, total)
        sb, bb = o.bits()
        got = np.unpackbits(rec[i], bitorder="little")
        assert np.array_equal(got[:80], sb) and np.array_equal(got[80:], bb), i


def test_bitsliced_calls_continue_and_export():
    # bitsliced calls of whole 80-clock bodies and of tails continue each
    # other exactly, and the state written back is the oracle's
    s = workloads.grain_streams(3 * 1024 + 17, seed=21)
    st = _gs(s)
    ks = (160, 37, 243, 80, 1000, 1, 16, 17)
    parts = [st.generate(k, "bitsliced").cpu().numpy().view(np.uint32) for k in ks]
    st.sync()
    total = sum(ks)
    ref = og.batch_bytes(s.keys, s.ivs, total, threads=THREADS)
    assert np.array_equal(np.concatenate(parts, axis=1), og.to_bitsliced(ref, total))
    rec = st.export_state()
    for i in (0, 31, 32, 1500, s.n - 1):
        o = og.init(s.keys[i].tobytes(), s.ivs[i].tobytes())
        og.keystream_from(o, total)
        sb, bb = o.bits()
        got = np.unpackbits(rec[i], bitorder="little")
        assert np.array_equal(got[:80], sb) and np.array_equal(got[80:], bb), i


def test_full_size_workload_sampled():
    s = workloads.grain_streams()
    n_bits = workloads.GRAIN_SCALE["n_bits"]
    st = _gs(s)
    out = st.generate(n_bits, "bytes")
    st.sync()
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([np.arange(32), np.arange(s.n - 32, s.n),
                                    rng.choice(s.n, 960, replace=False)]))
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = og.batch_bytes(s.keys[idx], s.ivs[idx], n_bits, threads=THREADS)
    assert np.array_equal(got, ref)


def test_rejections():
    import ctypes
    s = workloads.grain_streams(40, seed=13)
    st = _gs(s)
    L = N.lib()
    out = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    assert L.grain_generate(st._h, 64, ctypes.c_void_p(out.data_ptr()), N.LAYOUT_U32) == \
        N.E_LAYOUT
    assert L.grain_generate(st._h, 0, ctypes.c_void_p(out.data_ptr()), N.LAYOUT_BYTES) == N.E_ARG
    assert st.position() == 0


def test_reset_rekeys_in_place():
    a = workloads.grain_streams(64, seed=14)
    b = workloads.grain_streams(64, seed=15)
    st = _gs(a)
    st.generate(333, "bytes")
    st.reset(b.keys, b.ivs)                          # host inputs
    assert st.position() == 0
    got = st.generate(500, "bytes").cpu().numpy()
    st.reset(torch.from_numpy(a.keys).cuda(), torch.from_numpy(a.ivs).cuda())
    again = st.generate(500, "bytes").cpu().numpy()
    st.sync()
    assert np.array_equal(got, og.batch_bytes(b.keys, b.ivs, 500, threads=THREADS))
    assert np.array_equal(again, og.batch_bytes(a.keys, a.ivs, 500, threads=THREADS))
