"""Bitsliced LFSRs and CRC-8 on the GPU against the scalar oracle, bit for
bit: every instance / message of small cases that span several groups and
tiles with ragged tails, host and device inputs, unaligned messages, and
sampled messages of the full-size CRC workload."""
import os

import numpy as np
import pytest

from oracle import lfsr as olfsr
from paper_1909_04750_gb300 import _native as N

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


def _taps(rng, d):
    t = int(rng.integers(0, 1 << min(d, 62))) | 1
    return t & ((1 << d) - 1)


@pytest.mark.parametrize("d", [2, 4, 5, 16, 17, 31, 32, 33, 63, 64])
def test_lfsr_every_instance(d):
    from paper_1909_04750_gb300.lfsr import lfsr_generate, unbitslice
    rng = np.random.default_rng(d)
    n = 70                                              # 3 groups, ragged
    seeds = rng.integers(1, 1 << 62, n, dtype=np.uint64) & np.uint64((1 << d) - 1 if d < 64
                                                                      else (1 << 64) - 1)
    seeds[0] = 1
    taps = _taps(rng, d)
    for n_bits in (1, d - 1, d, d + 1, 3 * 64 + 7):
        if n_bits < 1:
            continue
        got = unbitslice(lfsr_generate(seeds, d, taps, n_bits).cpu().numpy(), n)
        for i in range(n):
            ref = olfsr.lfsr_bits(int(seeds[i]), d, taps, n_bits)
            assert np.array_equal(got[i], ref), (d, n_bits, i)


def _sparse_taps(rng, d, k):
    # a_0 = 1 plus k - 1 other distinct positions below d
    others = rng.choice(np.arange(1, d), size=k - 1, replace=False) if k > 1 else []
    t = 1
    for j in others:
        t |= 1 << int(j)
    return t


@pytest.mark.parametrize("d", [2, 5, 17, 33, 63, 64])
def test_lfsr_sparse_and_dense_taps_every_instance(d, monkeypatch):
    # up to 16 taps take the shared-memory kernel, more the mask kernel;
    # lengths span several 64-clock blocks and a ragged remainder, and the
    # same taps forced through the mask kernel give the same words
    from paper_1909_04750_gb300.lfsr import lfsr_generate, unbitslice
    rng = np.random.default_rng(100 + d)
    n = 45
    seeds = rng.integers(1, 1 << 62, n, dtype=np.uint64) & np.uint64((1 << d) - 1 if d < 64
                                                                      else (1 << 64) - 1)
    tap_sets = [_sparse_taps(rng, d, k) for k in sorted({1, 2, min(4, d), min(16, d),
                                                          min(17, d), d})]
    # low taps (newest tap at least 8 below the degree): the batched clocks
    tap_sets += [t & ((1 << d) - 1) for t in (0b11011, 0b1000_0101, 0b11)] if d >= 16 else []
    for taps in tap_sets:
        for n_bits in (d + 1, 64 + d - 1, 5 * 64 + d + 13):
            words = lfsr_generate(seeds, d, taps, n_bits)
            got = unbitslice(words.cpu().numpy(), n)
            for i in range(n):
                ref = olfsr.lfsr_bits(int(seeds[i]), d, taps, n_bits)
                assert np.array_equal(got[i], ref), (d, hex(taps), n_bits, i)
            for env in ("MICKEY_LFSR_DENSE", "MICKEY_LFSR_NOBATCH"):
                monkeypatch.setenv(env, "1")
                other = lfsr_generate(seeds, d, taps, n_bits)
                monkeypatch.delenv(env)
                assert torch.equal(words, other), (env, d, hex(taps), n_bits)


def test_lfsr_device_seeds_and_lane_padding():
    from paper_1909_04750_gb300.lfsr import lfsr_generate
    rng = np.random.default_rng(1)
    seeds = rng.integers(1, 1 << 40, 33, dtype=np.uint64)
    a = lfsr_generate(seeds, 40, 0b1000_0000_0000_0000_0000_0000_0000_0000_0000_0111, 500)
    b = lfsr_generate(torch.from_numpy(seeds.view(np.int64)).cuda(), 40,
                      0b1000_0000_0000_0000_0000_0000_0000_0000_0000_0111, 500)
    assert torch.equal(a, b)
    # lanes past the last instance stay zero
    assert int((a[:, 1].cpu().numpy().view(np.uint32) >> 1).max()) == 0


@pytest.mark.parametrize("ln", [0, 1, 7, 15, 16, 31, 32, 33, 100, 512, 1024, 1536])
def test_crc8_every_message(ln):
    from paper_1909_04750_gb300.lfsr import crc8
    rng = np.random.default_rng(ln)
    n = 5000                                            # 3 tiles of 2048, ragged
    data = rng.integers(0, 256, (n, ln), dtype=np.uint8)
    # 0x4D has no compile-time kernel: the run-time-mask form
    for poly, init, xorout in ((0x07, 0, 0), (0x1D, 0xFF, 0xFF), (0x2F, 0xFF, 0xFF),
                               (0x9B, 0x5A, 0x00), (0x4D, 0x00, 0xFF)):
        ref = olfsr.crc8_batch(data, poly, init, xorout, threads=THREADS)
        dev = crc8(torch.from_numpy(data).cuda(), poly, init, xorout).cpu().numpy()
        assert np.array_equal(dev, ref), (ln, hex(poly))
        host = crc8(data, poly, init, xorout)
        assert np.array_equal(host, ref), (ln, hex(poly))


def test_crc8_unaligned_messages():
    from paper_1909_04750_gb300.lfsr import crc8
    rng = np.random.default_rng(11)
    buf = torch.from_numpy(rng.integers(0, 256, 300 * 64 + 1, dtype=np.uint8)).cuda()
    data = buf[1:].view(300, 64)                        # 1-byte offset: no 16-byte loads
    ref = olfsr.crc8_batch(data.cpu().numpy(), 0x07)
    assert np.array_equal(crc8(data, 0x07).cpu().numpy(), ref)


def test_crc8_full_size_sampled():
    # the measured workload: 2^20 messages of 1 KiB
    from paper_1909_04750_gb300.lfsr import crc8
    n, ln = 1 << 20, 1024
    g = torch.Generator(device="cuda").manual_seed(5)
    data = torch.randint(0, 256, (n, ln), dtype=torch.uint8, device="cuda", generator=g)
    got = crc8(data, 0x1D, 0xFF, 0xFF).cpu().numpy()
    rng = np.random.default_rng(2)
    pick = np.unique(np.concatenate([[0, 1, 2047, 2048, n - 1], rng.integers(0, n, 4096)]))
    rows = data[torch.from_numpy(pick).cuda()].cpu().numpy()
    ref = olfsr.crc8_batch(rows, 0x1D, 0xFF, 0xFF, threads=THREADS)
    assert np.array_equal(got[pick], ref)


def test_lfsr_full_size_sampled(monkeypatch):
    # the measured workload: 2^20 LFSRs of degree 64 with the taps of
    # x^64 + x^4 + x^3 + x + 1, 4096 bits each, through the few-tap kernel
    # (checked on sampled instances) and the mask kernel (same words)
    from paper_1909_04750_gb300.lfsr import lfsr_generate
    n, nb, d, taps = 1 << 20, 4096, 64, 0b11011
    g = torch.Generator(device="cuda").manual_seed(5)
    seeds = torch.randint(1, 1 << 62, (n,), dtype=torch.int64, device="cuda", generator=g)
    words = lfsr_generate(seeds, d, taps, nb)
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([[0, 31, 32, n - 1], rng.integers(0, n, 64)]))
    sd = seeds.cpu().numpy().view(np.uint64)
    w = words.cpu().numpy().view(np.uint32)                 # [nb, G]
    for i in pick:
        got = ((w[:, i // 32] >> np.uint32(i % 32)) & 1).astype(np.uint8)
        assert np.array_equal(got, olfsr.lfsr_bits(int(sd[i]), d, taps, nb)), int(i)
    monkeypatch.setenv("MICKEY_LFSR_DENSE", "1")
    assert torch.equal(words, lfsr_generate(seeds, d, taps, nb))
