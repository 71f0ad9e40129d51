"""The Grain oracle pinned to facts outside itself: the specification's
known-answer vectors, the primitivity of the LFSR's feedback polynomial
(read off the oracle's own clock and checked here over GF(2) against the
prime factors of 2^80 - 1), the LFSR running free of the NFSR, the NFSR
feedback taking s_i linearly, and continuation of a stream."""
import os

import numpy as np
import pytest

from oracle import grain

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# 2^80 - 1 = 3 * 5^2 * 11 * 17 * 31 * 41 * 257 * 61681 * 4278255361
ORDER = (1 << 80) - 1
PRIMES = [3, 5, 11, 17, 31, 41, 257, 61681, 4278255361]


def _is_prime(p):
    if p < 2:
        return False
    k = 2
    while k * k <= p:
        if p % k == 0:
            return False
        k += 1
    return True


def pmod(a, m):
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def pmulmod(a, b, m):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a = pmod(a << 1, m)
    return pmod(r, m)


def ppowmod(e, m):
    """x^e mod m over GF(2)."""
    r, base = 1, pmod(2, m)
    while e:
        if e & 1:
            r = pmulmod(r, base, m)
        base = pmulmod(base, base, m)
        e >>= 1
    return r


def primitive(poly):
    return ppowmod(ORDER, poly) == 1 and all(ppowmod(ORDER // q, poly) != 1 for q in PRIMES)


def _kats():
    for line in open(os.path.join(GOLDEN, "grain_kat.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v, z = line.split()
            yield bytes.fromhex(k), bytes.fromhex(v), bytes.fromhex(z)


def test_factorisation_of_the_period():
    prod = 1
    for q in PRIMES:
        assert _is_prime(q)
        prod *= q
    assert prod * 5 == ORDER            # 5 appears squared


@pytest.mark.parametrize("key,iv,z", list(_kats()))
def test_known_answer_vectors(key, iv, z):
    assert grain.stream(key, iv, 8 * len(z)) == z


def _lfsr_taps():
    """Taps j with s_{i+80} depending on s_{i+j}, read off one clock of the
    oracle from unit states (NFSR zero, nothing added)."""
    taps = []
    for j in range(80):
        s = np.zeros(80, np.uint8)
        s[j] = 1
        st = grain.State.from_bits(s, np.zeros(80, np.uint8))
        grain.clock(st, 0)
        if st.bits()[0][79]:
            taps.append(j)
    return taps


def test_lfsr_feedback_polynomial_is_primitive():
    taps = _lfsr_taps()
    # characteristic polynomial of s_{i+80} = sum_j s_{i+j}
    poly = (1 << 80) | sum(1 << j for j in taps)
    assert 0 in taps                    # the recurrence has full order
    assert primitive(poly)
    # the check has teeth: moving any single tap breaks primitivity for
    # nearly every choice
    still = 0
    for j in taps[1:]:
        for d in (-1, 1):
            k = j + d
            if 0 < k < 80 and k not in taps:
                still += primitive(poly ^ (1 << j) ^ (1 << k))
    assert still <= 2


def test_lfsr_runs_free_of_the_nfsr():
    rng = np.random.default_rng(2)
    s = rng.integers(0, 2, 80).astype(np.uint8)
    a = grain.State.from_bits(s, rng.integers(0, 2, 80).astype(np.uint8))
    b = grain.State.from_bits(s, rng.integers(0, 2, 80).astype(np.uint8))
    for _ in range(500):
        grain.clock(a, 0)
        grain.clock(b, 0)
    assert np.array_equal(a.bits()[0], b.bits()[0])


def test_nfsr_feedback_takes_s0_linearly():
    # with the NFSR zero, g vanishes: the new NFSR bit is s_i alone
    for j in range(80):
        s = np.zeros(80, np.uint8)
        s[j] = 1
        st = grain.State.from_bits(s, np.zeros(80, np.uint8))
        grain.clock(st, 0)
        assert st.bits()[1][79] == (1 if j == 0 else 0), j
    # and flipping s_0 flips the new NFSR bit whatever the NFSR holds
    rng = np.random.default_rng(3)
    for _ in range(50):
        s = rng.integers(0, 2, 80).astype(np.uint8)
        b = rng.integers(0, 2, 80).astype(np.uint8)
        s2 = s.copy()
        s2[0] ^= 1
        x, y = grain.State.from_bits(s, b), grain.State.from_bits(s2, b)
        grain.clock(x, 0)
        grain.clock(y, 0)
        assert x.bits()[1][79] != y.bits()[1][79]


def test_initialisation_adds_the_output_into_both_feedbacks():
    # a clock with the output added differs from one without in exactly the
    # two new bits
    rng = np.random.default_rng(4)
    s = rng.integers(0, 2, 80).astype(np.uint8)
    b = rng.integers(0, 2, 80).astype(np.uint8)
    x, y = grain.State.from_bits(s, b), grain.State.from_bits(s, b)
    grain.clock(x, 0)
    grain.clock(y, 1)
    xs, xb = x.bits()
    ys, yb = y.bits()
    assert np.array_equal(xs[:79], ys[:79]) and np.array_equal(xb[:79], yb[:79])
    assert xs[79] != ys[79] and xb[79] != yb[79]


def test_continuation_and_batch():
    key, iv = bytes(range(10)), bytes(range(20, 28))
    whole = grain.stream(key, iv, 1000)
    st = grain.init(key, iv)
    a = grain.keystream_from(st, 600)
    b = grain.keystream_from(st, 400)
    bits = np.concatenate([np.unpackbits(np.frombuffer(a, np.uint8), bitorder="little")[:600],
                           np.unpackbits(np.frombuffer(b, np.uint8), bitorder="little")[:400]])
    assert np.packbits(bits, bitorder="little").tobytes() == whole
    keys = np.frombuffer(bytes(range(30)), np.uint8).reshape(3, 10)
    ivs = np.frombuffer(bytes(range(100, 124)), np.uint8).reshape(3, 8)
    rows = grain.batch_bytes(keys, ivs, 77, threads=2)
    for i in range(3):
        assert rows[i].tobytes() == grain.stream(keys[i].tobytes(), ivs[i].tobytes(), 77)


def test_bitsliced_layout_single_bits():
    rows = np.zeros((33, 2), np.uint8)
    rows[0, 0] = 0x01                    # instance 0, bit 0
    rows[32, 1] = 0x80                   # instance 32, bit 15
    w = grain.to_bitsliced(rows, 16)
    assert w.shape == (2, 16)
    assert w[0, 0] == 1 and w[1, 15] == 1 and w.sum() == 2
