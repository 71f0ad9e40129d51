"""The LFSR / CRC-8 oracle pinned to facts outside itself: the catalogued
CRC-8 check values, polynomial division over GF(2) (written out here with
Python integers), the CRC residue and linearity properties, the textbook
m-sequence of x^4 + x + 1, and the period 2^n - 1 of LFSRs whose polynomial
this file proves primitive."""
import os

import numpy as np
import pytest

from oracle import lfsr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            yield line


# ---------------------------------------------------------------- GF(2)[x]

def pmod(a: int, m: int) -> int:
    """a mod m for polynomials over GF(2) held as integers (bit k = x^k)."""
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def pmulmod(a: int, b: int, m: int) -> int:
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a = pmod(a << 1, m)
    return pmod(r, m)


def ppowmod(a: int, e: int, m: int) -> int:
    r = 1
    while e:
        if e & 1:
            r = pmulmod(r, a, m)
        a = pmulmod(a, a, m)
        e >>= 1
    return r


def primitive(c: int, n: int, primes) -> bool:
    order = (1 << n) - 1
    return ppowmod(2, order, c) == 1 and all(ppowmod(2, order // q, c) != 1 for q in primes)


# ---------------------------------------------------------------- CRC-8

def test_crc8_catalogue_check_values():
    for row in _rows("crc8_check.txt"):
        name, poly, init, xorout, check = row.split()
        assert lfsr.crc8(b"123456789", int(poly, 16), int(init, 16), int(xorout, 16)) == \
            int(check, 16), name


@pytest.mark.parametrize("poly", [0x07, 0x1D, 0x2F, 0x9B, 0x31])
def test_crc8_is_the_remainder_of_m_times_x8(poly):
    rng = np.random.default_rng(poly)
    P = 0x100 | poly
    for ln in (0, 1, 2, 5, 33):
        msg = rng.integers(0, 256, ln, dtype=np.uint8).tobytes()
        M = int.from_bytes(msg, "big") if msg else 0       # first bit = highest power
        assert lfsr.crc8(msg, poly) == pmod(M << 8, P), ln


@pytest.mark.parametrize("poly", [0x07, 0x1D, 0x2F])
def test_crc8_preset_and_final_xor(poly):
    # a preset register adds init(x) * x^(8L) mod P; the final XOR is a XOR
    rng = np.random.default_rng(3)
    P = 0x100 | poly
    for ln in (1, 4, 17):
        msg = rng.integers(0, 256, ln, dtype=np.uint8).tobytes()
        for init in (0x01, 0x80, 0xFF, 0x5A):
            want = pmod(int.from_bytes(msg, "big") << 8, P) ^ pmod(init << (8 * ln), P)
            assert lfsr.crc8(msg, poly, init, 0) == want
            assert lfsr.crc8(msg, poly, init, 0xA5) == want ^ 0xA5


def test_crc8_residue_and_linearity():
    rng = np.random.default_rng(9)
    for poly in (0x07, 0x1D):
        for ln in (1, 8, 31):
            a = rng.integers(0, 256, ln, dtype=np.uint8)
            b = rng.integers(0, 256, ln, dtype=np.uint8)
            ca = lfsr.crc8(a.tobytes(), poly)
            assert lfsr.crc8(a.tobytes() + bytes([ca]), poly) == 0
            assert lfsr.crc8((a ^ b).tobytes(), poly) == ca ^ lfsr.crc8(b.tobytes(), poly)


def test_crc8_batch_matches_single():
    rng = np.random.default_rng(4)
    data = rng.integers(0, 256, (37, 19), dtype=np.uint8)
    got = lfsr.crc8_batch(data, 0x1D, 0xFF, 0xFF, threads=4)
    assert [int(x) for x in got] == [lfsr.crc8(r.tobytes(), 0x1D, 0xFF, 0xFF) for r in data]


# ---------------------------------------------------------------- LFSR

def test_lfsr_textbook_m_sequence():
    (seq,) = list(_rows("lfsr_m_sequence.txt"))
    ref = np.array([int(c) for c in seq], np.uint8)
    got = lfsr.lfsr_bits(0b1000, 4, 0b0011, 3 * 15)
    assert np.array_equal(got[:15], ref)
    assert np.array_equal(got[15:30], ref) and np.array_equal(got[30:], ref)
    # the reciprocal polynomial x^4 + x^3 + 1 gives a different sequence
    assert not np.array_equal(lfsr.lfsr_bits(0b1000, 4, 0b1001, 15), ref)


def _period(bits: np.ndarray, n: int) -> int:
    first = bits[:n].tobytes()
    for p in range(1, len(bits) - n + 1):
        if bits[p:p + n].tobytes() == first:
            return p
    return -1


@pytest.mark.parametrize("n,primes", [(7, [127]), (12, [3, 5, 7, 13]), (16, [3, 5, 17, 257])])
def test_lfsr_period_of_primitive_polynomials(n, primes):
    # first polynomials c(x) = x^n + ... + 1 that are primitive, proved here;
    # the characteristic polynomial of the recurrence is x^n + sum a_j x^j
    found = 0
    for low in range(1, 1 << n, 2):
        c = (1 << n) | low
        if not primitive(c, n, primes):
            continue
        bits = lfsr.lfsr_bits(1, n, low, (1 << n) + n + 5)
        assert _period(bits, n) == (1 << n) - 1, hex(c)
        found += 1
        if found == 3:
            break
    assert found == 3
    # a reducible polynomial: (x^2 + x + 1)^2 = x^4 + x^2 + 1 -> shorter period
    assert _period(lfsr.lfsr_bits(1, 4, 0b0101, 40), 4) < 15


def test_lfsr_degree_64_runs():
    bits = lfsr.lfsr_bits((1 << 64) - 1, 64, 0b11011, 200)
    assert bits[:64].sum() == 64 and bits.shape == (200,)
