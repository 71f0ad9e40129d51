"""Pins of the scalar oracle against facts that do not come from the oracle.

* The MICKEY 2.0 specification's known-answer vectors (tests/golden/).
* R is a Galois LFSR whose feedback polynomial x^100 + sum_{i in RTAPS} x^i
  the specification makes primitive (maximal period); a mis-typed tap almost
  surely breaks primitivity.  Checked against the factorisation of 2^100 - 1.
* CLOCK_R with control 0 and input 0 is multiplication by x modulo that
  polynomial (an independent polynomial-arithmetic model); input 1 adds the
  tap vector; control 1 adds the identity.
* Layout conversions: round trips and hand-made single-bit cases.
* The input generator against splitmix64's published first outputs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1909_04750_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mickey2_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, iv, iv_len, ks = line.split()
            rows.append((bytes.fromhex(key), b"" if iv == "-" else bytes.fromhex(iv),
                         int(iv_len), bytes.fromhex(ks)))
    return rows


@pytest.mark.parametrize("row", _kat_rows(), ids=lambda r: "iv%d" % r[2])
def test_known_answer_vectors(row):
    key, iv, iv_len, prefix = row
    iv_buf = iv + bytes(10 - len(iv))
    got = oracle.stream(key, iv_buf, iv_len, 8 * len(prefix))
    assert got == prefix


def test_known_answer_vector_via_state_api():
    key, iv, iv_len, prefix = _kat_rows()[1]
    st = oracle.init(key, iv, iv_len)
    a = oracle.keystream_from(st, 24)
    b = oracle.keystream_from(st, 8 * len(prefix) - 24)
    assert a + b == prefix


# ---------------------------------------------------------------- GF(2)[x]

def _pmulmod(a, b, p):
    deg = p.bit_length() - 1
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if (a >> deg) & 1:
            a ^= p
    return r


def _ppowmod(a, e, p):
    r = 1
    while e:
        if e & 1:
            r = _pmulmod(r, a, p)
        a = _pmulmod(a, a, p)
        e >>= 1
    return r


FACTORS_2_100_M1 = [3, 5, 5, 5, 11, 31, 41, 101, 251, 601, 1801, 4051, 8101, 268501]


def _is_prime(q):
    if q < 2:
        return False
    d = 2
    while d * d <= q:
        if q % d == 0:
            return False
        d += 1
    return True


def _is_primitive(p, n=100):
    order = (1 << n) - 1
    if _ppowmod(2, order, p) != 1:       # "2" is the polynomial x
        return False
    return all(_ppowmod(2, order // q, p) != 1 for q in set(FACTORS_2_100_M1))


def test_factorisation_of_group_order():
    prod = 1
    for q in FACTORS_2_100_M1:
        assert _is_prime(q)
        prod *= q
    assert prod == (1 << 100) - 1


def _state_poly(bits):
    return sum(int(b) << i for i, b in enumerate(bits))


def _clock_r_bits(r_bits, inp, ctl):
    st = oracle.State.from_bits(r_bits, np.zeros(100, np.uint8))
    oracle.clock_r(st, inp, ctl)
    return st.bits()[0]


def _tap_poly():
    e99 = np.zeros(100, np.uint8)
    e99[99] = 1
    # from r = e_99: shift moves the bit out, feedback r99 = 1 lands on RTAPS
    return _state_poly(_clock_r_bits(e99, 0, 0))


def test_r_feedback_polynomial_is_primitive():
    taps = _tap_poly()
    table = oracle.tables()["rtaps"]
    assert taps == _state_poly(table)
    assert bin(taps).count("1") == 50
    assert _is_primitive((1 << 100) | taps)


def test_primitivity_check_discriminates_single_tap_errors():
    taps = _tap_poly()
    # every single-bit change of the tap set must (almost always) fail
    still_primitive = sum(_is_primitive((1 << 100) | (taps ^ (1 << i)))
                          for i in range(1, 100))
    assert still_primitive <= 3


def test_r_clock_is_multiplication_by_x():
    p = (1 << 100) | _tap_poly()
    bits = np.zeros(100, np.uint8)
    bits[0] = 1
    poly = 1
    for t in range(300):
        assert _state_poly(bits) == poly, t
        bits = _clock_r_bits(bits, 0, 0)
        poly = _pmulmod(poly, 2, p)


def test_r_clock_input_and_control_terms():
    rng = np.random.default_rng(7)
    taps = _tap_poly()
    for _ in range(20):
        a = rng.integers(0, 2, 100, dtype=np.uint8)
        base = _state_poly(_clock_r_bits(a, 0, 0))
        assert _state_poly(_clock_r_bits(a, 1, 0)) == base ^ taps
        assert _state_poly(_clock_r_bits(a, 0, 1)) == base ^ _state_poly(a)
        assert _state_poly(_clock_r_bits(a, 1, 1)) == base ^ taps ^ _state_poly(a)


def test_r_clock_is_gf2_affine():
    rng = np.random.default_rng(8)
    for inp in (0, 1):
        for ctl in (0, 1):
            zero = _state_poly(_clock_r_bits(np.zeros(100, np.uint8), inp, ctl))
            for _ in range(10):
                a = rng.integers(0, 2, 100, dtype=np.uint8)
                b = rng.integers(0, 2, 100, dtype=np.uint8)
                lhs = _state_poly(_clock_r_bits(a ^ b, inp, ctl)) ^ zero
                rhs = (_state_poly(_clock_r_bits(a, inp, ctl))
                       ^ _state_poly(_clock_r_bits(b, inp, ctl)))
                assert lhs == rhs


def test_clock_kg_uses_old_state_for_both_registers():
    # CLOCK_KG must equal CLOCK_R and CLOCK_S applied to copies of the old
    # state with the control bits computed before either register moves.
    rng = np.random.default_rng(9)
    for mixing in (0, 1):
        for inp in (0, 1):
            r = rng.integers(0, 2, 100, dtype=np.uint8)
            s = rng.integers(0, 2, 100, dtype=np.uint8)
            st = oracle.State.from_bits(r, s)
            oracle.clock_kg(st, mixing, inp)
            cr = int(s[34] ^ r[67])
            cs = int(s[67] ^ r[33])
            a = oracle.State.from_bits(r, s)
            oracle.clock_r(a, inp ^ (int(s[50]) if mixing else 0), cr)
            b = oracle.State.from_bits(r, s)
            oracle.clock_s(b, inp, cs)
            got_r, got_s = st.bits()
            assert np.array_equal(got_r, a.bits()[0])
            assert np.array_equal(got_s, b.bits()[1])


# ---------------------------------------------------------------- init / IV

def test_iv_bits_beyond_iv_len_are_ignored():
    key = bytes(range(10))
    a = bytes([0xA5] * 10)
    for L in (0, 1, 7, 13, 40, 79):
        b = bytearray(a)
        # flip every bit at index >= L
        for bit in range(L, 80):
            b[bit // 8] ^= 0x80 >> (bit % 8)
        assert oracle.stream(key, a, L, 256) == oracle.stream(key, bytes(b), L, 256)


def test_iv_len_over_80_is_rejected():
    with pytest.raises(ValueError):
        oracle.stream(bytes(10), bytes(10), 81, 8)


def test_distinct_iv_lengths_give_distinct_streams():
    key = bytes(range(10))
    iv = bytes(10)
    outs = {oracle.stream(key, iv, L, 128) for L in range(0, 81, 8)}
    assert len(outs) == 11


def test_batch_matches_single_streams():
    s = workloads.batched(40)
    n_bits = (s.n_bits % 3000 + 8) // 8 * 8
    rows1 = oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, n_bits, threads=1)
    rows4 = oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, n_bits, threads=4)
    for i in range(s.n):
        one = oracle.stream(s.keys[i].tobytes(), s.ivs[i].tobytes(), int(s.iv_lens[i]),
                            int(n_bits[i]))
        assert rows1[i].tobytes() == one
        assert rows4[i].tobytes() == one


def test_keystream_monobit_and_runs_sanity():
    # NIST-style sanity (Sec. V-D uses SP 800-22); not a parity check.
    n = 1 << 18
    bits = oracle.bits_of(np.frombuffer(
        oracle.stream(bytes(range(10)), bytes(10), 80, n), np.uint8)[None, :], n)[0]
    ones = int(bits.sum())
    assert abs(2 * ones - n) < 4 * np.sqrt(n)
    runs = 1 + int(np.count_nonzero(bits[1:] != bits[:-1]))
    pi = ones / n
    expect = 2 * n * pi * (1 - pi)
    assert abs(runs - expect) < 4 * 2 * np.sqrt(2 * n) * pi * (1 - pi)


# ---------------------------------------------------------------- layouts

def test_bitsliced_layout_single_bit():
    n, n_bits = 70, 64
    rows = np.zeros((n, n_bits // 8), np.uint8)
    rows[33, 0] = 0x80 >> 5            # instance 33, keystream bit 5
    bs = oracle.to_bitsliced(rows, n_bits)
    assert bs.shape == (3, n_bits)
    expect = np.zeros_like(bs)
    expect[1, 5] = 1 << 1               # group 1, lane 1
    assert np.array_equal(bs, expect)


def test_bitsliced_round_trip():
    rng = np.random.default_rng(3)
    for n, n_bits in ((32, 64), (45, 72), (1, 8), (97, 200)):
        rows = rng.integers(0, 256, (n, (n_bits + 7) // 8), dtype=np.uint8)
        if n_bits % 8:
            rows[:, -1] &= np.uint8((0xFF << (8 - n_bits % 8)) & 0xFF)
        bs = oracle.to_bitsliced(rows, n_bits)
        assert np.array_equal(oracle.from_bitsliced(bs, n), rows)


def test_u32_layout_is_big_endian_read():
    rng = np.random.default_rng(4)
    rows = rng.integers(0, 256, (5, 16), dtype=np.uint8)
    words = oracle.to_u32(rows, 128)
    for i in range(5):
        assert np.array_equal(words[i], np.frombuffer(rows[i].tobytes(), ">u4"))


def test_f32_layout_exact():
    w = np.array([0, 0xFF, 0x100, 0xFFFFFFFF, 0x80000000, 0x12345678], np.uint32)
    f = oracle.to_f32(w)
    assert f.dtype == np.float32
    assert np.all(f >= 0) and np.all(f < 1)
    assert np.array_equal((f.astype(np.float64) * 2 ** 24).astype(np.uint64),
                          (w >> 8).astype(np.uint64))
    assert f[3] == np.float32(1 - 2 ** -24)


# ---------------------------------------------------------------- inputs

def test_splitmix64_reference_outputs():
    # first outputs of the published splitmix64 generator seeded with 0
    got = [int(x) for x in workloads.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_workload_shapes():
    s = workloads.plain_small()
    assert s.n == 32 and int(s.n_bits[0]) == 65536 and set(s.iv_lens) == {80}
    r = workloads.batched(5000)
    assert set(np.unique(r.iv_lens)) == {0, 16, 32, 48, 64, 80}
    assert r.n_bits.min() >= 1024 and r.n_bits.max() <= 1 << 22
    assert np.all(r.n_bits % 8 == 0)
    # the key of instance i is draws 4i, 4i+1 (little-endian)
    d = workloads.splitmix64(2, 8)
    s2 = workloads.plain_scale(2)
    assert s2.keys[1, :8].tobytes() == int(d[4]).to_bytes(8, "little")
    assert s2.keys[1, 8:].tobytes() == int(d[5]).to_bytes(8, "little")[:2]
    assert s2.ivs[1, :8].tobytes() == int(d[6]).to_bytes(8, "little")
    assert s2.ivs[1, 8:].tobytes() == int(d[7]).to_bytes(8, "little")[:2]
