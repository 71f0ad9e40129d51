"""Seeded synthetic inputs (keys, IVs, IV lengths, stream lengths, arrivals).

This module holds input generation only -- none of the cipher's arithmetic --
so that the GPU path, the oracle-based tests and the benchmark can all draw
the same inputs from it.

Generator: splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): the state advances by the odd constant
0x9E3779B97F4A7C15 and each output is the state passed through two
xor-shift-multiply rounds (shifts 30, 27, 31; multipliers 0xBF58476D1CE4E5B9
and 0x94D049BB133111EB).  Draw k of seed s is therefore a pure function of
s + (k + 1) * 0x9E3779B97F4A7C15, which lets numpy produce millions at once.

Per-instance recipe (instance i uses draws D*i .. D*i + D - 1):
  key    = little-endian bytes of draw 0 (8 bytes), then bytes 0-1 of draw 1
  IV     = the same from draws 2 and 3
  D = 4 for the fixed-length workloads; D = 6 for the ragged one, where
  iv_len = 16 * (draw 4 mod 6) and the keystream length is
  floor(2 ** (10 + 12 * u)) rounded down to a multiple of 8 bits with
  u = (draw 5 >> 11) * 2**-53, i.e. log-uniform in [2**10, 2**22] bits.

The paper seeds its instances from an unspecified expansion of stored random
numbers (Sec. IV-D); these workloads replace that with splitmix64 draws of the
same shape: 80-bit keys and IVs, one per generator instance.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Draws start .. start+count-1 of splitmix64 seeded with `seed`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & (2**64 - 1)) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def _ten_bytes(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    n = lo.shape[0]
    out = np.empty((n, 10), np.uint8)
    out[:, :8] = lo.astype("<u8").view(np.uint8).reshape(n, 8)
    out[:, 8:] = hi.astype("<u8").view(np.uint8).reshape(n, 8)[:, :2]
    return out


@dataclass
class StreamSet:
    """Inputs for n independent keystreams."""
    name: str
    seed: int
    keys: np.ndarray          # uint8 [n, 10]
    ivs: np.ndarray           # uint8 [n, 10]
    iv_lens: np.ndarray       # uint32 [n], bits, 0..80
    n_bits: np.ndarray        # uint64 [n], keystream bits per stream
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.keys.shape[0])

    def subset(self, idx) -> "StreamSet":
        idx = np.asarray(idx)
        return StreamSet(self.name, self.seed, self.keys[idx], self.ivs[idx],
                         self.iv_lens[idx], self.n_bits[idx], dict(self.meta))


def fixed_streams(name: str, seed: int, n: int, n_bits: int,
                  iv_len: int = 80, first: int = 0) -> StreamSet:
    """Instances first .. first+n-1 of the workload: instance i takes draws
    4i .. 4i+3 (key low/high, IV low/high)."""
    d = splitmix64(seed, 4 * n, 4 * first).reshape(n, 4)
    return StreamSet(name, seed, _ten_bytes(d[:, 0], d[:, 1]),
                     _ten_bytes(d[:, 2], d[:, 3]),
                     np.full(n, iv_len, np.uint32), np.full(n, n_bits, np.uint64))


def ragged_streams(name: str, seed: int, n: int, lo_log2: int = 10,
                   hi_log2: int = 22) -> StreamSet:
    d = splitmix64(seed, 6 * n).reshape(n, 6)
    iv_lens = (16 * (d[:, 4] % np.uint64(6))).astype(np.uint32)
    u = (d[:, 5] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    nb = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.uint64)
    nb = (nb // np.uint64(8)) * np.uint64(8)
    return StreamSet(name, seed, _ten_bytes(d[:, 0], d[:, 1]),
                     _ten_bytes(d[:, 2], d[:, 3]), iv_lens, nb)


# The five workloads: sizes and seeds.
PLAIN_SMALL = dict(name="plain_small", seed=1, n=32, n_bits=65536)
PLAIN_SCALE = dict(name="plain_scale", seed=2, n=1 << 20, n_bits=1 << 14)
FUSED = dict(name="fused_u32_f32", seed=5, n=1 << 24, n_bits=1 << 12)
BATCHED = dict(name="batched_ragged", seed=3, n=100_000)


def plain_small() -> StreamSet:
    return fixed_streams(**PLAIN_SMALL)


def plain_scale(n: int | None = None) -> StreamSet:
    cfg = dict(PLAIN_SCALE)
    if n is not None:
        cfg["n"] = n
    return fixed_streams(**cfg)


def fused(n: int | None = None) -> StreamSet:
    cfg = dict(FUSED)
    if n is not None:
        cfg["n"] = n
    return fixed_streams(**cfg)


def batched(n: int | None = None) -> StreamSet:
    return ragged_streams(BATCHED["name"], BATCHED["seed"],
                          BATCHED["n"] if n is None else n)


# --------------------------------------------------------------------------
# Grain (the paper's second stream cipher): 80-bit keys, 64-bit IVs
# --------------------------------------------------------------------------

GRAIN_SCALE = dict(name="grain_scale", seed=6, n=1 << 20, n_bits=1 << 14)


@dataclass
class GrainSet:
    name: str
    seed: int
    keys: np.ndarray          # uint8 [n, 10]
    ivs: np.ndarray           # uint8 [n, 8]

    @property
    def n(self) -> int:
        return int(self.keys.shape[0])


def grain_streams(n: int | None = None, seed: int = GRAIN_SCALE["seed"]) -> GrainSet:
    """Instance i takes draws 3i .. 3i+2 of splitmix64(seed): key = the
    little-endian bytes of draw 0 and bytes 0-1 of draw 1, IV = the 8
    little-endian bytes of draw 2."""
    n = GRAIN_SCALE["n"] if n is None else n
    d = splitmix64(seed, 3 * n).reshape(n, 3)
    return GrainSet("grain_scale", seed, _ten_bytes(d[:, 0], d[:, 1]),
                    d[:, 2].astype("<u8").view(np.uint8).reshape(n, 8).copy())


# --------------------------------------------------------------------------
# served workload: a request trace
# --------------------------------------------------------------------------

@dataclass
class Request:
    arrival_s: float
    stream_id: int
    key: bytes
    iv: bytes
    iv_len: int
    n_bytes: int


def served_trace(seed: int = 4, rate_per_s: float = 1e4, duration_s: float = 30.0,
                 p_continue: float = 0.7, lo_log2_bytes: int = 10,
                 hi_log2_bytes: int = 26, max_requests: int | None = None):
    """Poisson arrivals at `rate_per_s` for `duration_s` seconds.

    Request j uses draws 4j .. 4j+3 of splitmix64(seed):
      draw 0: exponential inter-arrival gap, -ln(1 - u) / rate;
      draw 1: continue an existing stream (u < p_continue and at least one
              exists; the stream id is draw 2 mod the number of ids so far)
              or open a new id;
      draw 3: length log-uniform in [2**lo, 2**hi] bytes (whole bytes).
    A new stream id k takes key/IV from fixed_streams(seed + 1000) row k,
    with an 80-bit IV.
    """
    est = int(rate_per_s * duration_s * 1.2) + 64
    if max_requests is not None:
        est = min(est, max_requests)
    d = splitmix64(seed, 4 * est).reshape(est, 4)
    u = (d >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    gaps = -np.log1p(-u[:, 0]) / rate_per_s
    t = np.cumsum(gaps)
    keep = t < duration_s
    n_req = int(keep.sum())
    lengths = np.floor(2.0 ** (lo_log2_bytes + (hi_log2_bytes - lo_log2_bytes) * u[:, 3])).astype(np.int64)
    ids = np.empty(n_req, np.int64)
    n_ids = 0
    for j in range(n_req):
        if n_ids > 0 and u[j, 1] < p_continue:
            ids[j] = int(d[j, 2] % np.uint64(n_ids))
        else:
            ids[j] = n_ids
            n_ids += 1
    keys = fixed_streams("served_keys", seed + 1000, max(n_ids, 1), 0)
    reqs = [Request(float(t[j]), int(ids[j]), keys.keys[ids[j]].tobytes(),
                    keys.ivs[ids[j]].tobytes(), 80, int(lengths[j]))
            for j in range(n_req)]
    return reqs, keys.subset(np.arange(n_ids)) if n_ids else keys
