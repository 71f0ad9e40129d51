"""Benchmark of mickey_generate_ragged: every stream of a handle continues by
its own number of bits in one call.

    python -m paper_1909_04750_gb300.bench_ragged [--n N] [--max-bits B] [--calls K]

2^20 streams (seed 2) continue, `--calls` times back to back, by lengths
drawn uniformly from [max_bits / 2, max_bits] (seed 1; and once more with
every length max_bits), bytes layout at the packed offsets.  Prints one JSON
line: output Gbit/s of each case (CUDA events around the calls, outputs
larger than L2) and the share of the clocked bits that are output (a group
is clocked as often as its longest lane); `bench.py` adds a sampled check
of one more call's rows against the oracle.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import workloads
from .build import build
from .clocks import ClockSampler
from .streams import Streams


def _time(st, nb, out, calls):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    st.generate_ragged(nb, "bytes", out=out)          # warm-up
    torch.cuda.synchronize()
    ev[0].record(st.stream)
    for _ in range(calls):
        st.generate_ragged(nb, "bytes", out=out)
    ev[1].record(st.stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / calls


def measure(n: int = 1 << 20, max_bits: int = 1 << 14, calls: int = 5, verify=None) -> dict:
    """Time `calls` back-to-back calls of each case; `verify(s, rows,
    offsets, lengths, before)` checks the rows of one more spread call
    (stream i's bits before[i] .. before[i] + lengths[i] - 1) and returns a
    dict for the line."""
    s = workloads.plain_scale(n)
    st = Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    rng = np.random.default_rng(1)
    spread = rng.integers(max_bits // 2, max_bits + 1, n).astype(np.uint64)
    equal = np.full(n, max_bits, np.uint64)
    out = torch.empty(n * ((max_bits + 7) // 8), dtype=torch.uint8, device="cuda")
    sampler = ClockSampler(torch.cuda.current_device()).start()
    ms_spread = _time(st, spread, out, calls)
    ms_equal = _time(st, equal, out, calls)
    clocks = sampler.stop()
    line = {
        "metric": "ragged keystream Gbit/s (mickey_generate_ragged, bytes layout)",
        "streams": n,
        "spread": {"lengths": "uniform in [%d, %d]" % (max_bits // 2, max_bits),
                   "ms_per_call": ms_spread,
                   "gbit_s": float(spread.sum()) / (ms_spread * 1e-3) / 1e9,
                   "output_share_of_clocked_bits": float(spread.sum()) / float(
                       spread.reshape(-1, 32).max(axis=1).sum() * 32)},
        "equal": {"lengths": max_bits, "ms_per_call": ms_equal,
                  "gbit_s": float(equal.sum()) / (ms_equal * 1e-3) / 1e9},
        "clocks": clocks,
    }
    if verify is not None:
        # every stream has run calls + 1 spread and calls + 1 equal calls
        before = (calls + 1) * (spread + equal)
        rows, offs = st.generate_ragged(spread, "bytes", out=out)
        st.sync()
        line["verified"] = verify(s, rows, offs, spread, before)
    st.free()
    return line


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--max-bits", type=int, default=1 << 14)
    p.add_argument("--calls", type=int, default=5)
    a = p.parse_args()
    build()
    print(json.dumps(measure(a.n, a.max_bits, a.calls)), flush=True)


if __name__ == "__main__":
    main()
