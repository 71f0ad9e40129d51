"""Benchmark of bitsliced Grain: 2^20 instances x 2^14 keystream bits
(80-bit keys, 64-bit IVs from splitmix64 seed 6).

    python -m paper_1909_04750_gb300.bench_grain [--steps K] [--warmup W]

A step re-keys every instance (loading + 160 initialisation clocks) and
generates 2^14 bits of each, as row-major bytes (2 GiB) or in the bitsliced
layout.  Prints one JSON line: keystream Gbit/s of whole steps, and the
keystream kernel's integer-logic roofline fraction (37 logic ops per clock
per 32-lane group over its CUDA-event time).
"""
import argparse
import json
import statistics

import torch

from . import peak as P
from . import workloads
from .build import build
from .clocks import ClockSampler
from .grain import GrainStreams, ops_per_clock


def _time(st, keys, ivs, n_bits, layout, out, steps, flush):
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)                      # evict L2 between steps
        ev[k][0].record(st.stream)
        st.reset(keys, ivs)
        ev[k][1].record(st.stream)
        st.generate(n_bits, layout, out=out)
        ev[k][2].record(st.stream)
    torch.cuda.synchronize()
    return ([e[0].elapsed_time(e[2]) for e in ev], [e[1].elapsed_time(e[2]) for e in ev])


def measure(steps: int = 10, warmup: int = 3, n: int = workloads.GRAIN_SCALE["n"],
            n_bits: int = workloads.GRAIN_SCALE["n_bits"], peak=None, verify=None) -> dict:
    """`verify(grainset, out_bytes)` checks the last bytes step and returns a dict."""
    s = workloads.grain_streams(n)
    keys, ivs = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
    st = GrainStreams(keys, ivs)
    out = torch.empty((n, (n_bits + 7) // 8), dtype=torch.uint8, device="cuda")
    out_bs = torch.empty(((n + 31) // 32, n_bits), dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, warmup)):
        st.reset(keys, ivs)
        st.generate(n_bits, "bytes", out=out)
        st.reset(keys, ivs)
        st.generate(n_bits, "bitsliced", out=out_bs)
    torch.cuda.synchronize()
    pk = peak or P.measure()
    sampler = ClockSampler(torch.cuda.current_device()).start()
    step_ms, ks_ms = _time(st, keys, ivs, n_bits, "bytes", out, steps, flush)
    bs_step, bs_ks = _time(st, keys, ivs, n_bits, "bitsliced", out_bs, steps, flush)
    clocks = sampler.stop()
    groups = (n + 31) // 32
    mhz = clocks.get("sm_max_mhz") or P.max_sm_mhz() or pk["probe_sm_mhz"]
    peak = P.peak_tops(pk, mhz)
    ops = groups * n_bits * ops_per_clock(False)

    def roof(ms):
        achieved = ops / (statistics.mean(ms) * 1e-3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "ops_per_clock_per_group": ops_per_clock(False)}

    line = {
        "metric": "Grain keystream Gbit/s (2^20 instances x 2^14 bits)",
        "value": n * n_bits * steps / (sum(step_ms) * 1e-3) / 1e9, "unit": "Gbit/s",
        "ms_per_step": sum(step_ms) / steps, "steps": steps, "layout": "bytes",
        "bitsliced_gbit_s": n * n_bits * steps / (sum(bs_step) * 1e-3) / 1e9,
        "roofline": dict(roof(ks_ms), kernel="grain keystream kernel, bytes layout"),
        "roofline_bitsliced": dict(roof(bs_ks), kernel="grain keystream kernel, bitsliced"),
        "init_ms": statistics.mean(a - b for a, b in zip(step_ms, ks_ms)),
        "config": {"workload": "grain_scale: 2^20 Grain instances, 80-bit keys and 64-bit IVs "
                               "from splitmix64 seed 6, 160 initialisation clocks, 2^14 "
                               "keystream bits per instance", "instances": n,
                   "bits_per_instance": n_bits, "l2": "512 MiB buffer written between steps"},
        "clocks": clocks,
    }
    if verify is not None:
        line["verified"] = verify(s, out)
    st.free()
    del out, out_bs, flush
    torch.cuda.empty_cache()
    return line


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    a = p.parse_args()
    build()
    print(json.dumps(measure(a.steps, a.warmup)), flush=True)


if __name__ == "__main__":
    main()
