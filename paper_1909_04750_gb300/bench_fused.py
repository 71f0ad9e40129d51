"""Benchmark of the fused consumer output: 2^24 instances x 2^12 keystream
bits (seed 5), un-bitsliced in the keystream kernel into row-major u32
words (bit 32k the MSB of word k) and FP32 uniforms (word >> 8) * 2^-24.

    python -m paper_1909_04750_gb300.bench_fused [--steps K] [--warmup W]

A step re-keys every instance (load + 100 mixing preclocks) and generates
2^12 bits of each into the u32 block and the f32 block (8 GiB each, far
larger than L2).  Prints one JSON line: keystream Gbit/s of whole steps,
the keystream kernel's integer-logic roofline fraction (327 logic ops per
clock per 32-lane group over its CUDA-event time), the preclock kernel's
(329 ops per mixing clock, 260 clocks per group) and the HBM write rate.
"""
import argparse
import json
import statistics

import torch

from . import _native as N
from . import autotune, workloads
from . import peak as P
from .build import build
from .clocks import ClockSampler
from .streams import Streams, ops_per_clock


def measure(steps: int = 5, warmup: int = 3, n: int = workloads.FUSED["n"],
            n_bits: int = workloads.FUSED["n_bits"], peak=None, verify=None) -> dict:
    """Time `steps` fused steps; `peak` is peak.measure()'s dict (measured
    here if None); `verify(streamset, out)` checks the last step's output
    and returns a dict for the line."""
    s = workloads.fused(n)
    keys, ivs = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
    st = Streams(keys, ivs)
    out = torch.empty((2, n, n_bits // 32), dtype=torch.int32, device="cuda")
    tuned = autotune.tune(st, n_bits, N.LAYOUT_U32_F32)
    stream = st.stream
    for _ in range(max(3, warmup)):
        st.reset(keys, ivs)
        st.generate(n_bits, "u32_f32", out=out)
    torch.cuda.synchronize()
    pk = peak or P.measure()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    sampler = ClockSampler(torch.cuda.current_device()).start()
    for k in range(steps):
        ev[k][0].record(stream)
        st.reset(keys, ivs)
        ev[k][1].record(stream)
        st.generate(n_bits, "u32_f32", out=out)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    st.sync()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    ks_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    init_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    bits = n * n_bits
    groups = (n + 31) // 32
    mhz = clocks.get("sm_max_mhz") or P.max_sm_mhz() or pk["probe_sm_mhz"]
    peak = P.peak_tops(pk, mhz)
    achieved = groups * n_bits * ops_per_clock(False) / (ks_ms * 1e-3) / 1e12
    init_tops = groups * 260 * ops_per_clock(True) / (init_ms * 1e-3) / 1e12
    out_bytes = out.numel() * 4
    line = {
        "metric": "fused u32 + f32 keystream Gbit/s (2^24 instances x 2^12 bits)",
        "value": bits * steps / (sum(step_ms) * 1e-3) / 1e9, "unit": "Gbit/s",
        "ms_per_step": sum(step_ms) / steps, "steps": steps, "warmup": warmup,
        "keystream_kernel_ms": ks_ms, "init_ms": init_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak,
                     "frac_at_median_clock": (achieved / P.peak_tops(pk, clocks["sm_mhz"])
                                              if clocks.get("sm_mhz") else None),
                     "kernel": "keystream kernel, u32 + f32 layout"},
        "init_roofline_frac": init_tops / peak,
        "hbm_write_gb_s": out_bytes / (ks_ms * 1e-3) / 1e9,
        "output_bytes": out_bytes,
        "config": {"workload": "fused_u32_f32: 2^24 instances x 2^12 bits, seed 5, u32 words "
                               "and FP32 uniforms", "instances": n, "bits_per_instance": n_bits,
                   "launch": autotune.describe(tuned), "l2": "output 16 GiB > L2"},
        "clocks": clocks,
    }
    if verify is not None:
        line["verified"] = verify(s, out)
    st.free()
    del out
    torch.cuda.empty_cache()
    return line


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=workloads.FUSED["n"])
    p.add_argument("--n-bits", type=int, default=workloads.FUSED["n_bits"])
    a = p.parse_args()
    build()
    print(json.dumps(measure(a.steps, a.warmup, a.n, a.n_bits)), flush=True)


if __name__ == "__main__":
    main()
