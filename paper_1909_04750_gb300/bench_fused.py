"""Benchmark of the fused consumer output: 2^24 instances x 2^12 keystream
bits (seed 5), un-bitsliced in the keystream kernel into row-major u32
words (bit 32k the MSB of word k) and FP32 uniforms (word >> 8) * 2^-24.

    python -m paper_1909_04750_gb300.bench_fused [--steps K] [--warmup W]

A step re-keys every instance (load + 100 mixing preclocks) and generates
2^12 bits of each into the u32 block and the f32 block (8 GiB each, far
larger than L2).  Prints one JSON line: keystream Gbit/s of whole steps,
the keystream kernel's integer-logic roofline fraction (327 logic ops per
clock per 32-lane group over its CUDA-event time) and its HBM write rate.
"""
import argparse
import json
import statistics

import torch

from . import _native as N
from . import autotune, workloads
from .build import build
from .peak import lop3_peak_tops
from .streams import Streams, ops_per_clock


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--n", type=int, default=workloads.FUSED["n"])
    p.add_argument("--n-bits", type=int, default=workloads.FUSED["n_bits"])
    a = p.parse_args()
    build()
    s = workloads.fused(a.n)
    keys, ivs = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
    st = Streams(keys, ivs)
    out = torch.empty(2 * a.n * (a.n_bits // 32), dtype=torch.int32, device="cuda")
    tuned = autotune.tune(st, a.n_bits, N.LAYOUT_U32_F32)
    stream = st.stream
    for _ in range(max(3, a.warmup)):
        st.reset(keys, ivs)
        st.generate(a.n_bits, "u32_f32", out=out)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(a.steps)]
    for k in range(a.steps):
        ev[k][0].record(stream)
        st.reset(keys, ivs)
        ev[k][1].record(stream)
        st.generate(a.n_bits, "u32_f32", out=out)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    ks_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
    bits = a.n * a.n_bits
    groups = (a.n + 31) // 32
    peak = lop3_peak_tops()
    achieved = groups * a.n_bits * ops_per_clock(False) / (ks_ms * 1e-3) / 1e12
    out_bytes = out.numel() * 4
    print(json.dumps({
        "metric": "fused u32 + f32 keystream Gbit/s (2^24 instances x 2^12 bits)",
        "value": bits * a.steps / (sum(step_ms) * 1e-3) / 1e9, "unit": "Gbit/s",
        "ms_per_step": sum(step_ms) / a.steps, "steps": a.steps, "warmup": a.warmup,
        "keystream_kernel_ms": ks_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak},
        "hbm_write_gb_s": out_bytes / (ks_ms * 1e-3) / 1e9,
        "output_bytes": out_bytes,
        "config": {"workload": "fused_u32_f32", "instances": a.n, "bits_per_instance": a.n_bits,
                   "launch": autotune.describe(tuned), "l2": "output 16 GiB > L2"},
    }), flush=True)
    st.free()


if __name__ == "__main__":
    main()
