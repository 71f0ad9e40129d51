"""Benchmark of the bitsliced LFSR / CRC-8 library.

    python -m paper_1909_04750_gb300.bench_lfsr [--reps K]

CRC-8 (polynomial 0x1D, preset and final XOR 0xFF) of 2^20 messages of
1 KiB each (1 GiB, device-resident, far larger than L2): GB/s of message
bytes and the fraction of the measured HBM copy rate (the kernel reads each
byte once).  Fibonacci LFSRs of degree 64, 2^20 instances x 4096 bits:
with the four taps of x^64 + x^4 + x^3 + x + 1 (the sparse-tap kernel:
Gbit/s and the fraction of the measured HBM copy rate, the output words
being the only traffic that grows with the run), and the same LFSRs run
through the mask kernel (Gbit/s and the fraction of the LOP3 roofline: 64
logic ops per clock per 32 instances).  CUDA events; best of K.
"""
import argparse
import json
import os

import torch

from . import lfsr
from .build import build
from . import peak as P


def _hbm_peak_gbs() -> float | None:
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def _best_ms(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--reps", type=int, default=5)
    a = p.parse_args()
    build()
    n, ln = 1 << 20, 1024
    g = torch.Generator(device="cuda").manual_seed(5)
    data = torch.randint(0, 256, (n, ln), dtype=torch.uint8, device="cuda", generator=g)
    crc = torch.empty(n, dtype=torch.uint8, device="cuda")
    ms = _best_ms(lambda: lfsr.crc8(data, 0x1D, 0xFF, 0xFF, out=crc), a.reps)
    gbs = n * ln / (ms * 1e-3) / 1e9
    hbm = _hbm_peak_gbs()
    del data
    ni, nb, d = 1 << 20, 4096, 64
    seeds = torch.randint(1, 1 << 62, (ni,), dtype=torch.int64, device="cuda", generator=g)
    out = torch.empty((nb, (ni + 31) // 32), dtype=torch.int32, device="cuda")
    taps = 0b11011                                  # a_0, a_1, a_3, a_4
    ms2 = _best_ms(lambda: lfsr.lfsr_generate(seeds, d, taps, nb, out=out), a.reps)
    out_bytes = out.numel() * 4 + ni * 8              # output words + seeds read
    os.environ["MICKEY_LFSR_DENSE"] = "1"              # the same LFSRs, mask kernel
    try:
        ms3 = _best_ms(lambda: lfsr.lfsr_generate(seeds, d, taps, nb, out=out), a.reps)
    finally:
        del os.environ["MICKEY_LFSR_DENSE"]
    ops = (ni // 32) * (nb - d) * 64
    pk = P.measure()
    peak = P.peak_tops(pk, P.max_sm_mhz() or pk["probe_sm_mhz"])
    lfsr_gbs = out_bytes / (ms2 * 1e-3) / 1e9
    print(json.dumps({
        "crc8": {"messages": n, "bytes_each": ln, "ms": ms, "gb_s": gbs,
                 "hbm_frac": gbs / hbm if hbm else None,
                 "hbm_peak_gb_s": hbm, "peak_basis": "MEASURED_PEAKS.json hbm_gbs, of measured"},
        "lfsr": {"instances": ni, "degree": d, "taps": 4, "bits_each": nb, "ms": ms2,
                 "kernel": "lfsr_sparse_kernel", "gbit_s": ni * nb / (ms2 * 1e-3) / 1e9,
                 "roofline": {"bound": "hbm", "achieved_gb_s": lfsr_gbs, "peak_gb_s": hbm,
                              "frac": lfsr_gbs / hbm if hbm else None,
                              "bytes": out_bytes}},
        "lfsr_mask_kernel": {"instances": ni, "degree": d, "bits_each": nb, "ms": ms3,
                             "kernel": "lfsr_kernel<64>", "gbit_s": ni * nb / (ms3 * 1e-3) / 1e9,
                             "roofline": {"bound": "alu",
                                          "achieved_tops": ops / (ms3 * 1e-3) / 1e12,
                                          "peak_tops": peak,
                                          "frac": ops / (ms3 * 1e-3) / 1e12 / peak,
                                          "peak_basis": "%d SMs x %.2f LOP3/SM/clk "
                                                        "(mickey_probe_lop3) x max SM clock"
                                                        % (pk["n_sm"], pk["lop3_per_sm_clk"])}},
    }), flush=True)


if __name__ == "__main__":
    main()
