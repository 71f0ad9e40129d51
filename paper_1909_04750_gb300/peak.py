"""Measure the GPU's 3-input LOP3 rate (the keystream roofline's peak) and
the rate of the bare bitsliced clock (the ceiling of the keystream kernel).

    python -m paper_1909_04750_gb300.peak

The integer-logic roofline is SM count x LOP3 results per SM per SM-cycle x
SM clock.  The first two are read here from the device (its multiprocessor
count) and from the probe kernel (independent LOP3 chains, timed in SM
cycles, so the figure does not depend on the clock the GPU ran at); the
clock is the one the caller sampled (the maximum, and the median under
load).  On GB300 the probe gives 63.2-64.0 results per SM per cycle: the
integer-logic pipe is half a warp wide.
"""
import ctypes
import subprocess

from . import _native as N
from .build import build

CONFIGS = [(1, 128, 20000), (2, 128, 20000), (4, 256, 10000), (8, 256, 5000), (2, 1024, 5000)]
# the configurations measure() runs (a few ms each)
QUICK = [(2, 128, 20000), (4, 256, 10000)]


def probe_lop3(blocks_per_sm: int, threads: int, iters: int):
    """(LOP3 results per SM per SM-cycle, SM MHz seen, whole-GPU T ops/s)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    N.check(N.lib().mickey_probe_lop3(blocks_per_sm, threads, iters, ctypes.byref(a),
                                      ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sm_count() -> int:
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device())
               .multi_processor_count)


def max_sm_mhz(gpu_index: int = 0):
    """clocks.max.sm from nvidia-smi (a read-only query), or None."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip()
        return float(out.splitlines()[0])
    except Exception:
        return None


def measure(configs=QUICK) -> dict:
    """The roofline's factors on the current device: SM count and the best
    LOP3 rate per SM per cycle over `configs` of the probe."""
    rates = [probe_lop3(*c) for c in configs]
    best = max(rates, key=lambda r: r[0])
    return {"n_sm": sm_count(), "lop3_per_sm_clk": best[0], "probe_sm_mhz": best[1],
            "probe": "mickey_probe_lop3 %s (blocks/SM, threads, iterations); best of %d"
                     % (list(configs), len(configs))}


def peak_tops(m: dict, sm_mhz: float) -> float:
    """Integer-logic roofline in 10^12 ops/s at SM clock `sm_mhz`."""
    return m["n_sm"] * m["lop3_per_sm_clk"] * sm_mhz * 1e6 / 1e12


def main():
    build()
    for bps, thr, it in CONFIGS:
        a, b, c = probe_lop3(bps, thr, it)
        print("blocks/SM=%d threads=%d: %.1f LOP3/SM/clk at %.0f MHz, %.2f T ops/s"
              % (bps, thr, a, b, c), flush=True)
    m = measure()
    print("SMs: %d; roofline at %s MHz: %.2f T ops/s" % (
        m["n_sm"], max_sm_mhz(), peak_tops(m, max_sm_mhz() or m["probe_sm_mhz"])), flush=True)
    # the bare keystream clock: the ceiling of the kernel's clock warps
    for bps in (1, 2):
        a, b = ctypes.c_double(), ctypes.c_double()
        N.check(N.lib().mickey_probe_clock(bps, 8192, ctypes.byref(a), ctypes.byref(b)))
        print("bare clock, %d warp(s) per SM sub-partition: %.1f algorithmic ops/SM/clk "
              "= %.3f of %.1f, at %.0f MHz" % (bps, a.value, a.value / m["lop3_per_sm_clk"],
                                               m["lop3_per_sm_clk"], b.value), flush=True)
    # the bare Grain clock at 1 and 2 warps per SM sub-partition
    for bps in (2, 4):
        for store in (False, True):
            r, mhz = grain_clock(bps, store)
            print("bare Grain clock, %d warp(s) per SM sub-partition%s: %.1f ops/SM/clk = %.3f "
                  "of %.1f, at %.0f MHz" % (bps // 2, ", keystream words to shared memory"
                                            if store else "", r, r / m["lop3_per_sm_clk"],
                                            m["lop3_per_sm_clk"], mhz), flush=True)


def grain_clock(blocks_per_sm: int, store: bool, bodies: int = 200):
    """Bare Grain clock: (ops per SM per SM-cycle, SM MHz)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    N.check(N.lib().grain_probe_clock(blocks_per_sm, bodies, 1 if store else 0, ctypes.byref(a),
                                      ctypes.byref(b)))
    return a.value, b.value


if __name__ == "__main__":
    main()
