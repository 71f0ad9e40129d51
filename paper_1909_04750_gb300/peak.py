"""Measure the GPU's 3-input LOP3 rate (the keystream roofline's peak) and
the rate of the bare bitsliced clock (the ceiling of the keystream kernel).

    python -m paper_1909_04750_gb300.peak
"""
import ctypes

from . import _native as N
from .build import build

CONFIGS = [(1, 128, 20000), (2, 128, 20000), (4, 256, 10000), (8, 256, 5000), (2, 1024, 5000)]

# The integer-logic roofline: GB300 runs 64 three-input LOP3 per SM per
# clock (half the lanes per cycle; measured with the probe below, every
# configuration), 152 SMs, 2070 MHz maximum SM clock.
N_SM = 152
LOP3_PER_SM_CLK = 64.0
SM_MAX_MHZ = 2070.0


def lop3_peak_tops(n_sm: int = N_SM) -> float:
    """LOP3 roofline in 10^12 logic ops per second."""
    return n_sm * LOP3_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12


def main():
    build()
    L = N.lib()
    for bps, thr, it in CONFIGS:
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        N.check(L.mickey_probe_lop3(bps, thr, it, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)))
        print("blocks/SM=%d threads=%d: %.1f LOP3/SM/clk at %.0f MHz, %.2f T ops/s"
              % (bps, thr, a.value, b.value, c.value), flush=True)
    # the bare keystream clock: the ceiling of the kernel's clock warps
    for bps in (1, 2):
        a, b = ctypes.c_double(), ctypes.c_double()
        N.check(L.mickey_probe_clock(bps, 8192, ctypes.byref(a), ctypes.byref(b)))
        print("bare clock, %d warp(s) per SM sub-partition: %.1f algorithmic ops/SM/clk "
              "= %.3f of %.0f, at %.0f MHz" % (bps, a.value, a.value / LOP3_PER_SM_CLK,
                                               LOP3_PER_SM_CLK, b.value), flush=True)


if __name__ == "__main__":
    main()
