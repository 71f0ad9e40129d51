"""Measure the GPU's 3-input LOP3 rate (the keystream roofline's peak).

    python -m paper_1909_04750_gb300.peak
"""
import ctypes

from . import _native as N
from .build import build

CONFIGS = [(1, 128, 20000), (2, 128, 20000), (4, 256, 10000), (8, 256, 5000), (2, 1024, 5000)]


def main():
    build()
    L = N.lib()
    for bps, thr, it in CONFIGS:
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        N.check(L.mickey_probe_lop3(bps, thr, it, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)))
        print("blocks/SM=%d threads=%d: %.1f LOP3/SM/clk at %.0f MHz, %.2f T ops/s"
              % (bps, thr, a.value, b.value, c.value), flush=True)


if __name__ == "__main__":
    main()
