"""Bitsliced Fibonacci LFSRs and CRC-8 (C ABI: mickey_lfsr_generate,
mickey_crc8; include/bitslice_lfsr.h).  Marshalling only: the work runs in
the library's kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N


def _stream_ptr(stream) -> ctypes.c_void_p:
    return ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


def lfsr_generate(seeds, degree: int, taps: int, n_bits: int, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """n_bits output bits of len(seeds) LFSRs, word-major bitsliced:
    out[t, g] bit l = output bit t of instance 32g + l (int32 [n_bits, G])."""
    L = N.lib()
    if isinstance(seeds, torch.Tensor) and seeds.is_cuda:
        sd, mem = seeds.contiguous(), N.MEM_DEVICE
        ptr = sd.data_ptr()
        n = sd.numel()
    else:
        sd = np.ascontiguousarray(seeds, np.uint64)
        mem, ptr, n = N.MEM_HOST, sd.ctypes.data, sd.size
    G = (n + 31) // 32
    if out is None:
        out = torch.empty((n_bits, G), dtype=torch.int32, device="cuda")
    if out.numel() < n_bits * G:
        raise N.MickeyError(N.E_ARG, "output too small")
    N.check(L.mickey_lfsr_generate(ptr, n, degree, taps, n_bits,
                                   ctypes.c_void_p(out.data_ptr()), mem, _stream_ptr(stream)))
    return out


def crc8(data, poly: int, init: int = 0, xorout: int = 0, out: torch.Tensor | None = None,
         stream=None):
    """CRC-8 of every row of a uint8 [n, len] array or CUDA tensor."""
    L = N.lib()
    if isinstance(data, torch.Tensor) and data.is_cuda:
        d = data.contiguous()
        n, ln = d.shape
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=d.device)
        N.check(L.mickey_crc8(ctypes.c_void_p(d.data_ptr()), n, ln, poly, init, xorout,
                              ctypes.c_void_p(out.data_ptr()), N.MEM_DEVICE, _stream_ptr(stream)))
        return out
    d = np.ascontiguousarray(data, np.uint8)
    n, ln = d.shape
    res = np.zeros(n, np.uint8)
    N.check(L.mickey_crc8(d.ctypes.data, n, ln, poly, init, xorout, res.ctypes.data, N.MEM_HOST,
                          _stream_ptr(stream)))
    return res


def unbitslice(words: np.ndarray, n: int) -> np.ndarray:
    """[n_bits, G] word-major bitsliced words -> [n, n_bits] bits (for checks)."""
    w = np.ascontiguousarray(words).view(np.uint32)
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1       # [t, g, l]
    return bits.transpose(1, 2, 0).reshape(-1, w.shape[0])[:n].astype(np.uint8)
