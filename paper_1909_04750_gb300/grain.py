"""Torch-facing wrapper of the Grain C ABI (include/grain.h): device
buffers and streams from torch, all keystream work in libmickey's kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N

LAYOUTS = {"bitsliced": N.LAYOUT_BITSLICED_U32, "bytes": N.LAYOUT_BYTES}


def _lay(layout) -> int:
    return LAYOUTS[layout] if isinstance(layout, str) else int(layout)


class GrainStreams:
    """n independent Grain keystreams, bitsliced on one GPU.

    keys: uint8 [n, 10], ivs: uint8 [n, 8] (CUDA tensors or host arrays).
    """

    def __init__(self, keys, ivs, stream=None):
        self._L = N.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if isinstance(keys, torch.Tensor) and keys.is_cuda:
            k, v, mem = keys.contiguous(), ivs.contiguous(), N.MEM_DEVICE
            kp, vp = k.data_ptr(), v.data_ptr()
            self.n = k.numel() // 10
        else:
            k = np.ascontiguousarray(keys, np.uint8)
            v = np.ascontiguousarray(ivs, np.uint8)
            kp, vp, mem = k.ctypes.data, v.ctypes.data, N.MEM_HOST
            self.n = k.size // 10
        iv_bytes = v.numel() if isinstance(v, torch.Tensor) else v.size
        if iv_bytes != 8 * self.n:
            raise N.MickeyError(N.E_ARG, "ivs must hold 8 bytes per instance")
        self._keep = (k, v)
        self._h = N.check_ptr(self._L.grain_init_streams(
            kp, vp, self.n, mem, ctypes.c_void_p(self.stream.cuda_stream)))

    def generate(self, n_bits: int, layout="bytes", out: torch.Tensor | None = None):
        """Next n_bits of every stream into a device tensor (allocated if None)."""
        lay = _lay(layout)
        if out is None:
            if lay == N.LAYOUT_BITSLICED_U32:
                out = torch.empty(((self.n + 31) // 32, n_bits), dtype=torch.int32, device="cuda")
            else:
                out = torch.empty((self.n, (n_bits + 7) // 8), dtype=torch.uint8, device="cuda")
        need = self._L.grain_output_bytes(self.n, n_bits, lay)
        if need == 0 or out.numel() * out.element_size() < need:
            raise N.MickeyError(N.E_LAYOUT, "output tensor too small or layout invalid")
        self._L.grain_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream))
        N.check(self._L.grain_generate(self._h, n_bits, ctypes.c_void_p(out.data_ptr()), lay))
        return out

    def reset(self, keys, ivs):
        """Re-key every instance in place (device tensors or host arrays)."""
        if isinstance(keys, torch.Tensor) and keys.is_cuda:
            k, v, mem = keys.contiguous(), ivs.contiguous(), N.MEM_DEVICE
            kp, vp = k.data_ptr(), v.data_ptr()
        else:
            k, v = np.ascontiguousarray(keys, np.uint8), np.ascontiguousarray(ivs, np.uint8)
            kp, vp, mem = k.ctypes.data, v.ctypes.data, N.MEM_HOST
        self._keep = (k, v)
        self._L.grain_set_stream(self._h, ctypes.c_void_p(self.stream.cuda_stream))
        N.check(self._L.grain_reset_streams(self._h, kp, vp, mem))

    def sync(self):
        N.check(self._L.grain_sync(self._h))

    def position(self) -> int:
        return int(self._L.grain_position(self._h))

    def export_state(self) -> np.ndarray:
        st = np.zeros((self.n, 20), np.uint8)
        N.check(self._L.grain_export_state(self._h, st.ctypes.data))
        return st

    def free(self):
        if getattr(self, "_h", None):
            self._L.grain_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ops_per_clock(init: bool = False) -> int:
    return int(N.lib().grain_ops_per_clock(1 if init else 0))
