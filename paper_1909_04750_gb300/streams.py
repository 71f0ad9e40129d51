"""Torch-facing wrapper of the C ABI: device buffers and streams from torch,
all keystream work in libmickey's kernels."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N

LAYOUTS = {"bitsliced": N.LAYOUT_BITSLICED_U32, "bytes": N.LAYOUT_BYTES,
           "u32": N.LAYOUT_U32, "u32_f32": N.LAYOUT_U32_F32}


def layout_id(layout) -> int:
    return LAYOUTS[layout] if isinstance(layout, str) else int(layout)


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def output_shape(n: int, n_bits: int, layout) -> tuple:
    """Shape and dtype of one call's output tensor."""
    lay = layout_id(layout)
    if lay == N.LAYOUT_BITSLICED_U32:
        return ((n + 31) // 32, n_bits), torch.int32
    if lay == N.LAYOUT_BYTES:
        return (n, (n_bits + 7) // 8), torch.uint8
    if lay == N.LAYOUT_U32:
        return (n, n_bits // 32), torch.int32
    return (2, n, n_bits // 32), torch.int32   # [0] u32 words, [1] f32 bits


class Streams:
    """n independent MICKEY 2.0 keystreams, bitsliced on one GPU.

    keys, ivs: uint8 [n, 10] (torch CUDA tensors or host arrays);
    iv_lens: uint32/int32 [n] or None (80 bits each).
    """

    def __init__(self, keys, ivs, iv_lens=None, stream=None, _handle=None, _n=None):
        self._L = N.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if _handle is not None:
            self._h = _handle
            self.n = _n
            return
        args, mem, self._keep = self._marshal(keys, ivs, iv_lens)
        self.n = int(args[3])
        self._h = N.check_ptr(self._L.mickey_init_streams_ex(
            args[0], args[1], args[2], args[3], mem, _stream_ptr(self.stream)))

    @staticmethod
    def _marshal(keys, ivs, iv_lens):
        if isinstance(keys, torch.Tensor) and keys.is_cuda:
            keys = keys.contiguous().view(torch.uint8)
            ivs = ivs.contiguous().view(torch.uint8)
            n = keys.numel() // 10
            lens = None
            if iv_lens is not None:
                lens = iv_lens.to(device=keys.device, dtype=torch.int32).contiguous()
            keep = (keys, ivs, lens)
            return ((keys.data_ptr(), ivs.data_ptr(), lens.data_ptr() if lens is not None else None,
                     n), N.MEM_DEVICE, keep)
        k = np.ascontiguousarray(keys, np.uint8)
        v = np.ascontiguousarray(ivs, np.uint8)
        n = k.size // 10
        lens = None if iv_lens is None else np.ascontiguousarray(iv_lens, np.uint32)
        keep = (k, v, lens)
        return ((k.ctypes.data, v.ctypes.data, lens.ctypes.data if lens is not None else None,
                 n), N.MEM_HOST, keep)

    # -- keystream -----------------------------------------------------------------
    def generate(self, n_bits: int, layout="bytes", out: torch.Tensor | None = None):
        """Next n_bits of every stream into a device tensor (allocated if None)."""
        lay = layout_id(layout)
        if out is None:
            shape, dtype = output_shape(self.n, n_bits, lay)
            out = torch.empty(shape, dtype=dtype, device="cuda")
        need = self._L.mickey_output_bytes(self.n, n_bits, lay)
        if need == 0 or out.numel() * out.element_size() < need:
            raise N.MickeyError(N.E_LAYOUT, "output tensor too small or layout invalid")
        self._L.mickey_set_stream(self._h, _stream_ptr(self.stream))
        N.check(self._L.mickey_generate(self._h, n_bits, ctypes.c_void_p(out.data_ptr()), lay))
        return out

    def generate_ragged(self, n_bits, layout="bytes", out: torch.Tensor | None = None,
                        offsets=None):
        """Stream i continues by n_bits[i] bits in one launch.  Returns the
        output tensor (packed, allocated here when `out` is None) and the
        byte offsets used (per stream, or per group for "bitsliced")."""
        lay = layout_id(layout)
        nb = np.ascontiguousarray(n_bits, np.uint64)
        if nb.shape != (self.n,):
            raise N.MickeyError(N.E_ARG, "n_bits needs one value per stream")
        if offsets is None:
            total = int(self._L.mickey_ragged_output_bytes(self.n, nb.ctypes.data, lay))
            if total == 0 and nb.any():
                raise N.MickeyError(N.E_ARG, "lengths invalid for this layout (u32 needs multiples "
                                               "of 32; at most 2^34 bits per call)")
            if out is None:
                out = torch.empty(max(total, 16), dtype=torch.uint8, device="cuda")
            elif out.numel() * out.element_size() < total:
                raise N.MickeyError(N.E_ARG, "output tensor too small")
            offs = None
        else:
            offs = np.ascontiguousarray(offsets, np.uint64)
        self._L.mickey_set_stream(self._h, _stream_ptr(self.stream))
        N.check(self._L.mickey_generate_ragged(self._h, nb.ctypes.data,
                                               ctypes.c_void_p(out.data_ptr()),
                                               offs.ctypes.data if offs is not None else None,
                                               lay))
        if offs is None:
            offs = packed_offsets(nb, lay)
        return out, offs

    def generate_host(self, n_bits: int, layout="bytes", out: torch.Tensor | None = None):
        """Next n_bits into a host tensor (pinned if allocated here)."""
        lay = layout_id(layout)
        if out is None:
            shape, dtype = output_shape(self.n, n_bits, lay)
            out = torch.empty(shape, dtype=dtype, pin_memory=True)
        need = self._L.mickey_output_bytes(self.n, n_bits, lay)
        if need == 0 or out.numel() * out.element_size() < need:
            raise N.MickeyError(N.E_LAYOUT, "output tensor too small or layout invalid")
        self._L.mickey_set_stream(self._h, _stream_ptr(self.stream))
        N.check(self._L.mickey_generate_host(self._h, n_bits, ctypes.c_void_p(out.data_ptr()),
                                             lay))
        return out

    def reset(self, keys, ivs, iv_lens=None):
        args, mem, self._keep = self._marshal(keys, ivs, iv_lens)
        if int(args[3]) != self.n:
            raise N.MickeyError(N.E_ARG, "reset needs the same number of streams")
        self._L.mickey_set_stream(self._h, _stream_ptr(self.stream))
        N.check(self._L.mickey_reset_streams(self._h, args[0], args[1], args[2], mem))

    def sync(self):
        N.check(self._L.mickey_sync(self._h))

    def position(self, i: int = 0) -> int:
        return int(self._L.mickey_position(self._h, i))

    # -- checkpoint ----------------------------------------------------------------
    def export_state(self):
        states = np.zeros((self.n, 26), np.uint8)
        pos = np.zeros(self.n, np.uint64)
        N.check(self._L.mickey_export_state(self._h, states.ctypes.data, pos.ctypes.data))
        return states, pos

    @classmethod
    def import_state(cls, states, positions=None, stream=None):
        L = N.lib()
        st = np.ascontiguousarray(states, np.uint8).reshape(-1, 26)
        pos = None if positions is None else np.ascontiguousarray(positions, np.uint64)
        stream = stream if stream is not None else torch.cuda.current_stream()
        h = N.check_ptr(L.mickey_import_state(st.ctypes.data,
                                              pos.ctypes.data if pos is not None else None,
                                              st.shape[0], _stream_ptr(stream)))
        return cls(None, None, stream=stream, _handle=h, _n=st.shape[0])

    def free(self):
        if getattr(self, "_h", None):
            self._L.mickey_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def packed_offsets(n_bits, layout) -> np.ndarray:
    """Byte offsets of the packed output of a ragged call: per stream for the
    row layouts, per 32-lane group for the bitsliced layout."""
    nb = np.asarray(n_bits, np.uint64).astype(np.int64)
    lay = layout_id(layout)
    if lay == N.LAYOUT_BITSLICED_U32:
        pad = np.zeros(-nb.size % 32, np.int64)
        sizes = 4 * np.concatenate([nb, pad]).reshape(-1, 32).max(axis=1)
    elif lay == N.LAYOUT_U32:
        sizes = nb // 8
    else:
        sizes = (nb + 7) // 8
    return np.concatenate(([0], np.cumsum(sizes)[:-1])).astype(np.uint64)


def tables() -> np.ndarray:
    """The kernels' compile-time tables as [5, 100] 0/1 (RTAPS, COMP0, COMP1,
    FB0, FB1)."""
    m = (ctypes.c_uint32 * 20)()
    N.lib().mickey_tables(m)
    words = np.frombuffer(bytes(m), np.uint32).reshape(5, 4)
    bits = np.zeros((5, 100), np.uint8)
    for i in range(100):
        bits[:, i] = (words[:, i // 32] >> np.uint32(i % 32)) & 1
    return bits


def ops_per_clock(mixing: bool = False) -> int:
    return int(N.lib().mickey_ops_per_clock(1 if mixing else 0))
