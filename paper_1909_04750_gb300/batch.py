"""Batched generation of ragged streams (C ABI: mickey_batch_*), with its
autotuner."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import _native as N
from .autotune import CACHE_PATH, _device_key, _load, _save, _lock


class Batch:
    """n streams with their own keystream lengths and IV lengths, planned
    once (packing, work queue order, CUDA graph) and run many times."""

    def __init__(self, n_bits, iv_lens=None, stream=None):
        self._L = N.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nb = np.ascontiguousarray(n_bits, np.uint64)
        self.n = int(nb.shape[0])
        self.n_bits = nb
        lens = None if iv_lens is None else np.ascontiguousarray(iv_lens, np.uint32)
        self._h = N.check_ptr(self._L.mickey_batch_create(
            lens.ctypes.data if lens is not None else None, nb.ctypes.data, self.n,
            ctypes.c_void_p(self.stream.cuda_stream)))
        self.output_bytes = int(self._L.mickey_batch_output_bytes(self._h))
        self.offsets = np.zeros(self.n, np.uint64)
        N.check(self._L.mickey_batch_offsets(self._h, self.offsets.ctypes.data))
        mx, tot = ctypes.c_uint64(), ctypes.c_uint64()
        N.check(self._L.mickey_batch_clocks(self._h, ctypes.byref(mx), ctypes.byref(tot)))
        self.max_clocks, self.total_clocks = int(mx.value), int(tot.value)

    def run(self, keys, ivs, out: torch.Tensor | None = None) -> torch.Tensor:
        """Generate every stream; keys/ivs are CUDA tensors or host arrays."""
        if out is None:
            out = torch.empty(self.output_bytes, dtype=torch.uint8, device="cuda")
        if isinstance(keys, torch.Tensor) and keys.is_cuda:
            k, v, mem = keys.contiguous(), ivs.contiguous(), N.MEM_DEVICE
            kp, vp = k.data_ptr(), v.data_ptr()
        else:
            k, v, mem = np.ascontiguousarray(keys, np.uint8), np.ascontiguousarray(ivs, np.uint8), \
                N.MEM_HOST
            kp, vp = k.ctypes.data, v.ctypes.data
        self._keep = (k, v)
        N.check(self._L.mickey_batch_run(self._h, kp, vp, ctypes.c_void_p(out.data_ptr()), mem))
        return out

    def sync(self):
        N.check(self._L.mickey_batch_sync(self._h))

    def set_config(self, unroll: int, blocks_per_sm: int, split_clocks: int = 0,
                   split_mode: int | None = None):
        N.check(self._L.mickey_batch_set_config(self._h, unroll, blocks_per_sm, split_clocks))
        if split_mode is not None and split_mode != self._L.mickey_batch_get_split_mode(self._h):
            N.check(self._L.mickey_batch_set_split_mode(self._h, split_mode))

    def get_config(self):
        u, b = ctypes.c_int(), ctypes.c_int()
        sc, sg = ctypes.c_uint64(), ctypes.c_uint32()
        N.check(self._L.mickey_batch_get_config(self._h, ctypes.byref(u), ctypes.byref(b),
                                                ctypes.byref(sc), ctypes.byref(sg)))
        return {"unroll": int(u.value), "blocks_per_sm": int(b.value),
                "split_clocks": int(sc.value), "split_groups": int(sg.value),
                "split_mode": int(self._L.mickey_batch_get_split_mode(self._h))}

    def rows(self, out: torch.Tensor):
        """Per-stream byte strings (host), for checking."""
        host = out.cpu().numpy()
        return [host[int(o):int(o) + (int(b) + 7) // 8] for o, b in zip(self.offsets, self.n_bits)]

    def free(self):
        if getattr(self, "_h", None):
            self._L.mickey_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def shape_key(batch: Batch) -> str:
    h = int(np.bitwise_xor.reduce(batch.n_bits * np.uint64(0x9E3779B97F4A7C15)))
    return "%s|batch|n=%d|clocks=%d/%d|h=%x" % (_device_key(), batch.n, batch.max_clocks,
                                                batch.total_clocks, h)


def _time(batch, keys, ivs, out) -> float:
    batch.run(keys, ivs, out)
    batch.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(batch.stream)
    batch.run(keys, ivs, out)
    e1.record(batch.stream)
    batch.sync()
    return e0.elapsed_time(e1)


def tune(batch: Batch, keys, ivs, out: torch.Tensor, refresh: bool = False) -> dict:
    """Pick the split threshold (groups longer than it run one per warp), the
    blocks per SM and the unroll depth by timing whole runs; cached per GPU
    and batch shape."""
    key = shape_key(batch)
    with _lock:
        hit = None if refresh else _load().get(key)
    if hit is not None:
        batch.set_config(hit["unroll"], hit["blocks_per_sm"], hit["split_clocks"],
                         hit.get("split_mode", N.BATCH_SPLIT_SHARED))
        return hit
    cands = []

    def trial(u, b, sc, mode=N.BATCH_SPLIT_SHARED):
        batch.set_config(u, b, sc, mode)
        c = dict(batch.get_config(), ms=_time(batch, keys, ivs, out))
        cands.append(c)
        return c

    # the longest groups bound the run (one clock after another), so the
    # split threshold and the warps per SM sub-partition (which share its
    # issue slots with the critical group's warp) are searched together
    mx = batch.max_clocks
    for b in (1, 2):
        # no split path at all only where the longest group is short
        for sc in ((0,) if mx <= 1 << 16 else ()) + (mx // 4, mx // 8, mx // 16, mx // 32,
                                                     mx // 64):
            trial(4, b, sc)
    best = min(cands, key=lambda c: c["ms"])
    trial(2, best["blocks_per_sm"], best["split_clocks"])
    best = min(cands, key=lambda c: c["ms"])
    if best["split_groups"]:
        trial(best["unroll"], best["blocks_per_sm"], best["split_clocks"], N.BATCH_SPLIT_OWN)
        best = min(cands, key=lambda c: c["ms"])
    batch.set_config(best["unroll"], best["blocks_per_sm"], best["split_clocks"],
                     best["split_mode"])
    entry = dict(best, candidates=cands)
    with _lock:
        cache = _load()
        cache[key] = entry
        _save(cache)
    return entry
