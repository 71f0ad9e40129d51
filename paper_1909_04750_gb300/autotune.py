"""Autotuner for the keystream kernel's launch configuration.

For a (GPU, instance count, bits per call, layout) the library's
``mickey_tune`` times every compiled configuration -- grid, paired or
two-block persistent launch, 2 or 4 clocks per inner step, and the output
tile: direct 4-byte row stores or rows staged 2, 4 or 8 tiles deep (8-, 16-
or 32-byte row chunks) -- on the handle's own streams (state saved and
restored) and keeps the fastest; among candidates within 1 % of it the
deepest row staging wins (whole 32-byte sectors: the least DRAM traffic at
the same speed).  The
choice is cached in a JSON file next to the built library so later handles
of the same shape reuse it without timing.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

from . import _native as N

CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                          "tune_cache.json")
MODE_NAMES = {N.MODE_AUTO: "auto", N.MODE_GRID: "grid", N.MODE_PERSISTENT: "persistent",
              N.MODE_PERSISTENT2: "persistent x2"}
_lock = threading.Lock()


def _device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|sm%d" % (p.name, p.multi_processor_count)


def _load() -> dict:
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(cache: dict) -> None:
    os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
    tmp = CACHE_PATH + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE_PATH)


def shape_key(n: int, n_bits: int, layout: int) -> str:
    return "%s|n=%d|bits=%d|layout=%d" % (_device_key(), n, n_bits, layout)


def tune(streams, n_bits: int, layout: int, refresh: bool = False) -> dict:
    """Apply the best configuration for this shape to `streams` (timing it on
    the first use), and return {"mode", "unroll", "stage", "ms", "candidates"}."""
    L = N.lib()
    key = shape_key(streams.n, n_bits, layout)
    with _lock:
        cache = _load()
        hit = None if refresh else cache.get(key)
    if hit is not None:
        N.check(L.mickey_set_config(streams._h, layout, hit["mode"], hit["unroll"], hit["stage"]))
        return hit
    res = (N.TuneResult * 32)()
    count = ctypes.c_int(0)
    N.check(L.mickey_tune(streams._h, n_bits, layout, res, 32, ctypes.byref(count)))
    cands = [{"mode": MODE_NAMES[r.mode], "unroll": r.unroll, "stage": r.stage,
              "ms": float(r.ms)} for r in res[: count.value]]
    mode, unroll, stage = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    N.check(L.mickey_get_config(streams._h, layout, ctypes.byref(mode), ctypes.byref(unroll),
                                ctypes.byref(stage)))
    chosen = [c["ms"] for c in cands if (c["mode"], c["unroll"], c["stage"]) ==
              (MODE_NAMES[mode.value], unroll.value, stage.value)]
    best = chosen[0] if chosen else (min(c["ms"] for c in cands) if cands else None)
    entry = {"mode": mode.value, "unroll": unroll.value, "stage": stage.value, "ms": best,
             "candidates": cands}
    with _lock:
        cache = _load()
        cache[key] = entry
        _save(cache)
    return entry


def describe(entry: dict) -> str:
    st = entry["stage"]
    default = {N.MODE_PERSISTENT: 8, N.MODE_AUTO: 8}.get(entry["mode"], 4)
    depth = default if st == 1 else st
    rows = "direct rows" if not st else ("staged rows" if depth == default
                                         else "rows staged %d tiles" % depth)
    return "%s, %d clocks/step, %s" % (MODE_NAMES.get(entry["mode"], "?"), entry["unroll"], rows)
