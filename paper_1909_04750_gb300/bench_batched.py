"""Benchmark of the batched workload: 100,000 streams, keystream lengths
log-uniform in [2^10, 2^22] bits, IV lengths in {0, 16, ..., 80}, seed 3, in
one persistent launch replayed from a CUDA graph.

    python -m paper_1909_04750_gb300.bench_batched [--runs K] [--n N]

Prints one JSON line: Gbit/s over all streams, and the two lower bounds on a
run's time -- the work at the plain kernel's measured rate, and the critical
path (the longest group's clocks at the measured time per clock of a group
clocked alone by one warp; MICKEY has no jump-ahead, so a stream's bits are
produced one clock after another).

With --steady K it also runs K batches back to back, round-robin over
--pipeline handles on their own CUDA streams, so that a batch's groups start
on the SMs the previous batches' shorter groups have left while their
longest groups still run: the steady-state rate of a stream of batches,
which the critical path of a single batch does not bound.
"""
import argparse
import json
import statistics

import numpy as np
import torch

from . import _native as N
from . import workloads
from .batch import Batch, tune
from .build import build
from .clocks import ClockSampler
from .streams import Streams


def lone_split_ns_per_clock(n_bits: int = 1 << 18) -> float:
    """Time per clock of one 32-lane group clocked alone by one warp."""
    s = workloads.plain_scale(32)
    b = Batch(np.full(32, n_bits, np.uint64))
    b.set_config(4, 1, 1)
    k, v = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
    out = torch.empty(b.output_bytes, dtype=torch.uint8, device="cuda")
    b.run(k, v, out)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.run(k, v, out)
    e1.record(b.stream)
    b.sync()
    b.free()
    return e0.elapsed_time(e1) * 1e6 / n_bits


def lone_group_ns_per_clock(n_bits: int = 1 << 16) -> float:
    """Time per clock of one 32-lane group alone on the GPU."""
    s = workloads.plain_scale(32)
    st = Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    out = st.generate(n_bits, "bitsliced")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st.generate(n_bits, "bitsliced", out=out)
    e1.record()
    torch.cuda.synchronize()
    st.free()
    return e0.elapsed_time(e1) * 1e6 / n_bits


def measure(runs: int = 3, n: int = workloads.BATCHED["n"], steady: int = 12,
            pipeline: int = 0, steady_split: int = 0, plain_gbit_s=None, verify=None) -> dict:
    """Time one replay of the batched workload `runs` times (and, with
    `steady`, batches back to back); `verify(streamset, batch, out)` checks
    the last replay's output and returns a dict for the line."""
    s = workloads.batched(n)
    keys, ivs = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
    b = Batch(s.n_bits, s.iv_lens)
    out = torch.empty(b.output_bytes, dtype=torch.uint8, device="cuda")
    tuned = tune(b, keys, ivs, out)
    b.run(keys, ivs, out)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    sampler = ClockSampler(torch.cuda.current_device()).start()
    for _ in range(runs):
        e0.record(b.stream)
        b.run(keys, ivs, out)
        e1.record(b.stream)
        b.sync()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    ms = statistics.mean(times)
    bits = int(s.n_bits.sum())
    t_thread = lone_group_ns_per_clock()
    t_clk = lone_split_ns_per_clock()
    crit_ms = b.max_clocks * t_clk * 1e-6
    line = {
        "metric": "batched keystream Gbit/s (100k ragged streams, one persistent launch)",
        "value": bits / (ms * 1e-3) / 1e9, "unit": "Gbit/s", "ms_per_run": ms,
        "ms_runs": times, "runs": runs, "streams": b.n, "keystream_bits": bits,
        "groups_clocks_total": b.total_clocks, "longest_group_clocks": b.max_clocks,
        "lone_split_ns_per_clock": t_clk, "lone_thread_group_ns_per_clock": t_thread,
        "critical_path_ms": crit_ms, "frac_of_critical_path": crit_ms / ms,
        "bound": "critical path: the longest group's clocks one after another",
        "config": {"workload": "batched: 100,000 streams, lengths log-uniform in "
                               "[2^10, 2^22] bits, IV lengths {0,16,...,80}, seed 3",
                   "unroll": tuned["unroll"], "blocks_per_sm": tuned["blocks_per_sm"],
                   "split_clocks": tuned["split_clocks"],
                   "split_groups": tuned.get("split_groups")},
        "clocks": clocks,
    }
    if plain_gbit_s:
        line["work_bound_ms"] = bits / (plain_gbit_s * 1e9) * 1e3
        line["vs_plain"] = line["value"] / plain_gbit_s
    if verify is not None:
        line["verified"] = verify(s, b, out)
    max_clocks = b.max_clocks
    b.free()
    del out
    torch.cuda.empty_cache()
    if steady:
        sampler = ClockSampler(torch.cuda.current_device()).start()
        if steady_split or pipeline:
            cfg = dict(tuned)
            if steady_split:
                cfg["split_clocks"] = max_clocks // steady_split
            line["steady"] = steady_state(s, keys, ivs, cfg, steady, pipeline or 4)
        else:
            line["steady"] = steady_sweep(s, keys, ivs, tuned, max_clocks)
        line["steady"]["clocks"] = sampler.stop()
        line["steady"]["what"] = ("batches of the same workload back to back, round-robin over "
                                  "`pipeline` handles on their own CUDA streams")
        if plain_gbit_s:
            line["steady"]["vs_plain"] = line["steady"]["gbit_s"] / plain_gbit_s
    return line


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--runs", type=int, default=3)
    p.add_argument("--n", type=int, default=workloads.BATCHED["n"])
    p.add_argument("--plain-gbit-s", type=float, default=None,
                   help="plain-workload throughput for the work bound")
    p.add_argument("--steady", type=int, default=0, help="batches for the steady-state rate")
    p.add_argument("--pipeline", type=int, default=0,
                   help="handles (CUDA streams) in flight (0: sweep 4 and 8 with the split "
                        "arrangements)")
    p.add_argument("--steady-split", type=int, default=0,
                   help="split threshold for the steady-state run as max_clocks / this "
                        "(0: the tuned one)")
    a = p.parse_args()
    build()
    print(json.dumps(measure(a.runs, a.n, a.steady, a.pipeline, a.steady_split,
                             a.plain_gbit_s)), flush=True)


def steady_state(s, keys, ivs, cfg, k: int, pipeline: int) -> dict:
    """K batches back to back over `pipeline` handles on their own streams."""
    streams = [torch.cuda.Stream() for _ in range(pipeline)]
    hs = [Batch(s.n_bits, s.iv_lens, stream=st) for st in streams]
    outs = [torch.empty(hs[0].output_bytes, dtype=torch.uint8, device="cuda") for _ in hs]
    for h, o in zip(hs, outs):
        h.set_config(cfg["unroll"], cfg["blocks_per_sm"], cfg["split_clocks"],
                     cfg.get("split_mode", N.BATCH_SPLIT_SHARED))
        h.run(keys, ivs, o)                              # capture + warm-up
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    start.record()
    for st in streams:
        st.wait_event(start)
    done = []
    for j in range(k):
        h = hs[j % pipeline]
        h.run(keys, ivs, outs[j % pipeline])
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(h.stream)
        done.append(ev)
    torch.cuda.synchronize()
    ms = max(start.elapsed_time(e) for e in done)
    for h in hs:
        h.free()
    del outs
    torch.cuda.empty_cache()
    bits = int(s.n_bits.sum()) * k
    return {"batches": k, "pipeline": pipeline, "ms": ms, "ms_per_batch": ms / k,
            "gbit_s": bits / (ms * 1e-3) / 1e9, "split_clocks": cfg["split_clocks"],
            "split_mode": ["shared", "own"][cfg.get("split_mode", N.BATCH_SPLIT_SHARED)],
            "blocks_per_sm": cfg["blocks_per_sm"], "unroll": cfg["unroll"]}


def steady_sweep(s, keys, ivs, tuned, max_clocks: int, rounds: int = 3) -> dict:
    """The steady-state rate over a few launch arrangements (split mode,
    split threshold, batches in flight); returns the best with every
    candidate."""
    cands = []
    for mode in (N.BATCH_SPLIT_SHARED, N.BATCH_SPLIT_OWN):
        for sc in sorted({tuned["split_clocks"], max_clocks // 16}):
            for pipe in (4, 8):
                cfg = dict(tuned, split_clocks=sc, split_mode=mode)
                cands.append(steady_state(s, keys, ivs, cfg, rounds * pipe, pipe))
    best = dict(max(cands, key=lambda c: c["gbit_s"]))
    best["candidates"] = [{k: c[k] for k in ("gbit_s", "split_mode", "split_clocks", "pipeline")}
                          for c in cands]
    return best


if __name__ == "__main__":
    main()
