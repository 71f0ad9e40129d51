"""Benchmark of the served workload: Poisson arrivals at 10^4 requests/s for
30 s (seed 4), 70 % of requests continuing a resident stream, request
lengths log-uniform in [1 KiB, 64 MiB] of keystream, device-memory budget
16 GiB for stream states plus in-flight response chunks.

    python -m paper_1909_04750_gb300.bench_served [--duration S] [--saturate]

Prints one JSON line: p50 / p99 / mean latency (from a request's arrival to
the end of the step that produced its last byte), aggregate Gbit/s over the
run (served bits / time to the last completion), offered Gbit/s, and the
latency bound of the longest request (its bits at the split path's
measured time per clock: a stream's bits come out one clock after another).
With --saturate every request is handed over at t = 0, which measures the
server's capacity instead of its behaviour at the offered load.

Beside the measured figures it prints the sequential bound of the trace: each
request starting at its arrival or when the previous request of its stream
ends, whichever is later, and taking its bits times the measured time per
clock of one group clocked alone by one warp of the server's split kernel,
with unlimited capacity.
Requests of one stream continue one keystream, so they cannot overlap, and
MICKEY has no jump-ahead, so no schedule beats this at that time per clock.
"""
import argparse
import json

import numpy as np
import torch

from . import workloads
from .build import build
from .clocks import ClockSampler
from .serve import Server


def lone_serve_ns_per_clock(n_bits: int = 1 << 18) -> float:
    """Time per clock of one 32-lane group alone in the server's split
    kernel: one step of 32 fresh streams, n_bits each (the stream setup is
    in the timed span too; it is under 0.1 % of it)."""
    s = workloads.plain_scale(32)
    reqs = [workloads.Request(0.0, i, s.keys[i].tobytes(), s.ivs[i].tobytes(), 80, n_bits // 8)
            for i in range(32)]
    best = float("inf")
    for _ in range(2):
        srv = Server(32, split_quantum=n_bits, split_min_bits=0)
        srv.run(reqs, realtime=False)
        best = min(best, srv.stats["wall_ms"])
        srv.free()
    return best * 1e6 / n_bits


def sequential_bound(reqs, ns_per_clock: float, saturate: bool):
    """Finish time (s) of every request under the sequential bound."""
    free = {}
    fin = np.empty(len(reqs))
    for j, r in enumerate(reqs):
        start = max(0.0 if saturate else r.arrival_s, free.get(r.stream_id, 0.0))
        fin[j] = start + 8 * r.n_bytes * ns_per_clock * 1e-9
        free[r.stream_id] = fin[j]
    return fin


def measure(duration: float = 30.0, rate: float = 1e4, saturate: bool = False,
            quantum: int = 1 << 15, split_quantum: int = 1 << 17, split_min_bits: int = 0,
            max_split_groups=None, plain_gbit_s=None, verify=None) -> dict:
    """Serve the trace; `verify(server, requests, keyset)` checks the served
    streams after the run and returns a dict for the line."""
    reqs, keyset = workloads.served_trace(seed=4, rate_per_s=rate, duration_s=duration)
    bits = np.array([8 * r.n_bytes for r in reqs], np.int64)
    srv = Server(max(keyset.n, 1), budget_bytes=16 << 30, quantum=quantum,
                 split_quantum=split_quantum, split_min_bits=split_min_bits,
                 max_split_groups=max_split_groups)
    t_clk = lone_serve_ns_per_clock()
    sampler = ClockSampler(torch.cuda.current_device()).start()
    srv.run(reqs, realtime=not saturate)
    clocks = sampler.stop()
    st = dict(srv.stats)
    fin = sequential_bound(reqs, t_clk, saturate)
    lat = fin - (0.0 if saturate else np.array([r.arrival_s for r in reqs]))
    line = {
        "metric": "served keystream: p50/p99 latency and aggregate Gbit/s",
        "mode": "saturation (all requests at t=0)" if saturate else "Poisson arrivals",
        "requests": len(reqs), "streams": keyset.n,
        "continue_fraction": float(1 - keyset.n / max(len(reqs), 1)),
        "offered_gbit_s": float(bits.sum()) / duration / 1e9,
        "longest_request_bits": int(bits.max()),
        **st,
        "config": {"workload": "served: Poisson 10^4 requests/s for %g s, seed 4, 70 %% "
                               "continuing a resident stream, 1 KiB - 64 MiB per request, "
                               "16 GiB budget" % duration,
                   "quantum": quantum, "split_quantum": split_quantum,
                   "split_min_bits": split_min_bits,
                   "max_split_groups": srv.max_split_groups, "budget_bytes": 16 << 30},
        "clocks": clocks,
    }
    line["bound"] = {"ns_per_clock": t_clk, "end_ms": float(fin.max()) * 1e3,
                     "gbit_s": float(bits.sum()) / float(fin.max()) / 1e9,
                     "p50_ms": float(np.percentile(lat, 50)) * 1e3,
                     "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                     "what": "sequential bound: each request starts at its arrival or when "
                             "its stream's previous request ends, at the split kernel's "
                             "time per clock alone, unlimited capacity"}
    if plain_gbit_s:
        line["busy_vs_plain"] = st["busy_gbit_s"] / plain_gbit_s
    if verify is not None:
        line["verified"] = verify(srv, reqs, keyset)
    srv.free()
    torch.cuda.empty_cache()
    return line


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--duration", type=float, default=30.0)
    p.add_argument("--rate", type=float, default=1e4)
    p.add_argument("--saturate", action="store_true")
    p.add_argument("--quantum", type=int, default=1 << 15)
    p.add_argument("--split-quantum", type=int, default=1 << 17)
    p.add_argument("--split-min-bits", type=int, default=0)
    p.add_argument("--max-split-groups", type=int, default=None)
    a = p.parse_args()
    build()
    print(json.dumps(measure(a.duration, a.rate, a.saturate, a.quantum, a.split_quantum,
                             a.split_min_bits, a.max_split_groups)), flush=True)


if __name__ == "__main__":
    main()
