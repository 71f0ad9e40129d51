"""Run one workload shape through the library, for profilers.

    python -m paper_1909_04750_gb300.profile_case --n 1048576 --n-bits 2048 --layout bytes
    python -m paper_1909_04750_gb300.profile_case --case split --n 32 --n-bits 65536

``plain``: creates a handle for ``workloads.plain_scale(n)`` (device
inputs), then ``--reps`` times re-keys it and generates ``n_bits`` per
stream in ``layout`` (with ``--continue``, re-keys only before the first
generation, so that later launches clock no initialisation).  The launch configuration comes from the environment
(MICKEY_MODE, MICKEY_UNROLL, MICKEY_STAGE) or the library defaults, or with
``--autotune`` from the autotuner (as the benchmarks do; its trial launches
come first).

``split``: a batch of n streams of ``n_bits`` each whose groups all take the
one-warp-per-group path (split threshold 1 clock), run ``--reps`` times.

``batched``: the 100,000-stream ragged batch (seed 3), autotuned (cached),
replayed ``--reps`` times.

``lfsr``: Fibonacci LFSRs of degree 64 (x^64 + x^4 + x^3 + x + 1), n
instances x ``n_bits``, ``--reps`` times.

``crc8``: CRC-8 (0x1D, preset and final XOR 0xFF) of n messages of
``n_bits / 8`` bytes each (random, device-resident), ``--reps`` times.

``ragged``: a handle of n instances (seed 2) continues every stream by its
own length in one mickey_generate_ragged call, ``--reps`` times: every
length ``n_bits`` (``--spread 0``) or uniform in [n_bits - spread, n_bits].

``grain``: n Grain instances (seed 6) generate ``n_bits`` each in ``layout``
(bitsliced or bytes), ``--reps`` times.

``serve``: a server holding n streams serves one request of ``n_bits`` bits
per stream ``--reps`` times, each in one step of split groups only (the
split kernel launches one warp per group, so its counters come from the
working warps alone).
"""
import argparse

import torch

from . import workloads
from .build import build
from .streams import Streams


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--n-bits", type=int, default=2048)
    p.add_argument("--layout", default="bytes")
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--case", choices=("plain", "split", "serve", "crc8", "batched", "lfsr",
                                      "ragged", "grain"), default="plain")
    p.add_argument("--spread", type=int, default=0)
    p.add_argument("--autotune", action="store_true")
    p.add_argument("--continue", dest="cont", action="store_true")
    a = p.parse_args()
    build()
    if a.case == "batched":
        from .batch import Batch, tune
        s = workloads.batched()
        k, v = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
        b = Batch(s.n_bits, s.iv_lens)
        out = torch.empty(b.output_bytes, dtype=torch.uint8, device="cuda")
        print("config:", tune(b, k, v, out))
        for _ in range(a.reps):
            b.run(k, v, out)
        b.sync()
        print("ok", vars(a))
        return
    if a.case == "lfsr":
        from .lfsr import lfsr_generate
        g = torch.Generator(device="cuda").manual_seed(5)
        seeds = torch.randint(1, 1 << 62, (a.n,), dtype=torch.int64, device="cuda", generator=g)
        out = torch.empty((a.n_bits, (a.n + 31) // 32), dtype=torch.int32, device="cuda")
        for _ in range(a.reps):
            lfsr_generate(seeds, 64, 0b11011, a.n_bits, out=out)
        torch.cuda.synchronize()
        print("ok", vars(a))
        return
    if a.case == "crc8":
        from .lfsr import crc8
        g = torch.Generator(device="cuda").manual_seed(5)
        data = torch.randint(0, 256, (a.n, a.n_bits // 8), dtype=torch.uint8, device="cuda",
                             generator=g)
        for _ in range(a.reps):
            crc8(data, 0x1D, 0xFF, 0xFF)
        torch.cuda.synchronize()
        print("ok", vars(a))
        return
    if a.case == "serve":
        from .serve import Server
        s = workloads.plain_scale(a.n)
        srv = Server(a.n, split_quantum=a.n_bits, split_min_bits=0)
        reqs = [workloads.Request(0.0, i, s.keys[i].tobytes(), s.ivs[i].tobytes(), 80,
                                  a.n_bits // 8) for i in range(a.n)]
        for _ in range(a.reps):
            srv.run(reqs, realtime=False)
        torch.cuda.synchronize()
        srv.free()
        print("ok", vars(a))
        return
    if a.case == "grain":
        from .grain import GrainStreams
        s = workloads.grain_streams(a.n)
        st = GrainStreams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
        out = None
        for _ in range(a.reps):
            out = st.generate(a.n_bits, a.layout, out=out)
        st.sync()
        print("ok", vars(a))
        return
    if a.case == "ragged":
        import numpy as np
        s = workloads.plain_scale(a.n)
        st = Streams(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
        rng = np.random.default_rng(1)
        nb = np.full(a.n, a.n_bits, np.uint64)
        if a.spread:
            if not 0 < a.spread <= a.n_bits:
                raise SystemExit("--spread must be in [0, n_bits]")
            nb = rng.integers(a.n_bits - a.spread, a.n_bits + 1, a.n).astype(np.uint64)
        out = None
        for _ in range(a.reps):
            out, _ = st.generate_ragged(nb, a.layout, out=out)
        st.sync()
        print("ok", vars(a))
        return
    if a.case == "split":
        import numpy as np
        from .batch import Batch
        s = workloads.plain_scale(a.n)
        b = Batch(np.full(a.n, a.n_bits, np.uint64))
        b.set_config(4, 1, 1)
        k, v = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
        out = torch.empty(b.output_bytes, dtype=torch.uint8, device="cuda")
        for _ in range(a.reps):
            b.run(k, v, out)
        b.sync()
        print("ok", vars(a))
        return
    s = workloads.plain_scale(a.n)
    k, v = torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda()
    st = Streams(k, v)
    if a.autotune:
        from . import autotune
        from .streams import layout_id
        print("launch:", autotune.describe(autotune.tune(st, a.n_bits, layout_id(a.layout))))
    for rep in range(a.reps):
        if rep == 0 or not a.cont:
            st.reset(k, v)
        st.generate(a.n_bits, a.layout)
    st.sync()
    torch.cuda.synchronize()
    print("ok", vars(a))


if __name__ == "__main__":
    main()
