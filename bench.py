"""Keystream benchmark: bitsliced MICKEY 2.0 on GB300.

One step = the whole hot path over one batch of synthetic input: key/IV
loading + 100 mixing preclocks (two kernels) and keystream generation with
the un-bitslicing transpose to row-major bytes (one kernel), for the
plain-at-scale workload: 2^20 instances (32,768 bitsliced groups), 80-bit keys
and IVs from splitmix64 seed 2, 2^14 keystream bits per instance (2 GiB).

Prints one JSON line (rank 0).  ``--impl reference`` times the scalar CPU
oracle instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "keystream Gbit/s on 1 GB300 (bit-exact), % of int-LOP roofline; served p50/p99"
WORKLOAD = ("plain_scale: 2^20 MICKEY 2.0 instances (32768 bitsliced groups), 80-bit keys "
            "and IVs from splitmix64 seed 2, 100 mixing preclocks, 2^14 keystream bits "
            "per instance, row-major bytes output (2 GiB)")
# Integer-logic peak of the GB300: 152 SMs x 64 LOP3 results per SM per
# clock (measured with mickey_probe_lop3: 63.2-64.0 per SM-cycle over 1-8
# resident blocks) x the maximum SM clock of 2070 MHz = 20.14 T ops/s.
N_SM = 152
SM_MAX_MHZ = 2070.0
LOP3_PER_SM_CLK = 64.0

# DRAM traffic of one keystream launch of the plain workload at scale
# (dram__bytes_read.sum + dram__bytes_write.sum, one-pass ncu capture of the
# full-size launch in the autotuned configuration: 86.6 MB read + 2.189 GB
# written; algorithmic 2.20 GB = 2 GiB of output + the 26.2 MB state read
# and written).  It stands for the kernel sources it was measured on (their
# digest) and that launch configuration only; otherwise traffic is null.
KEYSTREAM_TRAFFIC = {"digest": "9321f55be9be5d8a", "launch": "persistent, 4 clocks/step, staged rows",
                     "bytes_per_launch": 2275657472}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--n-bits", type=int, default=1 << 14)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        load = [x for x in sm if x > 0.5 * (max(sm) if sm else 1)]
        out.update(sm_mhz=statistics.median(load) if load else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons),
                   samples=len(rows))
        return out


def cpu_baseline(n_bits: int, seconds: float = 3.0):
    """The scalar oracle on all host cores, on a bounded sample of the workload."""
    import oracle
    from paper_1909_04750_gb300 import workloads
    cores = os.cpu_count() or 1
    count = 4 * cores
    elapsed, total_bits = 0.0, 0
    while True:
        s = workloads.plain_scale(count)
        t = time.perf_counter()
        oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, n_bits, threads=cores)
        elapsed = time.perf_counter() - t
        total_bits = count * n_bits
        if elapsed >= seconds or count >= (1 << 20):
            break
        count = int(count * max(2.0, 1.2 * seconds / max(elapsed, 1e-3)))
    # one core: the same oracle on one thread, a smaller sample
    one = max(8, min(count // cores, 256))
    s1 = workloads.plain_scale(one)
    t = time.perf_counter()
    oracle.batch_bytes(s1.keys, s1.ivs, s1.iv_lens, n_bits, threads=1)
    one_core = one * n_bits / (time.perf_counter() - t) / 1e9
    return {"value": total_bits / elapsed / 1e9, "unit": "Gbit/s", "cores": cores,
            "kind": "oracle", "one_core_gbit_s": one_core,
            "sample": "%d instances x %d keystream bits (+260 init clocks each) of the same "
                      "workload, scalar C oracle, one instance per task; one core: %d "
                      "instances on one thread" % (count, n_bits, one)}


def run_reference(args, rank, world):
    """Reference arm: the scalar CPU oracle, timed on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_1909_04750_gb300 import workloads
    cores = os.cpu_count() or 1
    count = 64 * cores            # instances per step (bounded sample)
    s = workloads.plain_scale(count)
    for _ in range(args.warmup):
        oracle.batch_bytes(s.keys[:cores], s.ivs[:cores], s.iv_lens[:cores], args.n_bits,
                           threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, args.n_bits, threads=cores)
    dt = time.perf_counter() - t
    value = count * args.n_bits * args.steps / dt / 1e9
    sample = ("%d of the 2^20 instances x %d keystream bits per step, scalar C oracle on "
              "%d host threads" % (count, args.n_bits, cores))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gbit/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sampled_instances_per_step": count},
        "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_1909_04750_gb300 import _native as N
    from paper_1909_04750_gb300 import autotune, shard, workloads
    from paper_1909_04750_gb300.build import build, sources_digest
    from paper_1909_04750_gb300.streams import Streams, ops_per_clock

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # one rank compiles (if anything is stale) while the others wait, so no
    # two processes write the same build directory
    if rank == 0:
        build()
    shard.barrier()
    build()
    n, n_bits = args.n, args.n_bits
    # weak scaling: rank r runs its own 2^20 instances (draws offset by rank)
    s = shard.plain_shard(rank, world, n, n_bits)
    keys = torch.from_numpy(s.keys).cuda()
    ivs = torch.from_numpy(s.ivs).cuda()
    lens = torch.from_numpy(s.iv_lens.astype(np.int32)).cuda()
    stream = torch.cuda.current_stream()
    st = Streams(keys, ivs, lens)
    out = torch.empty((n, n_bits // 8), dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)

    # launch configuration from the autotuner (timed once per shape, cached)
    tuned = autotune.tune(st, n_bits, N.LAYOUT_BYTES)
    tuned_bs = autotune.tune(st, n_bits, N.LAYOUT_BITSLICED_U32)

    def step(layout="bytes", o=out):
        st.reset(keys, ivs, lens)
        st.generate(n_bits, layout, out=o)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    shard.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                           # evict L2 between steps
        ev[k][0].record(stream)
        st.reset(keys, ivs, lens)                       # load + preclock kernels
        ev[k][1].record(stream)
        st.generate(n_bits, "bytes", out=out)           # keystream + transpose kernel
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    shard.barrier()
    clocks = sampler.stop()
    st.sync()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    ks_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    total_ms = shard.max_over_ranks(sum(step_ms))
    bits_per_step = n * n_bits * world
    value = bits_per_step * args.steps / (total_ms * 1e-3) / 1e9

    # secondary: bitsliced-u32 layout, same step otherwise
    out_bs = torch.empty(((n + 31) // 32, n_bits), dtype=torch.int32, device="cuda")
    for _ in range(2):
        step("bitsliced", out_bs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bs_ms = 0.0
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e0.record(stream)
        step("bitsliced", out_bs)
        e1.record(stream)
        torch.cuda.synchronize()
        bs_ms += e0.elapsed_time(e1)
    bs_value = n * n_bits * args.steps / (bs_ms * 1e-3) / 1e9
    del out_bs

    # roofline of the dominant kernel (keystream + transpose)
    groups = (n + 31) // 32
    ops = groups * n_bits * ops_per_clock(False)
    ks_avg_s = statistics.mean(ks_ms) * 1e-3
    achieved = ops / ks_avg_s / 1e12
    peak = N_SM * LOP3_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    init_ops = groups * 260 * ops_per_clock(True)
    whole_ops = ops + init_ops
    alg_bytes = n * n_bits // 8 + 2 * groups * 200 * 4        # output + state in and out
    traffic = None
    if (sources_digest() == KEYSTREAM_TRAFFIC["digest"]
            and autotune.describe(tuned) == KEYSTREAM_TRAFFIC["launch"]
            and (n, n_bits) == (1 << 20, 1 << 14)):
        traffic = KEYSTREAM_TRAFFIC["bytes_per_launch"]

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty((n, n_bits // 8), dtype=torch.uint8, pin_memory=True)
        # the step's inputs live in pinned host memory (copied in every step)
        pk = torch.from_numpy(s.keys).pin_memory()
        pv = torch.from_numpy(s.ivs).pin_memory()
        pl = torch.from_numpy(s.iv_lens.astype(np.uint32).view(np.int32)).pin_memory()
        hk, hv, hl = pk.numpy(), pv.numpy(), pl.numpy().view(np.uint32)

        h = Streams(hk, hv, hl)            # host-memory inputs

        def e2e_step():
            h.reset(hk, hv, hl)              # H2D of keys/IVs/lengths + init kernels
            h.generate_host(n_bits, "bytes", out=host_out)   # chunked generate + D2H
        e2e_step()
        shard.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = shard.max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": bits_per_step * args.steps / dt / 1e9, "unit": "Gbit/s",
               "h2d_bytes_per_step": int(hk.nbytes + hv.nbytes + hl.nbytes) * world,
               "d2h_bytes_per_step": int(host_out.numel()) * world}
        h.free()
        del host_out

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(n_bits)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": n, "bits_per_instance": n_bits,
                       "layout": "bytes", "l2": "512 MiB buffer written between timed steps; "
                       "output 2 GiB > L2", "launch": autotune.describe(tuned),
                       "launch_bitsliced": autotune.describe(tuned_bs)},
            "pct_int_lop_roofline": 100.0 * (whole_ops / (total_ms / args.steps * 1e-3) / 1e12)
                                    / peak,
            "bitsliced_u32_gbit_s": bs_value,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_unit": "bytes per launch", "algorithmic_bytes": alg_bytes,
                         "kernel": "keystream kernel, bytes layout (%s)" % autotune.describe(tuned),
                         "ops_per_clock_per_group": ops_per_clock(False),
                         "peak_basis": "%d SMs x %g LOP3/SM/clk (mickey_probe_lop3) x %g MHz"
                                       % (N_SM, LOP3_PER_SM_CLK, SM_MAX_MHZ)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    st.free()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
