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
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "keystream Gbit/s on 1 GB300 (bit-exact), % of int-LOP roofline; served p50/p99"
WORKLOAD = ("plain_scale: 2^20 MICKEY 2.0 instances (32768 bitsliced groups), 80-bit keys "
            "and IVs from splitmix64 seed 2, 100 mixing preclocks, 2^14 keystream bits "
            "per instance, row-major bytes output (2 GiB)")
# The integer-logic roofline is measured in the same process: SM count from
# the device, LOP3 results per SM per SM-cycle from mickey_probe_lop3 (run
# before the timed region), at the maximum SM clock and at the median clock
# sampled during the timed region.

# DRAM traffic of one keystream launch of the plain workload at scale
# (dram__bytes_read.sum + dram__bytes_write.sum, one-pass ncu capture of the
# full-size launch in the autotuned configuration: 85.9 MB read + 2.190 GB
# written; algorithmic 2.20 GB = 2 GiB of output + the 26.2 MB state read
# and written).  It stands for the kernel sources it was measured on (their
# digest) and that launch with its row staging (the unroll depth does not
# change what is written; 4-tile staging moved 6.13 GB); otherwise traffic
# is null.
KEYSTREAM_TRAFFIC = {"digest": "9ad179c176d46a4f", "launch": ("persistent, ", " staged rows"),
                     "bytes_per_launch": 2275865856}


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
    p.add_argument("--no-extras", action="store_true",
                   help="skip the fused, batched and served workloads")
    p.add_argument("--served-duration", type=float, default=30.0)
    p.add_argument("--verify-rows", type=int, default=1024)
    return p.parse_args()


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


# ------------------------------------------------------------------ checks
# Sampled comparisons of timed outputs with the scalar oracle, run after the
# timed regions.  A mismatch is reported in the line and fails the run.

def _sample_rows(n: int, k: int, seed: int = 12345) -> np.ndarray:
    """k row indices of n: the first and the last 32-lane group, and random
    rows in between."""
    fixed = np.concatenate([np.arange(min(32, n)), np.arange(max(0, n - 32), n)])
    rng = np.random.default_rng(seed)
    extra = rng.choice(n, size=min(n, max(0, k - fixed.size)), replace=False)
    return np.unique(np.concatenate([fixed, extra]))


def verify_rows(s, out, n_bits: int, k: int) -> dict:
    """Rows of a row-major bytes output against the oracle."""
    import oracle
    import torch
    idx = _sample_rows(s.n, k)
    got = out[torch.from_numpy(idx).to(out.device)].cpu().numpy()
    ref = oracle.batch_bytes(s.keys[idx], s.ivs[idx], s.iv_lens[idx], n_bits,
                             threads=os.cpu_count() or 1)
    return {"rows": int(idx.size), "ok": bool(np.array_equal(got, ref)),
            "what": "row-major bytes of sampled instances (first and last group included) of "
                    "the last timed step == scalar oracle"}


def verify_fused(s, out, n_bits: int = 1 << 12, k: int = 1024) -> dict:
    import oracle
    import torch
    idx = _sample_rows(s.n, k)
    sel = torch.from_numpy(idx).to(out.device)
    got_u = out[0][sel].cpu().numpy().view(np.uint32)
    got_f = out[1][sel].cpu().numpy().view(np.float32)
    ref = oracle.batch_bytes(s.keys[idx], s.ivs[idx], s.iv_lens[idx], n_bits,
                             threads=os.cpu_count() or 1)
    ref_u = oracle.to_u32(ref, n_bits)
    ok = np.array_equal(got_u, ref_u) and np.array_equal(got_f, oracle.to_f32(ref_u))
    return {"rows": int(idx.size), "ok": bool(ok),
            "what": "u32 words and FP32 uniforms of sampled instances (first and last group "
                    "included) of the last timed step == scalar oracle"}


def verify_batched(s, b, out) -> dict:
    """Sampled streams of the last replay: the 4 longest, the 4 shortest, 8 of
    every IV length, 48 more at random."""
    import oracle
    n = s.n
    order = np.argsort(s.n_bits, kind="stable")
    rng = np.random.default_rng(7)
    pick = [order[-4:], order[:4], rng.choice(n, 48, replace=False)]
    for L in np.unique(s.iv_lens):
        cand = np.flatnonzero(s.iv_lens == L)
        pick.append(rng.choice(cand, min(8, cand.size), replace=False))
    idx = np.unique(np.concatenate(pick))
    ref = oracle.batch_bytes(s.keys[idx], s.ivs[idx], s.iv_lens[idx], s.n_bits[idx],
                             threads=os.cpu_count() or 1)
    host = out.cpu().numpy()
    ok = True
    for j, i in enumerate(idx):
        o, nb = int(b.offsets[i]), (int(s.n_bits[i]) + 7) // 8
        ok &= np.array_equal(host[o:o + nb], np.asarray(ref[j]).reshape(-1))
    return {"streams": int(idx.size), "ok": bool(ok),
            "bits": int(s.n_bits[idx].sum()),
            "what": "whole keystreams of sampled streams (longest, shortest, every IV length) "
                    "of the last replay == scalar oracle"}


def verify_served(srv, reqs, keyset, k: int = 96, max_bits: int = 1 << 21) -> dict:
    """Resident states after the run of sampled streams (those whose
    requests total at most max_bits, several with more than one request)
    against the oracle's state after the same number of keystream bits."""
    import oracle
    total, count = {}, {}
    for r in reqs:
        total[r.stream_id] = total.get(r.stream_id, 0) + 8 * r.n_bytes
        count[r.stream_id] = count.get(r.stream_id, 0) + 1
    small = [sid for sid, b in total.items() if b <= max_bits]
    multi = [sid for sid in small if count[sid] > 1]
    rng = np.random.default_rng(11)
    ids = sorted(set(multi[: k // 2]) | set(rng.choice(small, min(len(small), k // 2),
                                                       replace=False).tolist()))
    got = srv.read_states(np.array(ids, np.uint32))
    ok = True
    for j, sid in enumerate(ids):
        st = oracle.init(keyset.keys[sid].tobytes(), keyset.ivs[sid].tobytes(),
                         int(keyset.iv_lens[sid]))
        oracle.keystream_from(st, total[sid])
        r, s_ = st.bits()
        rec = np.unpackbits(got[j])
        ok &= np.array_equal(rec[:100], r) and np.array_equal(rec[104:204], s_)
    return {"streams": len(ids), "with_several_requests": int(sum(count[i] > 1 for i in ids)),
            "ok": bool(ok),
            "what": "resident state after every request of sampled streams == scalar oracle "
                    "state after the same keystream bits"}


def verify_grain(s, out, n_bits: int = 1 << 14, k: int = 1024) -> dict:
    """Sampled rows of the last Grain bytes step against the Grain oracle."""
    from oracle import grain as og
    import torch
    idx = _sample_rows(s.n, k)
    got = out[torch.from_numpy(idx).to(out.device)].cpu().numpy()
    ref = og.batch_bytes(s.keys[idx], s.ivs[idx], n_bits, threads=os.cpu_count() or 1)
    return {"rows": int(idx.size), "ok": bool(np.array_equal(got, ref)),
            "what": "row-major bytes of sampled Grain instances (first and last group "
                    "included) of the last timed step == scalar Grain oracle"}


def verify_ragged(s, rows, offs, lengths, before, k: int = 256) -> dict:
    """Sampled streams of one ragged call against the oracle: stream i's
    bits before[i] .. before[i] + lengths[i] - 1 at byte offsets[i]."""
    import oracle
    host = rows.cpu().numpy()
    idx = _sample_rows(s.n, k)
    sub = s.subset(idx)
    total = before[idx] + lengths[idx]
    ref = oracle.batch_bytes(sub.keys, sub.ivs, sub.iv_lens, total, threads=os.cpu_count() or 1)
    ok = True
    for j, i in enumerate(idx):
        want = np.packbits(np.unpackbits(np.asarray(ref[j], np.uint8))[int(before[i]):int(total[j])])
        ok &= bool(np.array_equal(host[int(offs[i]):int(offs[i]) + want.size], want))
    return {"rows": int(idx.size), "ok": ok,
            "what": "packed rows of sampled streams (first and last group included) of one "
                    "more ragged call == scalar oracle, at each stream's own position"}


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
    from paper_1909_04750_gb300 import autotune, shard
    from paper_1909_04750_gb300 import peak as P
    from paper_1909_04750_gb300.build import build, sources_digest
    from paper_1909_04750_gb300.clocks import ClockSampler
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
    # the roofline's factors, measured on this device before the timed region
    pk = P.measure()

    def step(layout="bytes", o=out):
        st.reset(keys, ivs, lens)
        st.generate(n_bits, layout, out=o)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local).start()
    shard.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                           # evict L2 between steps
        ev[k][0].record(stream)
        st.reset(keys, ivs, lens)                       # init kernel (load + preclock)
        ev[k][1].record(stream)
        st.generate(n_bits, "bytes", out=out)           # keystream + transpose kernel
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    shard.barrier()
    clocks = sampler.stop()
    st.sync()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    ks_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    init_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    total_ms = shard.max_over_ranks(sum(step_ms))
    bits_per_step = n * n_bits * world
    value = bits_per_step * args.steps / (total_ms * 1e-3) / 1e9
    # the last timed step's output against the oracle (every rank its own shard)
    verified = verify_rows(s, out, n_bits, args.verify_rows)

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
    sm_max = clocks.get("sm_max_mhz") or P.max_sm_mhz(local) or pk["probe_sm_mhz"]
    peak = P.peak_tops(pk, sm_max)
    peak_med = P.peak_tops(pk, clocks["sm_mhz"]) if clocks.get("sm_mhz") else None
    init_ops = groups * 260 * ops_per_clock(True)
    whole_ops = ops + init_ops
    alg_bytes = n * n_bits // 8 + 2 * groups * 200 * 4        # output + state in and out
    traffic = None
    if (sources_digest() == KEYSTREAM_TRAFFIC["digest"]
            and autotune.describe(tuned).startswith(KEYSTREAM_TRAFFIC["launch"][0])
            and autotune.describe(tuned).endswith(KEYSTREAM_TRAFFIC["launch"][1])
            and (n, n_bits) == (1 << 20, 1 << 14)):
        traffic = KEYSTREAM_TRAFFIC["bytes_per_launch"]

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host_out = torch.empty((n, n_bits // 8), dtype=torch.uint8, pin_memory=True)
        # the step's inputs live in pinned host memory (copied in every step)
        pk_ = torch.from_numpy(s.keys).pin_memory()
        pv = torch.from_numpy(s.ivs).pin_memory()
        pl = torch.from_numpy(s.iv_lens.astype(np.uint32).view(np.int32)).pin_memory()
        hk, hv, hl = pk_.numpy(), pv.numpy(), pl.numpy().view(np.uint32)

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
    st.free()
    del out, flush
    torch.cuda.empty_cache()

    # the other workloads (one GPU only: they would hold every GPU of a
    # multi-GPU run for minutes)
    extras = {}
    if world == 1 and not args.no_extras:
        from paper_1909_04750_gb300 import (bench_batched, bench_fused, bench_grain,
                                            bench_ragged, bench_served)
        extras["fused"] = bench_fused.measure(peak=pk, verify=verify_fused)
        extras["grain"] = bench_grain.measure(peak=pk, verify=verify_grain)
        extras["ragged"] = bench_ragged.measure(verify=verify_ragged)
        extras["batched"] = bench_batched.measure(plain_gbit_s=value, verify=verify_batched)
        extras["served"] = bench_served.measure(duration=args.served_duration,
                                                plain_gbit_s=value, verify=verify_served)

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
                         "unit": "Tops/s", "frac": achieved / peak,
                         "peak_at_median_clock": peak_med,
                         "frac_at_median_clock": achieved / peak_med if peak_med else None,
                         "traffic": traffic,
                         "traffic_unit": "bytes per launch", "algorithmic_bytes": alg_bytes,
                         "kernel": "keystream kernel, bytes layout (%s)" % autotune.describe(tuned),
                         "ops_per_clock_per_group": ops_per_clock(False),
                         "init_frac": init_ops / (statistics.mean(init_ms) * 1e-3) / 1e12 / peak,
                         "peak_basis": "%d SMs (device) x %.2f LOP3/SM/clk (mickey_probe_lop3, "
                                       "this process) x %g MHz (max SM clock)"
                                       % (pk["n_sm"], pk["lop3_per_sm_clk"], sm_max)},
            "verified": verified,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 2 * args.steps,          # init kernel + keystream kernel per step
            "clocks": clocks,
            **extras,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    bad = [k for k, v in [("plain", verified)] + [(k, e.get("verified")) for k, e in
                                                    extras.items()] if v and not v["ok"]]
    if bad:
        print("bench: output differs from the oracle in: %s" % ", ".join(bad), file=sys.stderr)
        sys.exit(1)


if __name__ == "__main__":
    main()
