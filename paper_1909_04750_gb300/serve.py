"""Continuous-batching keystream server over resident MICKEY 2.0 streams.

Requests (stream id, key, IV, length) arrive over time.  The scheduler loop:

* admits waiting requests in arrival order while the output-memory budget
  allows (a request's output buffer is reserved at admission and returned
  when its last step has completed); requests of one stream are served one
  after another, in arrival order;
* loads and preclocks the streams that appear for the first time (their
  state then stays in the device table, so follow-up requests continue the
  keystream where the previous one stopped);
* issues steps: all admitted requests with bits left are sorted by bits left
  and packed 32 per group; every lane of a group produces min(quantum,
  smallest bits left in the group) bits, so no request runs past its end; the
  groups with the most work left are clocked one warp per group (split path,
  with a larger quantum, since a stream's bits come out one clock after
  another and those requests bound the latency);
* keeps at most `max_inflight` steps queued on the GPU and timestamps each
  request's completion with the device time of the step that finished it;
  a stream's next request may start in the step after its previous request's
  last step, since steps run in order on one CUDA stream.

Requests that arrive while others run join the next step: their work
overlaps on the device with the requests already in flight.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N

NO_STREAM = 0xFFFFFFFF


@dataclass
class Job:
    idx: int
    stream_id: int
    key: bytes
    iv: bytes
    iv_len: int
    n_bits: int
    arrival_s: float
    done: int = 0
    buf: torch.Tensor | None = None
    finish_ms: float | None = None
    rejected: bool = False


class Server:
    def __init__(self, max_streams: int, budget_bytes: int = 16 << 30, quantum: int = 1 << 15,
                 split_quantum: int = 1 << 18, split_min_bits: int = 1 << 22,
                 max_split_groups: int | None = None, max_groups: int = 1 << 14,
                 max_inflight: int = 2, keep_outputs: bool = False, stream=None):
        if quantum % 32 or split_quantum % 32:
            raise ValueError("quanta must be multiples of 32 bits")
        self._L = N.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.max_streams = max_streams
        self.max_groups = max_groups
        self.budget = budget_bytes
        self.quantum, self.split_quantum = quantum, split_quantum
        self.split_min_bits = split_min_bits
        props = torch.cuda.get_device_properties(self.stream.device)
        self.max_split_groups = (max_split_groups if max_split_groups is not None
                                 else props.multi_processor_count)
        self.max_inflight = max_inflight
        self.keep_outputs = keep_outputs
        self._h = N.check_ptr(self._L.mickey_server_create(
            max_streams, max_groups, ctypes.c_void_p(self.stream.cuda_stream)))
        self.identity = {}                      # stream id -> (key, iv, iv_len)
        self.position = np.zeros(max_streams, np.uint64)
        self.steps = 0
        self.stats = {}

    # ------------------------------------------------------------------ helpers
    def _init_streams(self, jobs):
        if not jobs:
            return
        ids = np.array([j.stream_id for j in jobs], np.uint32)
        keys = np.frombuffer(b"".join(j.key for j in jobs), np.uint8)
        ivs = np.frombuffer(b"".join(j.iv for j in jobs), np.uint8)
        lens = np.array([j.iv_len for j in jobs], np.uint32)
        N.check(self._L.mickey_server_init_streams(self._h, ids.ctypes.data, keys.ctypes.data,
                                                   ivs.ctypes.data, lens.ctypes.data, len(jobs)))

    def _step(self, active):
        rem = np.array([j.n_bits - j.done for j in active], np.int64)
        order = np.argsort(-rem, kind="stable")
        n = len(active)
        n_long = int(np.count_nonzero(rem >= self.split_min_bits))
        ns = min((n_long + 31) // 32, self.max_split_groups)
        G = ns + (n - min(n, 32 * ns) + 31) // 32
        if G > self.max_groups:
            # serve the longest ones this step, the rest next step
            G = self.max_groups
        slots = np.full(32 * G, NO_STREAM, np.uint32)
        outs = np.zeros(32 * G, np.uint64)
        clocks = np.zeros(G, np.uint32)
        finishing = []
        pos = 0
        for g in range(G):
            take = order[pos:pos + 32]
            pos += len(take)
            if len(take) == 0:
                break
            q = self.split_quantum if g < ns else self.quantum
            k = int(min(q, rem[take].min()))
            clocks[g] = k
            for lane, t in enumerate(take):
                j = active[t]
                slots[32 * g + lane] = j.stream_id
                outs[32 * g + lane] = j.buf.data_ptr() + j.done // 8
                j.done += k
                if j.done == j.n_bits:
                    finishing.append(j)
        N.check(self._L.mickey_server_step(self._h, G, ns, slots.ctypes.data, outs.ctypes.data,
                                           clocks.ctypes.data))
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        self.steps += 1
        lanes = (slots != NO_STREAM).reshape(G, 32).sum(axis=1)
        return ev, finishing, int((clocks.astype(np.int64) * lanes).sum())

    # ------------------------------------------------------------------ main loop
    def run(self, requests, realtime: bool = True):
        """Serve `requests` (workloads.Request list, arrival order).  Returns
        the Job list; self.stats holds latency and throughput figures."""
        jobs = [Job(i, r.stream_id, r.key, r.iv, r.iv_len, 8 * r.n_bytes, r.arrival_s)
                for i, r in enumerate(requests)]
        nxt = 0
        waiting: deque = deque()
        active: list = []
        inflight: deque = deque()
        busy: set = set()
        used = 0
        served_bits = 0
        t0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(self.stream)
        t_start = time.perf_counter()

        def retire(block: bool):
            nonlocal used
            while inflight and (block or inflight[0][0].query()):
                ev, fin, _ = inflight.popleft()
                ev.synchronize()
                ms = t0.elapsed_time(ev)
                for j in fin:
                    j.finish_ms = ms
                    used -= j.buf.numel()
                    if not self.keep_outputs:
                        j.buf = None
                block = False

        while nxt < len(jobs) or waiting or active or inflight:
            now = time.perf_counter() - t_start
            while nxt < len(jobs) and (not realtime or jobs[nxt].arrival_s <= now):
                waiting.append(jobs[nxt])
                nxt += 1
            retire(block=len(inflight) >= self.max_inflight)
            # admission, arrival order; a stream's requests one at a time
            new_streams, blocked, keep = [], set(), deque()
            stop = False
            while waiting:
                j = waiting.popleft()
                if stop or j.stream_id in busy or j.stream_id in blocked:
                    blocked.add(j.stream_id)
                    keep.append(j)
                    continue
                ident = self.identity.get(j.stream_id)
                if ident is not None and ident != (j.key, j.iv, j.iv_len):
                    j.rejected = True          # key/IV differ from the resident stream's
                    continue
                nbytes = (j.n_bits + 7) // 8
                if used + nbytes > self.budget and used > 0:
                    stop = True
                    keep.append(j)
                    blocked.add(j.stream_id)
                    continue
                used += nbytes
                j.buf = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.stream.device)
                busy.add(j.stream_id)
                if ident is None:
                    self.identity[j.stream_id] = (j.key, j.iv, j.iv_len)
                    new_streams.append(j)
                if j.n_bits == 0:
                    j.finish_ms = 1e3 * (time.perf_counter() - t_start)
                    busy.discard(j.stream_id)
                    used -= nbytes
                    continue
                active.append(j)
            waiting = keep
            self._init_streams(new_streams)
            if active:
                ev, fin, bits = self._step(active)
                served_bits += bits
                inflight.append((ev, fin, bits))
                done_ids = {id(j) for j in fin}
                active = [j for j in active if id(j) not in done_ids]
                for j in fin:
                    # its last step is queued: the stream's next request may
                    # follow (steps run in order on one CUDA stream)
                    busy.discard(j.stream_id)
                    self.position[j.stream_id] += np.uint64(j.n_bits)
            elif inflight:
                retire(block=True)
            elif nxt < len(jobs):
                time.sleep(max(0.0, min(0.01, jobs[nxt].arrival_s - now)))
        torch.cuda.synchronize()
        lat = np.array([j.finish_ms - 1e3 * j.arrival_s for j in jobs
                        if j.finish_ms is not None and not j.rejected])
        end_ms = max((j.finish_ms for j in jobs if j.finish_ms is not None), default=0.0)
        self.stats = {
            "requests": len(jobs), "completed": int(lat.size),
            "rejected": sum(j.rejected for j in jobs), "steps": self.steps,
            "served_bits": served_bits, "wall_ms": end_ms,
            "gbit_s": served_bits / (end_ms * 1e-3) / 1e9 if end_ms > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_ms": float(lat.mean()) if lat.size else None,
        }
        return jobs

    def read_states(self, stream_ids):
        ids = np.ascontiguousarray(stream_ids, np.uint32)
        out = np.zeros((ids.size, 26), np.uint8)
        N.check(self._L.mickey_server_read_states(self._h, ids.ctypes.data, ids.size,
                                                  out.ctypes.data))
        return out

    def set_config(self, unroll: int, blocks_per_sm: int):
        N.check(self._L.mickey_server_set_config(self._h, unroll, blocks_per_sm))

    def free(self):
        if getattr(self, "_h", None):
            self._L.mickey_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
