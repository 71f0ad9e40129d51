"""Continuous-batching keystream server over resident MICKEY 2.0 streams.

Requests (stream id, key, IV, length) arrive over time.  The scheduler loop:

* appends each arrived request to its stream's chain: a stream's requests
  continue one keystream in arrival order, so the chain is one run of bits
  and a step may end one request and go on into the next (with per-request
  output buffers a step stops at request boundaries instead); steps run in
  order on one CUDA stream, so the state table is always up to date;
* loads and preclocks streams that appear for the first time; afterwards
  their state stays in the device table, so follow-up requests continue the
  keystream where the previous one stopped, without re-keying;
* issues steps over all admitted requests with bits left: sorted by bits
  left and packed 32 per group, every lane of a group produces min(quantum,
  smallest bits left in the group) bits, so no request runs past its end.
  A stream's bits come out one clock after another, so a request's latency
  is bound by its length times the time per clock: groups are clocked one
  warp per group (the split path, several times less time per clock than
  one thread per group) up to `max_split_groups` (by default 4 warps per SM
  sub-partition); only the groups with the least work left beyond that run
  one per thread;
* writes each step's bytes into a step arena (the response chunk of every
  request served by the step), counted against the device-memory budget
  until the step has completed; with `keep_outputs` each request instead
  gets a whole buffer reserved at admission (used by the tests);
* keeps at most `max_inflight` steps queued and timestamps a request's
  completion with the device time of the step that finished it.

Requests that arrive while others run join the next step, so their work
overlaps on the device with the requests already in flight.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque

import numpy as np
import torch

from . import _native as N

NO_STREAM = 0xFFFFFFFF


class Server:
    def __init__(self, max_streams: int, budget_bytes: int = 16 << 30, quantum: int = 1 << 15,
                 split_quantum: int = 1 << 17, split_min_bits: int = 0,
                 max_split_groups: int | None = None, max_groups: int = 1 << 16,
                 max_inflight: int = 2, keep_outputs: bool = False, stream=None):
        if quantum % 32 or split_quantum % 32:
            raise ValueError("quanta must be multiples of 32 bits")
        self._L = N.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.max_streams, self.max_groups = max_streams, max_groups
        self.budget = budget_bytes - 32 * max_streams          # the state table is resident
        self.quantum, self.split_quantum = quantum, split_quantum
        self.split_min_bits = split_min_bits
        sms = torch.cuda.get_device_properties(self.stream.device).multi_processor_count
        self.max_split_groups = max_split_groups if max_split_groups is not None else 16 * sms
        self.max_inflight, self.keep_outputs = max_inflight, keep_outputs
        self._h = N.check_ptr(self._L.mickey_server_create(
            max_streams, max_groups, ctypes.c_void_p(self.stream.cuda_stream)))
        self.identity = {}                      # stream id -> (key, iv, iv_len)
        self.steps = 0
        self.stats = {}
        self.outputs = {}                       # job index -> tensor (keep_outputs)

    # ------------------------------------------------------------------ steps
    def _init_streams(self, reqs, js):
        ids = np.array([reqs[j].stream_id for j in js], np.uint32)
        keys = np.frombuffer(b"".join(reqs[j].key for j in js), np.uint8)
        ivs = np.frombuffer(b"".join(reqs[j].iv for j in js), np.uint8)
        lens = np.array([reqs[j].iv_len for j in js], np.uint32)
        N.check(self._L.mickey_server_init_streams(self._h, ids.ctypes.data, keys.ctypes.data,
                                                   ivs.ctypes.data, lens.ctypes.data, len(js)))

    def _plan(self, rem):
        """Plan a step over the active streams with `rem` bits left each:
        (order of the served streams, longest first; bits per 32-lane group;
        number of split groups, which lead the order)."""
        order = np.argsort(-rem, kind="stable")
        n = order.size
        ns = min((int(np.count_nonzero(rem >= self.split_min_bits)) + 31) // 32,
                 self.max_split_groups)
        G = min((n + 31) // 32, self.max_groups)
        order = order[: 32 * G]
        srt = rem[order]
        last = np.minimum(np.arange(G) * 32 + 31, order.size - 1)
        quant = np.where(np.arange(G) < ns, self.split_quantum, self.quantum)
        k_g = np.minimum(quant, srt[last]).astype(np.int64)
        return order, k_g, min(ns, G)

    def _issue(self, act, rem, keep_ptr, reserve):
        """One step over the active streams `act` with `rem` bits left each
        (keep_ptr: per-stream output address in keep_outputs mode).  Returns
        (start event, end event, step arena or None, order, bits per lane)."""
        order, k_g, ns = self._plan(rem)
        G = k_g.size
        k_lane = np.repeat(k_g, 32)[: order.size]
        nbytes = int(k_lane.sum()) // 8
        slots = np.full(32 * G, NO_STREAM, np.uint32)
        slots[: order.size] = act[order]
        outs = np.zeros(32 * G, np.uint64)
        arena = None
        if self.keep_outputs:
            outs[: order.size] = keep_ptr[order]
        else:
            reserve(nbytes)
            arena = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.stream.device)
            offs = np.concatenate(([0], np.cumsum(k_lane[:-1] // 8)))
            outs[: order.size] = np.uint64(arena.data_ptr()) + offs.astype(np.uint64)
        clocks = np.ascontiguousarray(k_g, np.uint32)   # named: must outlive the call
        ev0 = torch.cuda.Event(enable_timing=True)
        ev0.record(self.stream)
        N.check(self._L.mickey_server_step(self._h, G, ns, slots.ctypes.data, outs.ctypes.data,
                                           clocks.ctypes.data))
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        self.steps += 1
        return ev0, ev, arena, order, k_lane

    # ------------------------------------------------------------------ main loop
    def run(self, requests, realtime: bool = True):
        """Serve `requests` (workloads.Request list in arrival order).
        Returns per-request completion times (ms of device time since the
        start, NaN if rejected); self.stats holds the summary, latency being
        measured from the moment the server saw the request (its arrival
        time when `realtime`, the start otherwise) to the end of the step
        that produced its last byte."""
        n = len(requests)
        bits = np.array([8 * r.n_bytes for r in requests], np.int64)
        arrival = np.array([r.arrival_s for r in requests], np.float64)
        finish = np.full(n, np.nan)
        release = np.zeros(n)             # ms since the start the server saw the request
        rejected = np.zeros(n, bool)
        S = self.max_streams
        # per stream (indexed by stream id), bits counted from the chain's start
        done = np.zeros(S, np.int64)      # produced
        end = np.zeros(S, np.int64)       # admitted (end of the last request in the chain)
        cur_end = np.zeros(S, np.int64)   # end of the first unfinished request
        cur_start = np.zeros(S, np.int64)
        cur_buf = np.zeros(S, np.uint64)  # its output buffer (keep_outputs)
        chains: dict = {}                 # stream -> deque of [job, start, end, buf]
        waiting: deque = deque()          # arrived, not yet admitted (keep_outputs budget)
        inflight: deque = deque()
        used = 0
        served = 0
        busy_ms = 0.0                     # device time spent in steps
        t0 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(self.stream)
        t_start = time.perf_counter()
        nxt = 0

        def retire(block: bool):
            nonlocal used, busy_ms
            while inflight and (block or inflight[0][1].query()):
                ev0, ev, fin, nb = inflight.popleft()
                ev.synchronize()
                finish[fin] = t0.elapsed_time(ev)
                busy_ms += ev0.elapsed_time(ev)
                used -= nb
                block = False

        def reserve(nb):
            nonlocal used
            while inflight and used + nb > self.budget:
                retire(block=True)
            used += nb

        def admit(j) -> bool:
            """Append job j to its stream's chain; False if the budget blocks it."""
            nonlocal used
            r = requests[j]
            sid = r.stream_id
            ident = self.identity.get(sid)
            if ident is not None and ident != (r.key, r.iv, r.iv_len):
                rejected[j] = True                 # key/IV differ from the resident stream's
                return True
            nb = int(bits[j]) // 8
            if self.keep_outputs and used > 0 and used + nb > self.budget:
                return False                       # wait for buffers to be released
            if ident is None:
                self.identity[sid] = (r.key, r.iv, r.iv_len)
                new_js.append(j)
            if bits[j] == 0:
                finish[j] = 1e3 * (time.perf_counter() - t_start)
                return True
            buf = 0
            if self.keep_outputs:
                t = torch.empty(nb, dtype=torch.uint8, device=self.stream.device)
                self.outputs[j] = t
                buf = t.data_ptr()
                used += nb
            q = chains.setdefault(sid, deque())
            a, b = int(end[sid]), int(end[sid] + bits[j])
            if not q:                              # the stream was idle
                cur_start[sid], cur_end[sid], cur_buf[sid] = a, b, buf
            q.append([j, a, b, buf])
            end[sid] = b
            return True

        while nxt < n or waiting or inflight or (end > done).any():
            now = time.perf_counter() - t_start
            while nxt < n and (not realtime or arrival[nxt] <= now):
                release[nxt] = 1e3 * now
                waiting.append(nxt)
                nxt += 1
            retire(block=len(inflight) >= self.max_inflight)
            new_js = []
            while waiting and admit(waiting[0]):
                waiting.popleft()
            if new_js:
                self._init_streams(requests, new_js)
            act = np.flatnonzero(end > done).astype(np.uint32)
            if act.size:
                lim = cur_end if self.keep_outputs else end
                rem = lim[act] - done[act]
                ptr = cur_buf[act] + ((done[act] - cur_start[act]) // 8).astype(np.uint64)
                ev0, ev, arena, order, k_lane = self._issue(act, rem, ptr, reserve)
                served += int(k_lane.sum())
                lanes = act[order]
                done[lanes] += k_lane
                fin = []
                for sid in lanes[done[lanes] >= cur_end[lanes]]:
                    q = chains[int(sid)]
                    while q and q[0][2] <= done[sid]:
                        fin.append(q.popleft()[0])
                    if q:
                        cur_start[sid], cur_end[sid], cur_buf[sid] = q[0][1], q[0][2], q[0][3]
                    else:                          # chain empty: restart its counts
                        done[sid] = end[sid] = cur_end[sid] = cur_start[sid] = 0
                fin = np.array(fin, np.int64)
                inflight.append((ev0, ev, fin, int(bits[fin].sum()) // 8 if arena is None
                                 else arena.numel()))
                del arena          # the caching allocator reuses it after the step
            elif inflight:
                retire(block=True)
            elif nxt < n:
                time.sleep(max(0.0, min(0.005, arrival[nxt] - now)))
        torch.cuda.synchronize()
        retire(block=True)
        ok = ~rejected & ~np.isnan(finish)
        lat = finish[ok] - release[ok]       # from hand-over to the last byte
        end_ms = float(np.nanmax(finish)) if ok.any() else 0.0
        self.stats = {
            "requests": n, "completed": int(ok.sum()), "rejected": int(rejected.sum()),
            "steps": self.steps, "served_bits": served, "wall_ms": end_ms,
            "gbit_s": served / (end_ms * 1e-3) / 1e9 if end_ms > 0 else 0.0,
            "busy_ms": busy_ms,
            "busy_gbit_s": served / (busy_ms * 1e-3) / 1e9 if busy_ms > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_ms": float(lat.mean()) if lat.size else None,
        }
        return finish

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
