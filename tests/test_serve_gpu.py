"""Continuous-batching server: every request's bytes against the scalar
oracle, the same request alone and in the mix, admission under a small
memory budget, and rejection of a changed key for a resident stream."""
import os

import numpy as np
import pytest

import oracle
from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04750_gb300 import build as B
    B.build()
    N.lib()


def _trace(duration_s=0.04, seed=4):
    reqs, keyset = workloads.served_trace(seed=seed, rate_per_s=1e4, duration_s=duration_s,
                                          lo_log2_bytes=0, hi_log2_bytes=12)
    return reqs, keyset


def _server(n_streams, **kw):
    from paper_1909_04750_gb300.serve import Server
    args = dict(budget_bytes=1 << 30, quantum=256, split_quantum=1024, split_min_bits=8 * 2048,
                max_split_groups=3, keep_outputs=True)
    args.update(kw)
    return Server(n_streams, **args)


def _per_stream(reqs, finish):
    out = {}
    for j, r in enumerate(reqs):
        if not np.isnan(finish[j]):
            out.setdefault(r.stream_id, []).append(j)
    return out


def _check_against_oracle(srv, reqs, finish):
    for sid, js in _per_stream(reqs, finish).items():
        total = sum(8 * reqs[j].n_bytes for j in js)
        r0 = reqs[js[0]]
        ref = oracle.stream(r0.key, r0.iv, r0.iv_len, total)
        got = b"".join(srv.outputs[j].cpu().numpy().tobytes() for j in js)
        assert got == ref, sid


def test_served_trace_matches_oracle_and_states():
    reqs, keyset = _trace()
    srv = _server(keyset.n)
    finish = srv.run(reqs, realtime=False)
    assert srv.stats["completed"] == len(reqs) and srv.steps > 3
    _check_against_oracle(srv, reqs, finish)
    # resident states equal the oracle's state after each stream's bits
    per = _per_stream(reqs, finish)
    ids = sorted(per)[:6]
    states = srv.read_states(ids)
    for k, sid in enumerate(ids):
        js = per[sid]
        r0 = reqs[js[0]]
        st = oracle.init(r0.key, r0.iv, r0.iv_len)
        oracle.keystream_from(st, sum(8 * reqs[j].n_bytes for j in js))
        r, s = st.bits()
        assert np.array_equal(states[k], np.concatenate([np.packbits(r), np.packbits(s)]))


def test_request_same_alone_and_in_mix():
    reqs, keyset = _trace(seed=9)
    mix = _server(keyset.n)
    fin = mix.run(reqs, realtime=False)
    by = _per_stream(reqs, fin)
    sid = max(by, key=lambda k: len(by[k]))       # the stream with most requests
    alone_reqs = [reqs[j] for j in by[sid]]
    alone = _server(keyset.n)
    alone.run(alone_reqs, realtime=False)
    for a, m in enumerate(by[sid]):
        assert torch.equal(alone.outputs[a], mix.outputs[m])


def test_small_budget_still_correct():
    reqs, keyset = _trace(duration_s=0.02, seed=5)
    srv = _server(keyset.n, budget_bytes=6000 + 32 * keyset.n, max_inflight=1)
    finish = srv.run(reqs, realtime=False)
    assert srv.stats["completed"] == len(reqs)
    _check_against_oracle(srv, reqs, finish)


def test_streaming_outputs_and_stats():
    # response chunks go to per-step arenas under the budget
    reqs, keyset = _trace(duration_s=0.03, seed=8)
    srv = _server(keyset.n, keep_outputs=False, budget_bytes=(1 << 20) + 32 * keyset.n)
    finish = srv.run(reqs, realtime=False)
    st = srv.stats
    assert st["completed"] == len(reqs) and st["served_bits"] == sum(8 * r.n_bytes for r in reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # states still advanced exactly
    per = _per_stream(reqs, finish)
    sid = sorted(per)[0]
    r0 = reqs[per[sid][0]]
    ost = oracle.init(r0.key, r0.iv, r0.iv_len)
    oracle.keystream_from(ost, sum(8 * reqs[j].n_bytes for j in per[sid]))
    r, s = ost.bits()
    assert np.array_equal(srv.read_states([sid])[0], np.concatenate([np.packbits(r),
                                                                    np.packbits(s)]))


def test_changed_key_for_resident_stream_is_rejected():
    reqs, keyset = _trace(duration_s=0.01, seed=6)
    r0 = reqs[0]
    bad = workloads.Request(r0.arrival_s + 1e-3, r0.stream_id, bytes(10), r0.iv, r0.iv_len, 64)
    srv = _server(keyset.n)
    finish = srv.run(reqs + [bad], realtime=False)
    assert np.isnan(finish[-1]) and srv.stats["rejected"] == 1
    _check_against_oracle(srv, reqs, finish[:-1])


def test_wide_step_many_groups():
    # 12,000 requests admitted together: more than 256 groups per step, so
    # the per-group arrays are past numpy's small-block cache and the step
    # metadata crosses several pages
    reqs, keyset = workloads.served_trace(seed=11, rate_per_s=1e6, duration_s=0.012,
                                          p_continue=0.2, lo_log2_bytes=2, hi_log2_bytes=9)
    assert len(reqs) > 9000
    srv = _server(keyset.n, quantum=1024, split_quantum=2048, split_min_bits=2048,
                  max_split_groups=40)
    finish = srv.run(reqs, realtime=False)
    assert srv.stats["completed"] == len(reqs)
    _check_against_oracle(srv, reqs, finish)


def test_served_trace_real_lengths_sampled():
    # the served workload's own length mix (1 KiB .. 64 MiB, 70 % continuing
    # streams), its first 50 ms of arrivals, through the default server
    # configuration; every request of the streams the oracle can replay
    # quickly is compared in full, and the first 64 KiB of the longest
    # streams' first requests
    from paper_1909_04750_gb300.serve import Server
    reqs, keyset = workloads.served_trace(seed=4, duration_s=0.05)
    srv = Server(keyset.n, budget_bytes=16 << 30, keep_outputs=True)
    finish = srv.run(reqs, realtime=False)
    assert srv.stats["completed"] == len(reqs)
    per = _per_stream(reqs, finish)
    tot = {sid: sum(8 * reqs[j].n_bytes for j in js) for sid, js in per.items()}
    short = sorted(sid for sid in per if tot[sid] <= 8_000_000)
    assert len(short) >= 32
    first = [reqs[per[sid][0]] for sid in short]
    ref = oracle.batch_bytes(np.frombuffer(b"".join(r.key for r in first), np.uint8),
                             np.frombuffer(b"".join(r.iv for r in first), np.uint8), 80,
                             np.array([tot[sid] for sid in short], np.uint64),
                             threads=os.cpu_count() or 4)
    for k, sid in enumerate(short):
        got = b"".join(srv.outputs[j].cpu().numpy().tobytes() for j in per[sid])
        assert got == ref[k].tobytes(), sid
    longest = sorted(per, key=lambda sid: -tot[sid])[:6]
    for sid in longest:
        r = reqs[per[sid][0]]
        head = srv.outputs[per[sid][0]][:65536].cpu().numpy().tobytes()
        assert head == oracle.stream(r.key, r.iv, 80, 8 * len(head)), sid
