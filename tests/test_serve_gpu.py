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


def _per_stream(jobs):
    out = {}
    for j in jobs:
        if not j.rejected:
            out.setdefault(j.stream_id, []).append(j)
    return out


def _check_against_oracle(jobs):
    for sid, js in _per_stream(jobs).items():
        total = sum(j.n_bits for j in js)
        j0 = js[0]
        ref = oracle.stream(j0.key, j0.iv, j0.iv_len, total)
        got = b"".join(j.buf[: j.n_bits // 8].cpu().numpy().tobytes() for j in js)
        assert got == ref, sid


def test_served_trace_matches_oracle_and_states():
    reqs, keyset = _trace()
    srv = _server(keyset.n)
    jobs = srv.run(reqs, realtime=False)
    assert srv.stats["completed"] == len(reqs) and srv.steps > 3
    _check_against_oracle(jobs)
    # resident states equal the oracle's state after each stream's bits
    ids = sorted(_per_stream(jobs))[:6]
    states = srv.read_states(ids)
    for k, sid in enumerate(ids):
        js = _per_stream(jobs)[sid]
        st = oracle.init(js[0].key, js[0].iv, js[0].iv_len)
        oracle.keystream_from(st, sum(j.n_bits for j in js))
        r, s = st.bits()
        assert np.array_equal(states[k], np.concatenate([np.packbits(r), np.packbits(s)]))


def test_request_same_alone_and_in_mix():
    reqs, keyset = _trace(seed=9)
    mix = _server(keyset.n).run(reqs, realtime=False)
    by = _per_stream(mix)
    sid = max(by, key=lambda k: len(by[k]))       # the stream with most requests
    alone_reqs = [r for r in reqs if r.stream_id == sid]
    alone = _server(keyset.n).run(alone_reqs, realtime=False)
    for a, m in zip(alone, by[sid]):
        assert a.n_bits == m.n_bits
        assert torch.equal(a.buf[: a.n_bits // 8], m.buf[: m.n_bits // 8])


def test_small_budget_still_correct():
    reqs, keyset = _trace(duration_s=0.02, seed=5)
    srv = _server(keyset.n, budget_bytes=6000, max_inflight=1)
    jobs = srv.run(reqs, realtime=False)
    assert srv.stats["completed"] == len(reqs)
    _check_against_oracle(jobs)


def test_changed_key_for_resident_stream_is_rejected():
    reqs, keyset = _trace(duration_s=0.01, seed=6)
    r0 = reqs[0]
    bad = workloads.Request(r0.arrival_s + 1e-3, r0.stream_id, bytes(10), r0.iv, r0.iv_len, 64)
    srv = _server(keyset.n)
    jobs = srv.run(reqs + [bad], realtime=False)
    assert jobs[-1].rejected and srv.stats["rejected"] == 1
    _check_against_oracle(jobs)
