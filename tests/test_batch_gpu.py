"""Batched ragged generation (one persistent launch, CUDA graph) against the
scalar oracle.  Every stream is compared bit for bit; the full-size 100,000
stream workload is compared on sampled streams."""
import os

import numpy as np
import pytest

import oracle
from paper_1909_04750_gb300 import _native as N
from paper_1909_04750_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_04750_gb300 import build as B
    B.build()
    N.lib()


def _oracle_rows(s, n_bits):
    return oracle.batch_bytes(s.keys, s.ivs, s.iv_lens, n_bits, threads=THREADS)


def _check(batch, out, s, idx=None):
    rows = batch.rows(out)
    idx = range(s.n) if idx is None else idx
    sub = s.subset(np.array(list(idx)))
    ref = _oracle_rows(sub, batch.n_bits[np.array(list(idx))])
    ref = list(ref) if isinstance(ref, list) else [r for r in ref]
    for k, i in enumerate(idx):
        assert rows[i].tobytes() == ref[k].tobytes(), i


def test_small_ragged_batch_every_stream():
    from paper_1909_04750_gb300.batch import Batch
    s = workloads.batched(3000)
    rng = np.random.default_rng(1)
    nb = rng.integers(0, 9000, s.n).astype(np.uint64)
    nb[:5] = [0, 1, 7, 33, 8191]            # empty, partial bytes, partial tiles
    s.n_bits = nb
    b = Batch(nb, s.iv_lens)
    out = b.run(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    b.sync()
    _check(b, out, s)


def test_batch_graph_replay_and_host_inputs():
    from paper_1909_04750_gb300.batch import Batch
    s = workloads.batched(700)
    nb = (s.n_bits % 5000).astype(np.uint64)
    s.n_bits = nb
    b = Batch(nb, s.iv_lens)
    o1 = b.run(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    b.sync()
    o2 = torch.zeros_like(o1)
    b.run(s.keys, s.ivs, o2)                 # host inputs, graph replayed
    b.sync()
    rows1, rows2 = b.rows(o1), b.rows(o2)
    assert all(x.tobytes() == y.tobytes() for x, y in zip(rows1, rows2))
    for u in (2, 4):
        for bps in (1, 2):
            b.set_config(u, bps, 0)
            o3 = b.run(s.keys, s.ivs)
            b.sync()
            assert all(x.tobytes() == y.tobytes() for x, y in zip(rows1, b.rows(o3)))
    _check(b, o1, s, idx=range(0, 700, 7))


@pytest.mark.parametrize("split_mode", [N.BATCH_SPLIT_SHARED, N.BATCH_SPLIT_OWN])
@pytest.mark.parametrize("split_clocks", [1, 3000, 7000])
def test_split_path_every_stream(split_clocks, split_mode):
    # groups needing more clocks than split_clocks run one per warp, in the
    # persistent kernel's warps or in a kernel of their own
    from paper_1909_04750_gb300.batch import Batch
    s = workloads.batched(2000)
    rng = np.random.default_rng(7)
    nb = rng.integers(0, 12000, s.n).astype(np.uint64)
    nb[:6] = [11999, 11998, 1, 0, 31, 8193]
    s.n_bits = nb
    b = Batch(nb, s.iv_lens)
    b.set_config(4, 2, split_clocks, split_mode)
    cfg = b.get_config()
    assert cfg["split_groups"] > 0 and cfg["split_mode"] == split_mode
    out = b.run(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    b.sync()
    _check(b, out, s)


def test_batch_rejects_bad_iv_length():
    from paper_1909_04750_gb300.batch import Batch
    with pytest.raises(N.MickeyError) as ei:
        Batch(np.full(10, 64, np.uint64), np.array([80] * 9 + [81], np.uint32))
    assert ei.value.code == N.E_IVLEN


@pytest.mark.parametrize("split_mode", [N.BATCH_SPLIT_SHARED, N.BATCH_SPLIT_OWN])
def test_batched_workload_full_size_sampled(split_mode):
    from paper_1909_04750_gb300.batch import Batch
    s = workloads.batched()
    b = Batch(s.n_bits, s.iv_lens)
    b.set_config(4, 1, b.max_clocks // 64, split_mode)
    assert b.n == 100_000 and b.max_clocks == int(s.n_bits.max())
    out = b.run(torch.from_numpy(s.keys).cuda(), torch.from_numpy(s.ivs).cuda())
    b.sync()
    order = np.argsort(-s.n_bits.astype(np.int64), kind="stable")
    rng = np.random.default_rng(3)
    pick = sorted(set(order[:8].tolist()) | set(order[-8:].tolist()) |
                  set(rng.integers(0, s.n, 4096).tolist()))
    _check(b, out, s, idx=pick)
    # every IV length bucket is represented
    assert set(s.iv_lens[pick]) == {0, 16, 32, 48, 64, 80}
