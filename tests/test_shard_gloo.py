"""Weak-scaling shards over two gloo ranks on the CPU: each rank draws its
own instances, the shards tile the single-process instance sequence, the
keystream of an instance is the same computed in its shard as alone (the
oracle, which is what a rank's GPU output is checked against), and the
timing reduction takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2
N_PER_RANK = 48
N_BITS = 256


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import oracle
        from paper_1909_04750_gb300 import shard
        s = shard.plain_shard(rank, WORLD, N_PER_RANK, N_BITS)
        # keystreams of a few of this rank's instances, computed in the rank
        pick = [0, 7, N_PER_RANK - 1]
        ks = np.stack([np.frombuffer(oracle.stream(s.keys[i].tobytes(), s.ivs[i].tobytes(),
                                                   80, N_BITS), np.uint8) for i in pick])
        keys = torch.from_numpy(s.keys.copy())
        gathered = [torch.empty_like(keys) for _ in range(WORLD)]
        dist.all_gather(gathered, keys)
        shard.barrier()
        t_max = shard.max_over_ranks(1.5 + rank)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), keys=s.keys, ivs=s.ivs, ks=ks,
                 gathered=np.stack([g.numpy() for g in gathered]), t_max=t_max)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def ranks(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("shards"))
    mp.start_processes(_rank_main, args=(_free_port(), out), nprocs=WORLD, join=True,
                       start_method="spawn")
    return [dict(np.load(os.path.join(out, "rank%d.npz" % r))) for r in range(WORLD)]


def test_shards_tile_the_single_process_sequence(ranks):
    from paper_1909_04750_gb300 import workloads
    full = workloads.fixed_streams("plain_scale", 2, WORLD * N_PER_RANK, N_BITS)
    for r, d in enumerate(ranks):
        sl = slice(r * N_PER_RANK, (r + 1) * N_PER_RANK)
        assert np.array_equal(d["keys"], full.keys[sl])
        assert np.array_equal(d["ivs"], full.ivs[sl])
    # every rank saw the same, disjoint shards
    allk = ranks[0]["gathered"].reshape(-1, 10)
    assert np.array_equal(ranks[1]["gathered"].reshape(-1, 10), allk)
    assert len({k.tobytes() for k in allk}) == WORLD * N_PER_RANK


def test_keystream_same_in_shard_and_alone(ranks):
    import oracle
    from paper_1909_04750_gb300 import workloads
    full = workloads.fixed_streams("plain_scale", 2, WORLD * N_PER_RANK, N_BITS)
    for r, d in enumerate(ranks):
        for k, i in enumerate([0, 7, N_PER_RANK - 1]):
            g = r * N_PER_RANK + i
            alone = oracle.stream(full.keys[g].tobytes(), full.ivs[g].tobytes(), 80, N_BITS)
            assert d["ks"][k].tobytes() == alone


def test_max_over_ranks(ranks):
    assert all(float(d["t_max"]) == 1.5 + (WORLD - 1) for d in ranks)


def test_bounds_and_single_process_fallbacks():
    from paper_1909_04750_gb300 import shard
    assert shard.bounds(0, 4, 10) == (0, 10) and shard.bounds(3, 4, 10) == (30, 40)
    with pytest.raises(ValueError):
        shard.bounds(4, 4, 10)
    assert shard.max_over_ranks(2.5) == 2.5     # no process group
    shard.barrier()
