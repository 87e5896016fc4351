"""Replica layout on two CPU ranks (gloo): shards, seeds and the max-reduced
job time, with each rank computing its shard of pairs (oracle, CPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2011_11134_gb300.replicas import replica_seed, shard_range


def test_shard_range_covers_exactly_once():
    for n in (0, 1, 7, 4096, 1_000_003):
        for world in (1, 2, 3, 8):
            got = [shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[r][1] == got[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_2011_11134_gb300 import workloads as W
    from paper_2011_11134_gb300.replicas import max_over_ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = W.paired_rect_4096(seed=0, n=1000)
    a, b = shard_range(1000, rank, world)
    o = oracle.iou_paired(d["p1"][a:b], d["p2"][a:b])
    np.save(os.path.join(out_dir, f"iou_{rank}.npy"), o["iou"])
    t = max_over_ranks(float(rank + 1) * 0.5)
    np.save(os.path.join(out_dir, f"t_{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path, orc):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    from paper_2011_11134_gb300 import workloads as W

    d = W.paired_rect_4096(seed=0, n=1000)
    full = orc.iou_paired(d["p1"], d["p2"])["iou"]
    parts = np.concatenate([np.load(tmp_path / f"iou_{r}.npy") for r in range(world)])
    np.testing.assert_array_equal(parts, full)
    for r in range(world):
        assert float(np.load(tmp_path / f"t_{r}.npy")[0]) == 1.0  # max of 0.5, 1.0
    assert replica_seed(3) == 3
