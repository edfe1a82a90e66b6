"""Two ranks over gloo (CPU): disjoint packet-id shards with a common weight
normalisation add up to the single-rank result.  The per-rank transport is the
oracle here; the GPU bench uses the same sharding with the CUDA library."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, out_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_1410_1629_gb300 import workloads as W
        from paper_1410_1629_gb300.sharding import shard
        prob = W.uniform_cube(channels=3)
        first, count, n_norm = shard(rank, world, n)
        r = O.run(prob, count, first_id=first, n_norm=n_norm)
        img = torch.from_numpy(r["images"][0].copy())
        ab = torch.from_numpy(r["absorption"].copy())
        st = torch.from_numpy(r["stats"].copy())
        cn = torch.from_numpy(r["counters"].astype(np.int64))
        for t in (img, ab, st, cn):
            dist.all_reduce(t)
        if rank == 0:
            np.savez(out_path, img=img.numpy(), ab=ab.numpy(), st=st.numpy(), cn=cn.numpy())
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_add_up_to_one_run(tmp_path):
    from oracle import oracle as O
    from paper_1410_1629_gb300 import workloads as W
    O.build()
    n = 1500
    out = str(tmp_path / "sum.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), n, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    ref = O.run(W.uniform_cube(channels=3), 2 * n)
    np.testing.assert_allclose(got["img"], ref["images"][0], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(got["ab"], ref["absorption"], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(got["st"], ref["stats"], rtol=1e-12)
    assert np.array_equal(got["cn"], ref["counters"].astype(np.int64))


def test_shard_arguments():
    from paper_1410_1629_gb300.sharding import shard
    assert shard(0, 1, 10) == (0, 10, 10)
    assert shard(3, 4, 10) == (30, 10, 40)
    with pytest.raises(ValueError):
        shard(4, 4, 10)
