"""Run-range sharding through the library: two processes, each with its own
context on the same GPU, search disjoint run ranges of one search with
xyz_search_range, gather their pair lists over a gloo group and merge them
on the host; the merged list must equal the whole search and the oracle's.
The two processes' kernels never wait on one another (the only exchange is
the host-side gather after both searches returned)."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data():
    from paper_1610_05108_gb300 import synth
    return synth.iid(300, 5000, 7, flip=0.15)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1610_05108_gb300 import shard, xyz
    xyz.load()
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = _data()
        L, M, kappa, seed = 60, 10, 0.3, 31
        with xyz.create(d.X, d.Y) as ctx:
            merged = shard.search_sharded(lambda a, b: ctx.search_range(a, b, M, kappa, seed), L, rank, world)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), merged)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_search_two_processes_one_gpu(tmp_path, orc):
    import torch.multiprocessing as mp

    from paper_1610_05108_gb300 import build, xyz
    build.build()
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    d = _data()
    L, M, kappa, seed = 60, 10, 0.3, 31
    want = orc.xyz(d.X, d.Y, L, M, kappa, seed).astype(np.int64)
    xyz.load()
    with xyz.create(d.X, d.Y) as ctx:
        res = ctx.search(L, M, kappa, seed)
    whole = np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int64)
    assert len(want) > 0 and np.array_equal(whole, want)
    for r in range(world):
        assert np.array_equal(np.load(os.path.join(tmp_path, f"rank{r}.npy")), want)
