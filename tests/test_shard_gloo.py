"""Run-range sharding across processes: world-size-2 gloo ranks on CPU, each
searching its run range with the oracle, gathered and merged on the host,
must equal the single-process search."""
import os
import socket

import numpy as np
import pytest

from paper_1610_05108_gb300 import shard


def test_run_ranges_cover_disjointly():
    for L in (0, 1, 2, 7, 100, 15259):
        for world in (1, 2, 3, 8):
            rr = shard.run_ranges(L, world)
            assert len(rr) == world
            assert rr[0][0] == 0 and rr[-1][1] == L
            for (a, b), (c, d) in zip(rr, rr[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in rr]
            assert max(sizes) - min(sizes) <= 1


def test_merge_rejects_disagreeing_counts():
    a = np.array([[1, 2, 10]])
    b = np.array([[1, 2, 11]])
    with pytest.raises(ValueError):
        shard.merge_pairs([a, b])
    m = shard.merge_pairs([np.array([[3, 4, 5], [1, 2, 9]]), np.array([[1, 2, 9]])])
    assert m.tolist() == [[1, 2, 9], [3, 4, 5]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1610_05108_gb300 import shard as sh
    from paper_1610_05108_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = synth.iid(120, 400, 5, flip=0.2)
        L, M, kappa, seed = 23, 6, 0.2, 77
        merged = sh.search_sharded(lambda a, b: oracle.xyz_range(d.X, d.Y, a, b, M, kappa, seed),
                                   L, rank, world)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), merged)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_search_equals_whole_search_gloo(tmp_path, orc):
    import torch.multiprocessing as mp

    from paper_1610_05108_gb300 import synth
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    d = synth.iid(120, 400, 5, flip=0.2)
    whole = orc.xyz(d.X, d.Y, 23, 6, 0.2, 77)
    assert len(whole) > 0
    for r in range(world):
        got = np.load(os.path.join(tmp_path, f"rank{r}.npy"))
        assert np.array_equal(got, whole.astype(np.int64))
