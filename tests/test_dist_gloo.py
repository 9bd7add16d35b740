"""The multi-rank path on the CPU (gloo, world size 2): element shards are
disjoint and cover the mesh, the sharded residual (computed per rank, no
exchange) equals the unsharded one, and the timing reduction takes the
maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2306_11665_gb300 import dist as D


def test_shard_cover_and_balance():
    for n in (0, 1, 7, 64, 32768, 100001):
        for world in (1, 2, 3, 8):
            ranges = [D.shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(10, 2, 2)
    assert D.aggregate_throughput(4.096e6, 4, 0.5) == pytest.approx(4 * 4.096e6 / 0.5)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import oracle as O
    from paper_2306_11665_gb300 import inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u, Ja = I.workload(3, 3, 0, 3)                     # 27 elements, the same mesh on every rank
    e0, e1 = D.shard(u.shape[0], rank, world)
    r = O.volume_sf(3, 3, 0, O.FLUX_EULER, u[e0:e1], Ja[e0:e1])   # no exchange of element data
    np.save(os.path.join(out_dir, f"r{rank}.npy"), r)
    t = D.max_over_ranks(1.0 + rank, dist)             # each rank's "time"
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_sharded_equals_whole(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    import oracle as O
    from paper_2306_11665_gb300 import inputs as I
    u, Ja = I.workload(3, 3, 0, 3)
    whole = O.volume_sf(3, 3, 0, O.FLUX_EULER, u, Ja)
    parts = np.concatenate([np.load(tmp_path / f"r{r}.npy") for r in range(world)])
    assert np.array_equal(parts, whole)
    for r in range(world):
        assert np.load(tmp_path / f"t{r}.npy")[0] == world   # max over ranks of 1, 2
