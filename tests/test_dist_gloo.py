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


def _bench_worker(rank, world, port, out_dir):
    """bench.py's timed region and throughput aggregation on a gloo world,
    with a CPU stand-in for the device step (rank r sleeps (r + 1) ms per
    step) and a host timer."""
    import sys
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = D.rank_world()
    assert (r, w) == (rank, world)
    calls = []

    def step():
        calls.append(1)
        time.sleep(0.001 * (rank + 1))

    def host_timer(fn, k):
        t0 = time.perf_counter()
        for _ in range(k):
            fn()
        dt = (time.perf_counter() - t0) * 1e3
        return dt, dt / k

    steps, warmup = 20, 3
    t_total, t_launch = bench.timed_region(step, steps, warmup, dist, lambda: None, host_timer)
    value = D.aggregate_throughput(1000.0, world, t_total / steps * 1e-3)
    np.save(os.path.join(out_dir, f"b{rank}.npy"), np.array([t_total, t_launch, value, len(calls)]))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_world2_bench_timed_region_takes_max_over_ranks(tmp_path):
    world = 2
    mp.start_processes(_bench_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"b{r}.npy") for r in range(world)]
    # every rank reports the same (maximum) duration: the slower rank's
    assert res[0][0] == res[1][0]
    assert res[0][0] >= 20 * 2.0 * 0.9          # rank 1 sleeps 2 ms per step
    assert res[1][1] > res[0][1]                # per-rank launch means differ
    # whole-job throughput: all ranks' units over the slowest rank's time
    assert res[0][2] == pytest.approx(1000.0 * world / (res[0][0] / 20 * 1e-3))
    # exactly warmup + steps calls of the step on each rank
    assert res[0][3] == res[1][3] == 23
