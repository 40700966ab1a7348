"""The replica harness of bench.py on CPU: world size 2 over gloo.  Each rank
reports its own time and update count; the job value must use the max time
over ranks and the sum of updates (replicas only: no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    dist = bench.dist_init(w, "gloo")
    bench.barrier(dist)
    my_ms = 10.0 + 5.0 * rank            # rank 1 is the slow replica
    my_updates = 1000.0 * (rank + 1)
    ms = bench.max_over_ranks(dist, my_ms)
    upd = bench.sum_over_ranks(dist, my_updates)
    out[rank] = bench.whole_job_mlups(upd, ms)
    bench.barrier(dist)
    dist.destroy_process_group()


def test_replicas_use_max_time_and_summed_updates():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    expect = 3000.0 / (15.0e-3) / 1e6
    assert out[0] == pytest.approx(expect) and out[1] == pytest.approx(expect)


def test_single_rank_is_identity():
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 2.0) == 2.0
    assert bench.whole_job_mlups(1e6, 1.0) == pytest.approx(1000.0)
