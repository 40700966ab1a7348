"""The halo exchange of block sharding on the CPU, over gloo with world size
2 (the paper partitions its blocks over processes and exchanges the
populations that leave each partition, Sections 1 and 3.2).  Each rank holds
the x-slab of one part of a periodic grid (the cuts of lbm_shard_plan) in
float64, sends the boundary layers' populations that cross each cut
(e_x = +1 of its last layer to the right neighbour, e_x = -1 of its first
layer to the left one, the periodic wrap included), receives its two halo
layers, pull-streams and collides its own cells with the oracle's collision,
and must get the oracle's unsharded step on that slab.  The populations of
the halo layers that are not exchanged are NaN, so a pull that would need one
fails the comparison: the exchange plan (which layer, which populations, in
which direction) is complete.  The plan itself is host code of the library
(no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, model, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import synth
    from oracle.collision import Model
    from oracle.lattice import velocities, weights
    from oracle.solver import NestedSolver
    from paper_1206_0389_gb300 import lbm
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nb, omega, cs = (4, 2, 2), 1.6, 0.1 if model == "d3q19" else 0.0
    cuts = lbm.lbm_shard_plan(nb, world)
    Q = 19 if model == "d3q19" else 27
    NX, NY, NZ = 8 * nb[0], 8 * nb[1], 8 * nb[2]
    w = weights(Q).numpy()
    base = w if model == "d3q27" else 0.01 * w
    f = synth.random_distributions(Q, (NZ, NY, NX), 31, amp=0.05, base=base)
    # the unsharded step (every rank computes it for the comparison)
    full = NestedSolver(model, nb, periodic_x=True, omega=omega, cs=cs)
    full.set_state(0, torch.from_numpy(f))
    full.step(1)
    expect = full.state(0).numpy()
    x0, x1 = 8 * cuts[rank], 8 * cuts[rank + 1]
    mine = f[:, :, :, x0:x1]
    e = velocities(Q).numpy()
    plus = [i for i in range(Q) if e[i, 0] == 1]
    minus = [i for i in range(Q) if e[i, 0] == -1]
    right, left = (rank + 1) % world, (rank - 1) % world
    # exchange: e_x = +1 of my last layer to the right, e_x = -1 of my first to the left
    send_r = torch.from_numpy(np.ascontiguousarray(mine[plus, :, :, -1]))
    send_l = torch.from_numpy(np.ascontiguousarray(mine[minus, :, :, 0]))
    recv_l = torch.empty_like(send_r)
    recv_r = torch.empty_like(send_l)
    reqs = [dist.isend(send_r, right), dist.isend(send_l, left), dist.irecv(recv_l, left), dist.irecv(recv_r, right)]
    for q in reqs:
        q.wait()
    pad = np.full((Q, NZ, NY, x1 - x0 + 2), np.nan)
    pad[:, :, :, 1:-1] = mine
    pad[plus, :, :, 0] = recv_l.numpy()
    pad[minus, :, :, -1] = recv_r.numpy()
    pre = np.empty_like(mine)
    for i in range(Q):
        ex, ey, ez = (int(v) for v in e[i])
        pre[i] = np.roll(pad[i], shift=(ez, ey, ex), axis=(0, 1, 2))[:, :, 1:-1]
    ok_pull = bool(np.isfinite(pre).all())
    got, _ = Model(model).collide(torch.from_numpy(pre.reshape(Q, -1)), omega, cs)
    got = got.numpy().reshape(mine.shape)
    err = float(np.abs(got - expect[:, :, :, x0:x1]).max()) if ok_pull else float("inf")
    out[rank] = (ok_pull, err, cuts, len(plus))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("model", ["d3q19", "d3q27"])
def test_halo_exchange_over_gloo_reproduces_the_unsharded_step(model):
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), model, out), nprocs=world, join=True)
    for r in range(world):
        ok_pull, err, cuts, nq = out[r]
        assert cuts == [0, 2, 4]
        assert nq == (5 if model == "d3q19" else 9)      # populations crossing each cut
        assert ok_pull, "a pull needed a halo population that is not exchanged"
        assert err <= 1e-14, err


def test_shard_plan_cuts_keep_clear_of_refinement_and_balance_work():
    import synth
    from paper_1206_0389_gb300 import lbm
    assert lbm.lbm_shard_plan((8, 2, 2), 4) == [0, 2, 4, 6, 8]
    assert lbm.lbm_shard_plan((9, 2, 2), 3, periodic_x=False) == [0, 3, 6, 9]
    flags, _ = synth.jet_paper_scale()                  # refined over x < 192 (24 columns)
    cuts = lbm.lbm_shard_plan((64, 32, 32), 4, periodic_x=False, refine=flags)
    assert cuts[0] == 0 and cuts[-1] == 64 and cuts[1] >= 26
    assert all(b - a >= 1 for a, b in zip(cuts, cuts[1:]))
    # the parts after the refined one share the rest evenly
    rest = [b - a for a, b in zip(cuts[1:], cuts[2:])]
    assert max(rest) - min(rest) <= 1
    flags2, _ = synth.jet_two_level(8, 4, 4, radius=8.0)  # refined along the whole x extent
    with pytest.raises(lbm.LbmError):
        lbm.lbm_shard_plan((8, 4, 4), 2, periodic_x=False, refine=flags2)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_shard_plan((2, 2, 2), 3)                  # more parts than columns
