"""Multi-rank host logic on CPU (gloo, world size 2): points sharded across
ranks with their global index as restart key give the same rounds as one
process, the solved flags combine with an OR, the step time reduces with MAX,
and the ERWA counts summed over ranks give the single-process weights."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2308_15020_gb300 import gen

B_PER_RANK = 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = gen.uniform_3sat_100(4)
    x_all = gen.uniform_points(B_PER_RANK * world, inst.n, 9, dtype=np.float64)
    mine = x_all[rank * B_PER_RANK:(rank + 1) * B_PER_RANK]
    x1, solved, nun = O.step(inst, mine, T=30, lr=0.1, seed=3, epoch=2, b_offset=rank * B_PER_RANK, restart=True,
                             nthreads=1)
    xs = [torch.zeros(B_PER_RANK, inst.n, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(xs, torch.from_numpy(x1))
    any_solved = torch.tensor([int(solved.any())])
    dist.all_reduce(any_solved, op=dist.ReduceOp.MAX)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((torch.cat(xs).numpy(), int(any_solved.item()), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_rounds_equal_single_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got, any_solved, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst = gen.uniform_3sat_100(4)
    x_all = gen.uniform_points(B_PER_RANK * world, inst.n, 9, dtype=np.float64)
    want, solved, _ = O.step(inst, x_all, T=30, lr=0.1, seed=3, epoch=2, b_offset=0, restart=True, nthreads=1)
    assert np.array_equal(got, want)
    assert any_solved == int(solved.any())
    assert tmax == 2.0


def _erwa_worker(rank, world, port, out):
    from paper_2308_15020_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = gen.cnf_xor_2000(3, n=300)
    B = 13  # uneven split
    off, nb = shard.shard(B, rank, world)
    x_all = gen.uniform_points(B, inst.n, 21, dtype=np.float64)
    w = np.asarray(inst.weights, dtype=np.float64)
    for r in range(3):
        x1, solved, _ = O.step(inst, x_all[off:off + nb], T=5, lr=0.1, seed=4, epoch=r, b_offset=off, restart=False,
                               nthreads=1, weights=w)
        U = torch.from_numpy(O.unsat_counts(inst, x1))
        any_solved = shard.combine_round(torch.from_numpy(solved), U)
        w = O.erwa(U.numpy(), w, 0.4)
        x_all[off:off + nb] = O.rephase(x1, 2 if r % 2 == 0 else 1, solved, seed=4, epoch=100 + r, b_offset=off)
    xs = [torch.zeros(B, inst.n, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(xs, torch.from_numpy(x_all))
    if rank == 0:
        out.put((w, any_solved, [s.numpy() for s in xs]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_erwa_equals_single_process():
    from paper_2308_15020_gb300 import shard

    world = 2
    assert [shard.shard(13, r, 2) for r in range(2)] == [(0, 7), (7, 6)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_erwa_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    w_got, any_solved, xs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the same three rounds in one process over all 13 points
    inst = gen.cnf_xor_2000(3, n=300)
    x = gen.uniform_points(13, inst.n, 21, dtype=np.float64)
    w = np.asarray(inst.weights, dtype=np.float64)
    for r in range(3):
        x1, solved, _ = O.step(inst, x, T=5, lr=0.1, seed=4, epoch=r, restart=False, nthreads=1, weights=w)
        w = O.erwa(O.unsat_counts(inst, x1), w, 0.4)
        x = O.rephase(x1, 2 if r % 2 == 0 else 1, solved, seed=4, epoch=100 + r)
    assert np.array_equal(w_got, w)
    assert any_solved == bool(solved.any())
    got = np.concatenate([xs[0][:7], xs[1][7:]])
    assert np.array_equal(got, x)
