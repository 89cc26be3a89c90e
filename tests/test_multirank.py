"""Multi-rank host logic on CPU (gloo, world size 2): points sharded across
ranks with their global index as restart key give the same rounds as one
process, the solved flags combine with an OR, and the step time reduces with MAX."""
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
