"""Restart sharding across ranks (the multi-GPU path) on CPU with gloo.

Restarts are independent (Sec. 3.3), so N GPUs each run their own block of
restarts with no data-path collective; initial points are keyed by the
global restart id (r_offset), so the union of the shards equals one run over
all restarts.  Timing takes the maximum over ranks.  The per-rank compute here
is the CPU oracle (the shard/merge logic is what is under test).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from oracle import cls as ocls

R_LOCAL, STEPS, LR, SEED = 6, 3, 0.1, 42


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _solve(inst, X):
    for _ in range(STEPS):
        _, g, _ = ocls.objective_grad(inst, X.astype(np.float64))
        X = ocls.pgd_step(X, g.astype(np.float32), LR)
    nsat, _, _ = ocls.score(inst, X)
    return X, nsat


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = W.random_ksat(n=30, m=120)
    X = ocls.init_uniform(inst.n, R_LOCAL, SEED, r_offset=rank * R_LOCAL)
    X, nsat = _solve(inst, X)
    got = [torch.zeros(R_LOCAL, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, torch.from_numpy(nsat))
    t = torch.tensor([float(rank + 1)])            # this rank's time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((torch.cat(got).numpy(), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_restarts_equal_single_run(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst = W.random_ksat(n=30, m=120)
    X = ocls.init_uniform(inst.n, world * R_LOCAL, SEED)
    _, nsat = _solve(inst, X)
    assert np.array_equal(merged, nsat)
    assert tmax == float(world)
