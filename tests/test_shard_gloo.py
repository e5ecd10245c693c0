"""Multi-rank partitioning of independent evaluations, checked on CPU with gloo ranks.

The partition must cover every item exactly once, balance the estimated cost, and the
gathered results (here computed per rank by the CPU oracle standing in for each rank's
GPU) must match the single-process evaluation item by item."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2312_17396_gb300 import inputs, shard


def test_partition_covers_and_balances():
    mats, degs = inputs.uneven_batch(200, 8, 256, 0.1, 10.0, seed=3)
    ns = [a.shape[0] for a in mats]
    norms = [float(np.abs(a).sum(axis=0).max()) for a in mats]
    for world in (1, 2, 3, 8):
        sh = shard.partition(ns, degs, norms, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(mats)))
        loads = shard.shard_loads(ns, degs, norms, sh)
        biggest = max(shard.cost(n, m, a) for n, m, a in zip(ns, degs, norms))
        assert max(loads) - min(loads) <= biggest      # LPT bound
    assert shard.partition(ns, degs, norms, 4) == shard.partition(ns, degs, norms, 4)


def test_cost_model_counts():
    assert shard.cost(10, 16, 0.5) == (3 + 4) * 1000       # s = 4, r = 4, no squaring
    assert shard.cost(10, 30, 4.0) == (5 + 5 + 2) * 1000   # s = 6, r = 5, sigma = 2
    assert shard.squarings(32.0) == 5 and shard.squarings(33.0) == 6 and shard.squarings(1.0) == 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mats, degs = inputs.uneven_batch(9, 3, 12, 0.2, 6.0, seed=5)
    ns = [a.shape[0] for a in mats]
    norms = [float(np.abs(a).sum(axis=0).max()) for a in mats]
    mine = shard.partition(ns, degs, norms, world)[rank]
    res = []
    for i in mine:   # each rank's evaluation (CPU oracle standing in for the rank's GPU)
        sg = oracle.sigma_for(mats[i])
        eh, el = oracle.expm_ss_dd(mats[i], degs[i], sg)
        res.append(torch.from_numpy(eh + el))
    allres = shard.gather_results(mine, res, len(mats))
    if rank == 0:
        q.put([r.numpy() for r in allres])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_in_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mats, degs = inputs.uneven_batch(9, 3, 12, 0.2, 6.0, seed=5)
    for A, m, E in zip(mats, degs, got):
        sg = oracle.sigma_for(A)
        eh, el = oracle.expm_ss_dd(A, m, sg)
        assert np.array_equal(E, eh + el)
