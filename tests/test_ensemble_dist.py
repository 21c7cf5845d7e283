"""Event sharding across ranks, on CPU: world-size-2 gloo process groups run
the host logic of paper_1604_03360_gb300.ensemble with a CPU shard runner (the
oracle), including a rank that raises and has its events reassigned."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1604_03360_gb300.ensemble import lpt_shards, run_ensemble

SIZES = [(8, 7, 6), (5, 9, 7), (10, 6, 5), (6, 6, 6), (7, 5, 9)]


def _oracle_runner(fail_rank, rank, rnd_box):
    import oracle
    import workloads as W

    def run(events):
        rnd_box[0] += 1
        if rank == fail_rank and rnd_box[0] == 1:
            raise RuntimeError("injected failure on rank %d" % rank)
        out = {}
        for e in events:
            g, w = W.lumpy(n=SIZES[e], seed=300 + e)
            c = oracle.make_cfg(g.n, g.dx, cfl=g.cfl)
            u, t, k = oracle.run(c, oracle.prim2con(w), 2)
            out[e] = (t, k, float(np.sum(u[0])))
        return out
    return run


def _worker(rank, world, port, fail_rank, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [int(np.prod(s)) for s in SIZES]
        res, fails = run_ensemble(costs, _oracle_runner(fail_rank, rank, [0]), rank, world, dist)
        q.put((rank, res, fails))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run(world, fail_rank):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, fail_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def _serial():
    res, fails = run_ensemble([int(np.prod(s)) for s in SIZES], _oracle_runner(-1, 0, [0]), 0, 1, None)
    assert not fails
    return res


def test_lpt_balances_and_covers():
    costs = [9, 7, 6, 5, 5, 4, 3, 1]
    sh = lpt_shards(costs, [0, 1, 2])
    assert sorted(i for v in sh.values() for i in v) == list(range(len(costs)))
    loads = [sum(costs[i] for i in v) for v in sh.values()]
    assert max(loads) - min(loads) <= max(costs)


def test_two_ranks_match_serial():
    ref = _serial()
    for rank, res, fails in _run(2, fail_rank=-1):
        assert not fails
        assert res.keys() == ref.keys()
        for e in ref:
            assert res[e] == ref[e]


def test_failed_rank_events_are_reassigned():
    ref = _serial()
    for rank, res, fails in _run(2, fail_rank=1):
        assert len(fails) == 1 and fails[0][1] == 1 and "injected failure" in fails[0][2]
        assert res.keys() == ref.keys()
        for e in ref:
            assert res[e] == ref[e]
