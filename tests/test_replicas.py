"""Replica (multi-rank) host logic of bench.py on CPU with gloo, world size 2.

Each rank counts its own graph (replicas, weak scaling); the only collectives
are the barrier and the max / sum reductions of the timing.  Here the ranks
run the oracle instead of a GPU so the rank plumbing is exercised without one.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2403_02997_gb300 import gen

    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    spec = bench.replica_spec(gen.rmat_spec(10, 8, 2), r)
    src, dst = spec.edges()
    res = oracle.count(spec.n, src, dst, 0)
    bench.barrier(w)
    t_max = bench.max_over_ranks(float(rank + 1), w)
    e_sum = bench.sum_over_ranks(float(res["m"]), w)
    out[rank] = (spec.seed, res["T"], t_max, e_sum, res["m"])
    dist.destroy_process_group()


def test_two_rank_replicas():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    seeds = [out[r][0] for r in range(world)]
    assert len(set(seeds)) == world                  # each rank has its own replica graph
    assert all(out[r][2] == float(world) for r in range(world))       # max over ranks
    total = sum(out[r][4] for r in range(world))
    assert all(out[r][3] == float(total) for r in range(world))       # whole-job edges
