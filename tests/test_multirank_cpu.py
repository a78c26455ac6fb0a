"""The benchmark's multi-rank path (a job of N workloads split over N ranks by the longest-
processing-time rule, weak scaling, time = slowest rank, work = sum over ranks) with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank takes its share of the job, as bench.py does under torchrun
    b, s = bench.rank_inputs(rank, world)
    import oracle
    recs = int(oracle.rec_offsets(b, s)[-1])
    ms = 10.0 * (rank + 1)
    t, r = bench.aggregate_over_ranks(ms, recs, world, torch.device("cpu"))
    q.put((rank, recs, t, r))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    total = sum(o[1] for o in out)
    import bench
    import oracle
    b, s = bench.make_inputs(bench.CFG["seed"], 2 * bench.CFG["programs"])
    assert total == int(oracle.rec_offsets(b, s)[-1])     # the shares cover the whole job
    for rank, recs, t, r in out:
        assert t == 20.0            # the slowest rank's time
        assert r == total           # all ranks' recommendations
    assert abs(out[0][1] - out[1][1]) < 0.02 * total     # balanced shares
