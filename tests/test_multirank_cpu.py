"""The benchmark's multi-rank path (one batch per rank, weak scaling, time = slowest rank,
work = sum over ranks) with two gloo ranks on the CPU."""
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
    from paper_1910_07776_gb300 import synth
    # each rank draws its own batch (seed = rank), as bench.py does under torchrun
    b = synth.make_batch(2, versions=(16, 64), feat=16, seed=rank)
    s = synth.make_half_splits_fast(b, 8, seed=rank)
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
    for rank, recs, t, r in out:
        assert t == 20.0            # the slowest rank's time
        assert r == total           # all ranks' recommendations
    assert out[0][1] != out[1][1]   # different batches per rank
