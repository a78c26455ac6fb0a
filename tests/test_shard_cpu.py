"""The multi-GPU form of the batched pass, on the CPU: the longest-processing-time partition of
one batch's programs (balance against brute force and the list-scheduling bound), and two gloo
ranks that each run the FP64 reference on their share -- the summed counters and the gathered
recommendations equal one rank's run over the whole batch bit for bit -- and that average the
surrogate's gradients over halves of a minibatch (equal to the whole minibatch's gradient)."""
import itertools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1910_07776_gb300 import shard, synth


def _brute_opt(costs, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = np.zeros(m)
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, loads.max())
    return best


@pytest.mark.parametrize("m", [2, 3])
def test_lpt_is_within_grahams_bound_of_the_optimum(m):
    rng = np.random.default_rng(m)
    for _ in range(20):
        costs = rng.integers(1, 50, size=8).astype(float)
        parts = shard.lpt_partition(costs, m)
        assert sorted(np.concatenate(parts).tolist()) == list(range(8))
        worst = max(costs[p].sum() for p in parts)
        assert worst <= (4 / 3 - 1 / (3 * m)) * _brute_opt(costs, m) + 1e-9


def test_lpt_on_many_programs_meets_the_list_scheduling_bound():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0, 1, size=1000)
    for m in (2, 4, 8):
        parts = shard.lpt_partition(costs, m)
        loads = [costs[p].sum() for p in parts]
        assert max(loads) <= costs.sum() / m + costs.max()
        assert max(loads) / min(loads) < 1.01


def test_program_costs_grow_with_splits_versions_and_features():
    def cost(V, F, S):
        b = synth.make_batch(1, versions=V, feat=F, seed=3)
        return shard.program_costs(b, synth.make_splits(b, "half", S, seed=3))[0]
    assert cost(16, 64, 10) < cost(64, 64, 10) < cost(64, 256, 10) < cost(64, 256, 20)


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _job():
    b = synth.make_batch(7, versions=(8, 64), feat=12, seed=13)
    s = synth.make_splits(b, "half", 11, seed=13)
    return b, s


def _cv_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    b, s = _job()
    mine = shard.lpt_partition(shard.program_costs(b, s), world)[rank]
    sb, ss = shard.shard(b, s, mine)
    r = oracle.cv_batch(sb, ss)
    cnt = torch.from_numpy(r.counters.astype(np.uint64).view(np.int64).copy())
    shard.allreduce_counters(cnt)
    codes = shard.gather_rec_codes(b, s, mine, r.rec_offsets, r.rec_code)
    if rank == 0:
        q.put((cnt.numpy().view(np.uint64).tolist(), codes.tolist(), [len(p) for p in [mine]]))
    dist.destroy_process_group()


def _grad_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import mlp
    rng = np.random.default_rng(17)
    X = rng.normal(size=(16, 256))
    Y = 0.3 * rng.normal(size=(16, 6))
    p = mlp.init_params(17)
    half = slice(8 * rank, 8 * (rank + 1))
    _, g = mlp.loss_and_grads(p, X[half], Y[half])
    out = {}
    for k in mlp.NAMES:
        t = torch.from_numpy(g[k].copy())
        shard.allreduce_mean_(t)
        out[k] = t.numpy()
    if rank == 0:
        _, full = mlp.loss_and_grads(p, X, Y)
        q.put(max(float(np.abs(out[k] - full[k]).max() / (np.abs(full[k]).max() + 1e-300)) for k in mlp.NAMES))
    dist.destroy_process_group()


def _spawn(target, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = q.get(timeout=180)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return res


def test_two_ranks_on_lpt_shards_equal_one_rank_on_the_batch():
    import oracle
    counters, codes, _ = _spawn(_cv_worker)
    b, s = _job()
    ref = oracle.cv_batch(b, s)
    assert counters == ref.counters.astype(np.uint64).tolist()
    assert codes == ref.rec_code.tolist()


def test_data_parallel_gradient_average_equals_the_whole_minibatch():
    assert _spawn(_grad_worker) < 1e-12
