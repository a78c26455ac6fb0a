"""One job's programs split across ranks (one process per GPU), and the merge of what the ranks
produce: the multi-GPU form of the batched cross-validation pass.

The programs of a batch, and the train/test splits of each, are independent: every fit uses
its own program's versions only (Sec. 5: the models are trained and scored per program and
split).  So the ranks exchange nothing on the data path.  Programs are assigned by the
longest-processing-time rule on an estimate of their work, S_p (n_p^3 + V_p^2 F_p) with S_p
splits, V_p versions, F_p features and n_p the mean number of training pairs per fit; the job
ends with a sum of the 16 accuracy counters over the ranks and, when wanted, a gather of the
recommendations in the batch's split order.  The surrogate's data-parallel training averages
each step's gradients over the ranks (allreduce_mean_) before the optimizer step.

Host-side logic only (numpy and torch.distributed); every step of the pass runs in the CUDA
library on each rank."""
from __future__ import annotations

import heapq
from typing import List, Sequence, Tuple

import numpy as np

from . import synth


def _popcount64(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    c = np.zeros(x.shape, dtype=np.int64)
    for b in range(64):
        c += ((x >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return c


def program_costs(batch: synth.ProgramBatch, splits: synth.Splits) -> np.ndarray:
    """Estimated work of each program, S_p (n_p^3 + V_p^2 F_p): S_p fits' factorisations of
    n_p pairs (n_p = the pairs of each optimization present in the program, times the mean
    fraction of its splits' train masks squared, averaged over the six optimizations) and the
    program's Gram block (V_p^2 F_p)."""
    P = batch.n_programs
    out = np.zeros(P, dtype=np.float64)
    for p in range(P):
        m = batch.masks[batch.program_rows(p)].astype(np.int64)
        V, F = len(m), float(batch.feat_width[p])
        s0, s1 = int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])
        S = s1 - s0
        if S == 0 or V == 0:
            out[p] = V * V * F
            continue
        present = set(int(x) for x in m)
        pairs = np.mean([sum(1 for x in m if not (x >> j) & 1 and (int(x) | (1 << j)) in present)
                         for j in range(6)])
        full = np.uint64((1 << V) - 1) if V < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        frac = float(np.mean(_popcount64(splits.train_masks[s0:s1] & full))) / V
        n = pairs * frac * frac
        out[p] = S * (n ** 3 + V * V * F)
    return out


def lpt_partition(costs: Sequence[float], world: int) -> List[np.ndarray]:
    """Longest processing time first: programs in descending cost (ties: lower index first),
    each to the rank with the least load so far (ties: lower rank).  Returns each rank's
    programs in ascending order.  The largest load is at most (4/3 - 1/(3 world)) times the
    optimum (Graham 1969)."""
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    own: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        own[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [np.array(sorted(o), dtype=np.int64) for o in own]


def shard(batch: synth.ProgramBatch, splits: synth.Splits,
          programs: Sequence[int]) -> Tuple[synth.ProgramBatch, synth.Splits]:
    """The sub-batch of the given programs (in that order) and their splits."""
    sub = synth.take_programs(batch, list(int(p) for p in programs))
    offs, tm = [0], []
    for p in programs:
        s0, s1 = int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])
        tm.append(splits.train_masks[s0:s1])
        offs.append(offs[-1] + (s1 - s0))
    tms = np.concatenate(tm) if tm else np.zeros(0, dtype=np.uint64)
    return sub, synth.Splits(split_offsets=np.array(offs, dtype=np.int64), train_masks=tms.astype(np.uint64))


def allreduce_counters(counters, group=None):
    """Sum of the 16 accuracy counters (uint64) over the ranks, in place; returns them."""
    import torch
    import torch.distributed as dist
    t = counters.view(torch.int64) if counters.dtype != torch.int64 else counters
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return counters


def allreduce_mean_(tensor, group=None):
    """Average of a tensor over the ranks, in place (the data-parallel gradient exchange)."""
    import torch.distributed as dist
    dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    tensor /= dist.get_world_size(group)
    return tensor


def gather_rec_codes(batch: synth.ProgramBatch, splits: synth.Splits, programs: Sequence[int],
                     rec_offsets: np.ndarray, rec_code: np.ndarray, group=None):
    """This rank's recommendation codes (rows of its shard's splits, program by program in
    `programs` order) gathered on rank 0 into the full batch's row order (split by split,
    test slots ascending).  Returns the full array on rank 0, None elsewhere."""
    import torch.distributed as dist
    obj = (np.asarray(programs, dtype=np.int64), np.asarray(rec_offsets, dtype=np.int64),
           np.asarray(rec_code))
    got = [None] * dist.get_world_size(group)
    dist.all_gather_object(got, obj, group=group)
    if dist.get_rank(group) != 0:
        return None
    V = np.diff(batch.row_offsets).astype(np.int64)
    S = splits.n_splits
    split_prog = np.repeat(np.arange(batch.n_programs), np.diff(splits.split_offsets))
    full = np.where(V[split_prog] >= 64, np.uint64(0xFFFFFFFFFFFFFFFF),
                    (np.uint64(1) << V[split_prog].astype(np.uint64)) - np.uint64(1))
    rows = V[split_prog] - _popcount64(splits.train_masks & full)
    g_off = np.zeros(S + 1, dtype=np.int64)
    g_off[1:] = np.cumsum(rows)
    out = np.zeros(int(g_off[-1]), dtype=np.asarray(rec_code).dtype)
    for progs, ro, code in got:
        k = 0                                   # split index inside the shard
        for p in progs:
            s0, s1 = int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])
            for s in range(s0, s1):
                out[g_off[s]:g_off[s + 1]] = code[ro[k]:ro[k + 1]]
                k += 1
    return out
