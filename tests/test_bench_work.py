"""The benchmark's algorithmic work (the numerators of its roofline fractions) against counts
made another way: the FP64 operations of a fit by walking the loops of the register solver's
square-root-free LDL^T (factorisation, two forward solves, intercept, backward solve,
predictions) one operation at a time; the Gram's flops by a loop over the entries and
features of each program; the standardization's bytes from the arrays it reads and writes;
and the row / prediction counts from the FP64 oracle's own counters."""
import os
import sys

import numpy as np

import oracle
from paper_1910_07776_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _walk_fit(n, preds):
    """Operations of one fit of n pairs and its predictions, counted while walking the same
    loops as the solver: returns (FMAs, multiplies, reciprocals)."""
    fma = mul = rcp = 0
    for i in range(n):                 # factorisation, row i
        for k in range(i):
            for _m in range(k):
                fma += 1               # s -= c_m L_km
            mul += 1                   # L_ik = c_k / d_k
        for _m in range(i):
            fma += 1                   # d -= c_m L_im
        rcp += 1                       # 1 / d_i
    for i in range(n):                 # forward solves, two right-hand sides
        for _k in range(i):
            fma += 2
    for _i in range(n):                # num and den
        mul += 1
        fma += 2
    mul += 1                           # b = num / den
    rcp += 1
    for _i in range(n):                # D^-1 (t_y - b t_1)
        fma += 1
        mul += 1
    for i in range(n - 1, -1, -1):     # backward solve
        for _k in range(i + 1, n):
            fma += 1
    for _t in range(preds):            # b + sum_a alpha_a K[t][v_a]
        for _a in range(n):
            fma += 1
    return fma, mul, rcp


def test_fit_flops_match_an_operation_walk():
    for n in range(2, 40):
        for preds in (0, 1, 7):
            f, m, r = _walk_fit(n, preds)
            assert 2 * f + m + r == bench.fit_flops(n) + 2 * n * preds, (n, preds)


def _brute(batch, splits, k, nreg):
    small = large = 0.0
    rows = preds = 0
    for p in range(batch.n_programs):
        m = [int(x) for x in batch.masks[batch.program_rows(p)]]
        V = len(m)
        slot = {x: i for i, x in enumerate(m)}
        for s in range(int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])):
            T = int(splits.train_masks[s])
            train = [v for v in range(V) if (T >> v) & 1]
            test = [t for t in range(V) if not (T >> t) & 1]
            rows += len(test)
            for j in range(6):
                n = sum(1 for v in train if not (m[v] >> j) & 1 and (m[v] | 1 << j) in slot
                        and (T >> slot[m[v] | 1 << j]) & 1)
                cnt = sum(1 for t in test if not (m[t] >> j) & 1)
                if n > 0:
                    preds += cnt
                if n >= 2:             # one pair: alpha = 0 and b = y, no arithmetic
                    f, mu, r = _walk_fit(n, cnt)
                    if n <= nreg:
                        small += 2 * f + mu + r
                    else:
                        large += 2 * f + mu + r
    rank_bytes = rows * (1 + 4 + 4 + 8 * k) + 8 * preds
    return small, large, rows, preds, rank_bytes


def test_algorithmic_work_matches_brute_force_and_the_oracle():
    batch = synth.make_batch(4, versions=(6, 40), feat=12, dtype=np.float32, seed=7)
    splits = synth.make_splits(batch, "frac", 9, seed=7)
    w = bench.algorithmic_work(batch, splits, k=3, nreg=10)
    small, large, rows, preds, rank_bytes = _brute(batch, splits, 3, 10)
    assert np.isclose(w["solve_small"], small, rtol=1e-12)
    assert np.isclose(w["solve_large"], large, rtol=1e-12)
    assert (w["rows"], w["preds"]) == (rows, preds)
    assert w["rank_bytes"] == rank_bytes
    # the oracle counts the same rows and predictions (no fit fails on these inputs)
    r = oracle.cv_batch(batch, splits)
    assert (r.fit_status != oracle.FIT_NOTPD).all()
    assert r.counter("n_rows") == rows and r.counter("n_pred") == preds
    # the Gram: one dot product of F features (an FMA each) per entry of the upper triangle
    gram = 0
    for p in range(batch.n_programs):
        V, F = batch.versions(p), int(batch.feat_width[p])
        for a in range(V):
            for b in range(a, V):
                gram += 2 * F
    assert w["gram_flops"] == gram
    # the standardization reads X (float32 here) and writes Z (float64), both [rows][F]
    Z = np.empty(batch.X.shape[0], dtype=np.float64)
    assert w["std_bytes"] == batch.X.nbytes + Z.nbytes
    assert w["mask_bytes"] == splits.train_masks.nbytes
