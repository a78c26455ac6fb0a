"""The benchmark's algorithmic work (the numerators of its roofline fractions) against a
brute-force count over the pairs, splits and candidate rows, and its row / prediction counts
against the FP64 oracle's own counters."""
import os
import sys

import numpy as np

import oracle
from paper_1910_07776_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


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
                if n >= 2:
                    fl = n ** 3 / 3 + 4 * n * n + 4 * n + 2 * n * cnt
                    if n <= nreg:
                        small += fl
                    else:
                        large += fl
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
    # the other stages' minimum work
    V = np.diff(batch.row_offsets).astype(float)
    assert w["gram_flops"] == float(np.sum(V * (V + 1) / 2 * 12 * 2))
    assert w["std_bytes"] == float(np.sum(V * 12) * (4 + 8))
    assert w["mask_bytes"] == float(splits.n_splits * 8)
