"""Pins of the oracle's instance-based learner (Sec. 3.4: IBK, k = 10 nearest neighbours by
Euclidean distance; the neighbours' labels are continuous log speedups and their mean is the
prediction).  Each pin comes from outside the oracle's own code: a numpy brute force, the
paper's remark that IBK reproduces the labels of its training instances, closed forms."""
import numpy as np
import pytest

import oracle
from paper_1910_07776_gb300 import synth


def _brute(Z, y, zt, k):
    """Nearest k by (squared distance, index), mean of their labels in index order."""
    d = ((Z - zt) ** 2).sum(axis=1)
    order = np.lexsort((np.arange(len(d)), d))[:k]
    return float(np.sum(y[np.sort(order)]) / len(order))


@pytest.mark.parametrize("k", [1, 3, 10, 40])
def test_ibk_single_prediction_matches_brute_force(k):
    rng = np.random.default_rng(k)
    for trial in range(40):
        n = int(rng.integers(1, 33))
        F = int(rng.integers(1, 20))
        Z = rng.normal(size=(n, F))
        if n > 3:                                   # exact ties: repeated training rows
            Z[1] = Z[0]
            Z[n - 1] = Z[2]
        y = rng.normal(size=n)
        zt = Z[int(rng.integers(0, n))] if trial % 3 == 0 else rng.normal(size=F)
        assert abs(oracle.ibk_predict(Z, y, zt, k) - _brute(Z, y, zt, k)) <= 1e-12


def test_ibk_reproduces_a_training_label_exactly():
    # Sec. 6: IBK stores all training instances, so a test vector equal to one of them is
    # predicted with that instance's label (k = 1)
    rng = np.random.default_rng(3)
    Z = rng.normal(size=(20, 8))
    y = rng.normal(size=20)
    for i in range(20):
        assert oracle.ibk_predict(Z, y, Z[i].copy(), 1) == y[i]


def test_ibk_fewer_pairs_than_k_predict_the_train_mean():
    # n <= k: every training pair is a neighbour, so each candidate of the fit gets the mean
    # label of the fit's training pairs, whatever its features
    batch = synth.make_batch(3, versions=(12, 24), feat=16, dtype=np.float64, seed=5)
    splits = synth.make_splits(batch, "half", 6, seed=5)
    r = oracle.cv_batch(batch, splits, model="ibk")
    checked = 0
    row = 0
    for p in range(batch.n_programs):
        V = batch.versions(p)
        rows = batch.program_rows(p)
        m = batch.masks[rows].astype(int)
        lt = batch.log_time[rows]
        slot = {int(x): i for i, x in enumerate(m)}
        for s in range(splits.split_offsets[p], splits.split_offsets[p + 1]):
            T = int(splits.train_masks[s])
            labels = {}
            for j in range(6):
                ys = [lt[v] - lt[slot[m[v] | 1 << j]] for v in range(V)
                      if not (m[v] >> j) & 1 and (m[v] | 1 << j) in slot
                      and (T >> v) & 1 and (T >> slot[m[v] | 1 << j]) & 1]
                labels[j] = ys
            for t in range(V):
                if (T >> t) & 1:
                    continue
                for j in range(6):
                    ys = labels[j]
                    if (m[t] >> j) & 1 or not ys or len(ys) > oracle.IBK_NEIGHBORS:
                        continue
                    assert abs(r.pred_all[row, j] - np.sum(ys) / len(ys)) <= 1e-13
                    checked += 1
                row += 1
    assert checked > 100


def test_ibk_cv_batch_matches_a_brute_force_pass():
    # leave-one-version-out on all 64 masks: 31 training pairs per fit, so the k-nearest
    # selection decides every prediction; the brute force reuses only the oracle's Z
    batch = synth.make_batch(2, versions=64, feat=24, dtype=np.float64, seed=9)
    splits = synth.make_splits(batch, "lovo")
    r = oracle.cv_batch(batch, splits, model="ibk")
    row = 0
    for p in range(batch.n_programs):
        V = batch.versions(p)
        rows = batch.program_rows(p)
        m = batch.masks[rows].astype(int)
        lt = batch.log_time[rows]
        o = int(batch.x_offsets[p])
        F = int(batch.feat_width[p])
        Z = r.Z[o:o + V * F].reshape(V, F)
        slot = {int(x): i for i, x in enumerate(m)}
        for s in range(splits.split_offsets[p], splits.split_offsets[p + 1]):
            T = int(splits.train_masks[s])
            for t in range(V):
                if (T >> t) & 1:
                    continue
                for j in range(6):
                    if (m[t] >> j) & 1:
                        assert np.isnan(r.pred_all[row, j])
                        continue
                    vs = [v for v in range(V) if not (m[v] >> j) & 1 and (m[v] | 1 << j) in slot
                          and (T >> v) & 1 and (T >> slot[m[v] | 1 << j]) & 1]
                    ys = np.array([lt[v] - lt[slot[m[v] | 1 << j]] for v in vs])
                    want = _brute(Z[vs], ys, Z[t], oracle.IBK_NEIGHBORS)
                    assert abs(r.pred_all[row, j] - want) <= 1e-13
                row += 1
    assert r.counter("fit_ok") == splits.n_splits * 6


def test_ibk_is_invariant_to_feature_order():
    rng = np.random.default_rng(11)
    Z = rng.normal(size=(30, 12))
    y = rng.normal(size=30)
    zt = rng.normal(size=12)
    perm = rng.permutation(12)
    a = oracle.ibk_predict(Z, y, zt, 10)
    b = oracle.ibk_predict(Z[:, perm], y, zt[perm], 10)
    assert abs(a - b) <= 1e-13


@pytest.mark.parametrize("n", [65, 96, 128, 257])
@pytest.mark.parametrize("k", [10, 64])
def test_ibk_many_training_pairs_match_brute_force(n, k):
    # the transfer protocol pools up to 32 pairs per run (Sec. 5, Table 2): 96 for three
    # runs, 128 for four; the neighbour list must not depend on n being small
    rng = np.random.default_rng(n * 7 + k)
    F = 9
    Z = rng.normal(size=(n, F))
    Z[n - 1] = Z[0]                                 # exact ties across the whole range
    Z[n // 2] = Z[3]
    y = rng.normal(size=n)
    for trial in range(6):
        zt = Z[int(rng.integers(0, n))] if trial % 2 else rng.normal(size=F)
        assert abs(oracle.ibk_predict(Z, y, zt, k) - _brute(Z, y, zt, k)) <= 1e-12


def test_ibk_rejects_out_of_range_k():
    Z = np.zeros((3, 2))
    with pytest.raises(ValueError):
        oracle.ibk_predict(Z, np.zeros(3), np.zeros(2), 65)
    with pytest.raises(ValueError):
        oracle.ibk_predict(Z, np.zeros(3), np.zeros(2), 0)
