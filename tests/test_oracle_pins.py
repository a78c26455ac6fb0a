"""Pins for the FP64 CPU reference, against facts that do not come from the reference itself:
closed forms, library routines that solve the same problem another way, exact rational
arithmetic, invariants and brute force on tiny inputs.  No GPU needed."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1910_07776_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- standardization (Sec. 2)
def test_standardize_worked_example_closed_form():
    # log values 0,1,2,3: mean 1.5, population variance 1.25 (a sample variance would be 5/3)
    X = np.exp(np.array([[0.0], [1.0], [2.0], [3.0]]))
    Z, mu, sg = oracle.standardize(X)
    s = math.sqrt(1.25)
    np.testing.assert_allclose(mu, [1.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(sg, [s], rtol=1e-15)
    np.testing.assert_allclose(Z[:, 0], [-1.5 / s, -0.5 / s, 0.5 / s, 1.5 / s], rtol=1e-14)


def test_standardize_cycle_normalisation_removes_runtime():
    # Sec. 2: counters are divided by the cycle count so features do not depend on run time
    rng = np.random.default_rng(1)
    x = np.exp(rng.normal(size=(12, 7)))
    c = np.exp(rng.normal(5, 2, size=12))
    Z1, mu1, _ = oracle.standardize(x * c[:, None], cycles=c)
    Z2, mu2, _ = oracle.standardize(x)
    np.testing.assert_allclose(Z1, Z2, atol=1e-12)
    np.testing.assert_allclose(mu1, mu2, atol=1e-12)
    # without the divisor the answer must change (cycles differ per row)
    Z3, _, _ = oracle.standardize(x * c[:, None])
    assert np.abs(Z3 - Z2).max() > 1e-3


def test_standardize_matches_scipy_zscore_and_moments():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(2)
    X = np.exp(rng.normal(0, 1.5, size=(40, 33)))
    Z, mu, sg = oracle.standardize(X)
    ref = scipy_stats.zscore(np.log(X), axis=0, ddof=0)
    np.testing.assert_allclose(Z, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Z.mean(0), 0, atol=1e-13)
    np.testing.assert_allclose(Z.var(0), 1, rtol=1e-12)
    # a column scale factor is a log shift: z unchanged
    Zs, _, _ = oracle.standardize(X * np.exp(rng.normal(size=33))[None, :])
    np.testing.assert_allclose(Zs, Z, atol=1e-11)


def test_standardize_degenerate_cases():
    X = np.ones((5, 3))
    X[:, 1] = [1, 2, 3, 4, 5]
    X[2, 2] = 0.0   # clamps at eps before the log
    Z, mu, sg = oracle.standardize(X)
    assert np.all(Z[:, 0] == 0.0) and sg[0] == 0.0 and mu[0] == 0.0
    assert np.isclose(mu[2], math.log(1e-30) / 5, rtol=1e-14)
    assert np.all(np.isfinite(Z))


# ---------------------------------------------------------------- pairs (Sec. 3.3)
def test_pairs_all_64_masks():
    masks = np.arange(64, dtype=np.uint8)
    for j in range(6):
        b, a = oracle.pairs(masks, j)
        assert len(b) == 32                      # 32 versions without j, each paired once
        assert np.all((masks[b] >> j) & 1 == 0)
        assert np.all(masks[a] == (masks[b] | (1 << j)))
        assert len(set(b) | set(a)) == 64        # pairs partition the versions


def test_pairs_random_subsets_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(50):
        V = int(rng.integers(1, 65))
        masks = np.sort(rng.choice(64, size=V, replace=False)).astype(np.uint8)
        present = set(int(m) for m in masks)
        for j in range(6):
            b, a = oracle.pairs(masks, j)
            expect = sorted(m for m in present if not (m >> j) & 1 and (m | (1 << j)) in present)
            assert sorted(int(masks[v]) for v in b) == expect


def test_leave_one_out_leaves_31_pairs_per_optimization():
    # Sec. 5: removing one version always leaves exactly 31 of the 32 pairs of each optimization
    masks = np.arange(64, dtype=np.uint8)
    for t in range(64):
        T = set(range(64)) - {t}
        for j in range(6):
            b, a = oracle.pairs(masks, j)
            assert sum(1 for v, w in zip(b, a) if v in T and w in T) == 31


# ---------------------------------------------------------------- Cholesky
def test_cholesky_against_numpy_and_non_pd():
    rng = np.random.default_rng(4)
    for n in (1, 2, 7, 31):
        A = rng.normal(size=(n, n + 3))
        A = A @ A.T + 1e-3 * np.eye(n)
        st, L = oracle.cholesky(A)
        assert st == 0
        np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-10, atol=1e-12)
    st, _ = oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert st == 1


# ---------------------------------------------------------------- ridge (Sec. 3.4 family)
def test_ridge_noiseless_recovery_closed_form():
    rng = np.random.default_rng(5)
    n, F = 40, 6
    Z = rng.normal(size=(n, F))
    beta = rng.normal(size=F)
    b = 0.7
    st, bh, b0 = oracle.ridge_fit(Z, b + Z @ beta, 0.0)
    assert st == oracle.FIT_OK
    np.testing.assert_allclose(bh, beta, rtol=1e-11, atol=1e-12)
    assert abs(b0 - b) < 1e-12


def test_ridge_matches_augmented_least_squares_and_sklearn():
    rng = np.random.default_rng(6)
    for n, F, lam in [(31, 96, 1e-3), (8, 256, 1e-3), (50, 10, 0.5), (3, 2, 2.0)]:
        Z = rng.normal(size=(n, F))
        y = rng.normal(size=n)
        st, beta, b = oracle.ridge_fit(Z, y, lam)
        assert st == oracle.FIT_OK
        # a different algorithm: SVD least squares of [Zc; sqrt(lam) I] beta = [yc; 0]
        zb, yb = Z.mean(0), y.mean()
        A = np.vstack([Z - zb, math.sqrt(lam) * np.eye(F)])
        rhs = np.concatenate([y - yb, np.zeros(F)])
        ref = np.linalg.lstsq(A, rhs, rcond=None)[0]
        scale = np.abs(ref).max()
        np.testing.assert_allclose(beta, ref, rtol=0, atol=1e-9 * max(scale, 1.0) * 10)
        assert abs(b - (yb - zb @ ref)) < 1e-8
        sk = pytest.importorskip("sklearn.linear_model")
        m = sk.Ridge(alpha=lam, fit_intercept=True, solver="svd").fit(Z, y)
        np.testing.assert_allclose(beta, m.coef_, rtol=0, atol=1e-8 * max(scale, 1.0))


def test_ridge_stationarity_and_convexity():
    rng = np.random.default_rng(7)
    n, F, lam = 12, 20, 1e-2
    Z, y = rng.normal(size=(n, F)), rng.normal(size=n)
    st, beta, b = oracle.ridge_fit(Z, y, lam)
    res = y - b - Z @ beta
    assert abs(res.sum()) < 1e-10                              # d/db = 0
    np.testing.assert_allclose(Z.T @ res, lam * beta, atol=1e-10)   # d/dbeta = 0

    def obj(bb, be):
        r = y - bb - Z @ be
        return r @ r + lam * be @ be
    f0 = obj(b, beta)
    for _ in range(20):
        assert obj(b + 1e-3 * rng.normal(), beta + 1e-3 * rng.normal(size=F)) >= f0


def test_ridge_exact_rational_tiny():
    # exact arithmetic on small integers: solve the 2x2 centred normal equations in Fractions
    Z = [[1, 2], [3, -1], [0, 4], [2, 2]]
    y = [1, 0, 3, -2]
    lam = Fraction(1, 1000)
    n = len(y)
    zb = [Fraction(sum(r[f] for r in Z), n) for f in range(2)]
    yb = Fraction(sum(y), n)
    Zc = [[Fraction(r[f]) - zb[f] for f in range(2)] for r in Z]
    yc = [Fraction(v) - yb for v in y]
    G = [[sum(Zc[i][f] * Zc[i][g] for i in range(n)) + (lam if f == g else 0) for g in range(2)]
         for f in range(2)]
    r = [sum(Zc[i][f] * yc[i] for i in range(n)) for f in range(2)]
    det = G[0][0] * G[1][1] - G[0][1] * G[1][0]
    bx = [(r[0] * G[1][1] - G[0][1] * r[1]) / det, (G[0][0] * r[1] - G[1][0] * r[0]) / det]
    b0 = yb - zb[0] * bx[0] - zb[1] * bx[1]
    st, beta, b = oracle.ridge_fit(np.array(Z, float), np.array(y, float), float(lam))
    assert st == 0
    np.testing.assert_allclose(beta, [float(v) for v in bx], rtol=1e-13)
    assert abs(b - float(b0)) < 1e-13


def test_ridge_limits_and_degenerate():
    rng = np.random.default_rng(8)
    Z, y = rng.normal(size=(9, 5)), rng.normal(size=9)
    st, beta, b = oracle.ridge_fit(Z, y, 1e14)          # lambda -> infinity: the train mean
    assert np.abs(beta).max() < 1e-12 and abs(b - y.mean()) < 1e-10
    st, beta, b = oracle.ridge_fit(np.zeros((0, 5)), np.zeros(0), 1e-3)
    assert st == oracle.FIT_EMPTY
    st, beta, b = oracle.ridge_fit(Z[:1], y[:1], 1e-3)   # one pair: constant model
    assert st == oracle.FIT_OK and np.all(beta == 0) and b == y[0]
    st, beta, b = oracle.ridge_fit(Z[:3], y[:3], 0.0)    # lambda 0 and rank < F: not PD
    assert st == oracle.FIT_NOTPD


def test_ridge_primal_equals_dual_form():
    # (Zc^T Zc + lam I)^-1 Zc^T = Zc^T (Zc Zc^T + lam I)^-1: predictions agree
    rng = np.random.default_rng(9)
    n, F, lam = 11, 64, 1e-3
    Z, y = rng.normal(size=(n, F)), rng.normal(size=n)
    zt = rng.normal(size=F)
    st, beta, b = oracle.ridge_fit(Z, y, lam)
    Zc = Z - Z.mean(0)
    alpha = np.linalg.solve(Zc @ Zc.T + lam * np.eye(n), y - y.mean())
    dual = y.mean() + (zt - Z.mean(0)) @ Zc.T @ alpha
    assert abs((b + zt @ beta) - dual) < 1e-9


# ---------------------------------------------------------------- ranking (Tier 3)
def test_rank_ties_threshold_and_validity():
    pred = np.array([0.1, 0.2, 0.2, 0.05, 0.3, 0.2])
    assert list(oracle.rank(pred, np.ones(6), 3, 0.0)) == [4, 1, 2]
    assert list(oracle.rank(pred, np.ones(6), 6, 0.1)) == [4, 1, 2, 5, 0]   # inclusive
    v = np.array([1, 0, 1, 1, 0, 1])
    assert list(oracle.rank(pred, v, 3, -1.0)) == [2, 5, 0]
    assert list(oracle.rank(pred, np.zeros(6), 3, -1.0)) == []


def test_rank_brute_force_over_orders():
    rng = np.random.default_rng(10)
    for _ in range(300):
        pred = np.round(rng.normal(size=6), 1)        # rounding makes ties common
        valid = rng.random(6) < 0.8
        k = int(rng.integers(1, 7))
        lt = float(np.round(rng.normal() * 0.5, 1))
        got = list(oracle.rank(pred, valid, k, lt))
        cands = [j for j in range(6) if valid[j] and pred[j] >= lt]
        # the answer is the lexicographically smallest list among the orders of the
        # candidates that are sorted by value, truncated to k
        best = None
        for perm in itertools.permutations(cands):
            if all(pred[perm[i]] >= pred[perm[i + 1]] for i in range(len(perm) - 1)):
                cand = list(perm[:k])
                if best is None or cand < best:
                    best = cand
        assert got == (best or [])


# ---------------------------------------------------------------- the whole pass (Sec. 5)
def _python_counters(batch, splits, res, k, log_tau):
    """Re-derive the accuracy counters from the reference's own predictions and lists."""
    cnt = np.zeros(16, dtype=np.int64)
    recs = oracle.decode_rec(res.rec_code)
    row = 0
    for p in range(batch.n_programs):
        rs = batch.program_rows(p)
        m = batch.masks[rs].astype(int)
        lt = batch.log_time[rs]
        slot = {int(mm): i for i, mm in enumerate(m)}
        V = len(m)
        for s in range(int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])):
            T = int(splits.train_masks[s])
            for t in range(V):
                if (T >> t) & 1:
                    continue
                pr = res.pred_all[row]
                act = {}
                for j in range(6):
                    if (m[t] >> j) & 1 or np.isnan(pr[j]):
                        continue
                    w = slot.get(m[t] | (1 << j))
                    if w is not None:
                        act[j] = lt[t] - lt[w]
                cnt[0] += 1
                cnt[1] += int(np.sum(~np.isnan(pr)))
                cnt[2] += len(act)
                cnt[3] += sum(1 for j, a in act.items() if (pr[j] > 0) == (a > 0))
                rl = recs[row]
                cnt[4] += len(rl)
                cnt[5] += sum(1 for j in rl if j in act)
                cnt[6] += sum(1 for j in rl if j in act and act[j] > 0)
                if act:
                    cnt[7] += 1
                    bp = max(act, key=lambda j: (pr[j], -j))
                    ba = max(act, key=lambda j: (act[j], -j))
                    cnt[8] += int(bp == ba)
                # the list itself: sorted, above threshold, at most k, candidates only
                vals = [pr[j] for j in rl]
                assert all(vals[i] >= vals[i + 1] for i in range(len(vals) - 1))
                assert all(v >= log_tau for v in vals) and len(rl) <= k
                assert all(not (m[t] >> j) & 1 for j in rl)
                row += 1
    return cnt


@pytest.mark.parametrize("kind", ["lovo", "half"])
def test_cv_batch_counters_and_lists(kind):
    batch = synth.make_batch(2, versions=(20, 64), feat=24, seed=11)
    splits = synth.make_splits(batch, kind=kind, n_splits=8, seed=11)
    res = oracle.cv_batch(batch, splits, lam=1e-3, k=3, tau=1.05)
    cnt = _python_counters(batch, splits, res, 3, math.log(1.05))
    np.testing.assert_array_equal(res.counters[:9].astype(np.int64), cnt[:9])
    # rec rows: one per held-out version of each split
    pc = [batch.versions(p) - bin(int(t) & ((1 << batch.versions(p)) - 1)).count("1")
          for p in range(batch.n_programs)
          for t in splits.train_masks[splits.split_offsets[p]:splits.split_offsets[p + 1]]]
    assert res.rec_offsets[-1] == sum(pc) == res.counter("n_rows")


def test_cv_batch_predictions_equal_single_fits():
    batch = synth.make_batch(1, versions=64, feat=16, seed=12, dtype=np.float32)
    splits = synth.make_splits(batch, kind="half", n_splits=3, seed=12)
    res = oracle.cv_batch(batch, splits)
    Z = res.Z.reshape(64, 16)
    m = batch.masks.astype(int)
    slot = {mm: i for i, mm in enumerate(m)}
    row = 0
    for s in range(3):
        T = int(splits.train_masks[s])
        fits = []
        for j in range(6):
            rows = [(v, slot[m[v] | (1 << j)]) for v in range(64)
                    if not (m[v] >> j) & 1 and (T >> v) & 1 and (T >> slot[m[v] | (1 << j)]) & 1]
            y = np.array([batch.log_time[v] - batch.log_time[w] for v, w in rows])
            fits.append(oracle.ridge_fit(Z[[v for v, _ in rows]], y, 1e-3))
        for t in range(64):
            if (T >> t) & 1:
                continue
            for j in range(6):
                if (m[t] >> j) & 1:
                    assert np.isnan(res.pred_all[row, j])
                else:
                    st, beta, b = fits[j]
                    assert abs(res.pred_all[row, j] - (b + Z[t] @ beta)) < 1e-12
            row += 1


def test_pure_main_effects_are_recovered_exactly():
    # log t(m) = -sum_{j in m} a_j: every pair's label is a_j, so every fit is the constant a_j
    # and every candidate's prediction is a_j.  Checks the label's sign (before - after), the
    # candidate set and the ranking on all 64 masks; sign and top-1 accuracy are 100 %.
    batch = synth.make_batch(1, versions=64, feat=12, seed=13)
    a = np.array([0.2, -0.1, 0.08, 0.3, 0.02, -0.4])
    bits = (batch.masks[:, None].astype(int) >> np.arange(6)) & 1
    batch.log_time = -(bits @ a)
    splits = synth.make_splits(batch, kind="lovo")
    res = oracle.cv_batch(batch, splits, lam=1e-3, k=3, tau=1.05)
    for row, t in enumerate(range(64)):
        for j in range(6):
            if bits[t, j]:
                assert np.isnan(res.pred_all[row, j])
            else:
                assert abs(res.pred_all[row, j] - a[j]) < 1e-12
    recs = oracle.decode_rec(res.rec_code)
    order = [3, 0, 2]    # a_j >= log 1.05 = 0.0488 in descending order
    for t in range(64):
        assert recs[t] == [j for j in order if not bits[t, j]]
    assert res.counter("sign_hits") == res.counter("n_scored") > 0
    assert res.counter("top1_hits") == res.counter("top1_rows")


def test_constant_times_give_no_recommendation():
    batch = synth.make_batch(1, versions=40, feat=8, seed=14)
    batch.log_time = np.zeros_like(batch.log_time)
    splits = synth.make_splits(batch, kind="half", n_splits=4)
    res = oracle.cv_batch(batch, splits)
    assert res.counter("n_rec") == 0
    ok = ~np.isnan(res.pred_all)
    assert np.all(res.pred_all[ok] == 0.0)
