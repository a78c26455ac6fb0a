"""Pins of the oracle's Table 2 transfer (Sec. 5): a model trained on a group of runs predicts,
ranks and scores another run, input or program.  Each pin comes from outside the oracle's own
code: the whole chain redone with numpy (pooled z-scores, pairs by brute force over the masks,
ridge by SVD least squares, IBK by sorting), an invariance of ridge under duplicated data,
and closed-form counts."""
import math

import numpy as np
import pytest

import oracle
from paper_1910_07776_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _numpy_transfer(train, test, groups, lam, opt_mask, model, rank_all=False, eps=1e-30):
    """Predictions [R][6] (NaN where none) redone with numpy from the definitions."""
    Q = test.n_programs
    out = []
    for q in range(Q):
        runs = range(int(groups[q]), int(groups[q + 1]))
        logs, masks, lts = [], [], []
        for r in runs:
            rows = train.program_rows(r)
            x = train.program_X(r).astype(np.float64)
            if train.cycles is not None:
                x = x / train.cycles[rows][:, None]
            logs.append(np.log(np.maximum(x, eps)))
            masks.append(train.masks[rows].astype(int))
            lts.append(train.log_time[rows])
        L = np.vstack(logs)
        mu, sd = L.mean(0), L.std(0)
        ok = sd > 1e-12
        Z = np.where(ok, (L - mu) / np.where(ok, sd, 1.0), 0.0)
        rows = test.program_rows(q)
        xb = test.program_X(q).astype(np.float64)
        if test.cycles is not None:
            xb = xb / test.cycles[rows][:, None]
        ZB = np.where(ok, (np.log(np.maximum(xb, eps)) - mu) / np.where(ok, sd, 1.0), 0.0)
        mb = test.masks[rows].astype(int)
        starts = np.cumsum([0] + [len(m) for m in masks])
        pred = np.full((len(mb), 6), np.nan)
        for j in range(6):
            zs, ys = [], []
            for ri, (m, lt) in enumerate(zip(masks, lts)):     # pairs within each run
                slot = {int(v): i for i, v in enumerate(m)}
                for v in range(len(m)):
                    if (m[v] >> j) & 1 or (m[v] | (1 << j)) not in slot:
                        continue
                    w = slot[m[v] | (1 << j)]
                    zs.append(Z[starts[ri] + v])
                    ys.append(lt[v] - lt[w])
            if not zs:
                continue
            Zj, yj = np.array(zs), np.array(ys)
            for t in range(len(mb)):
                if not ((opt_mask >> j) & 1) or (not rank_all and (mb[t] >> j) & 1):
                    continue
                if model == "ridge":
                    zb, yb = Zj.mean(0), yj.mean()
                    F = Zj.shape[1]
                    A = np.vstack([Zj - zb, math.sqrt(lam) * np.eye(F)])
                    beta = np.linalg.lstsq(A, np.concatenate([yj - yb, np.zeros(F)]), rcond=None)[0]
                    pred[t, j] = yb - zb @ beta + ZB[t] @ beta
                else:
                    d = ((Zj - ZB[t]) ** 2).sum(1)
                    sel = np.sort(np.lexsort((np.arange(len(d)), d))[:10])
                    pred[t, j] = yj[sel].sum() / len(sel)
        out.append(pred)
    return np.vstack(out)


def _small_runs(seed, inputs=2, runs=3, feat=10):
    return synth.make_runs(codes=(("BH", inputs), ("NB", inputs)), runs=runs, feat=feat, seed=seed)


@pytest.mark.parametrize("experiment", [1, 3, 5])
@pytest.mark.parametrize("model", ["ridge", "ibk"])
def test_transfer_matches_numpy_restatement(experiment, model):
    runs = _small_runs(7 + experiment)
    pr = synth.table2_problems(runs, experiment)
    res = oracle.transfer(pr.train, pr.test, pr.groups, lam=1e-3, opt_mask=pr.opt_mask, model=model)
    ref = _numpy_transfer(pr.train, pr.test, pr.groups, 1e-3, pr.opt_mask, model)
    assert np.array_equal(np.isnan(res.pred_all), np.isnan(ref))
    m = ~np.isnan(ref)
    tol = 1e-8 if model == "ridge" else 1e-12
    np.testing.assert_allclose(res.pred_all[m], ref[m], rtol=0, atol=tol)


def test_transfer_ragged_runs_and_rank_all_match_numpy():
    b = synth.make_batch(9, versions=(6, 40), feat=7, seed=21)
    train = synth.take_programs(b, [0, 1, 2, 3, 4, 5])
    test = synth.take_programs(b, [6, 7, 8])
    groups = np.array([0, 1, 3, 6])
    for model in ("ridge", "ibk"):
        for flags, ra in ((0, False), (oracle.RANK_ALL, True)):
            res = oracle.transfer(train, test, groups, flags=flags, opt_mask=0b101101, model=model)
            ref = _numpy_transfer(train, test, groups, 1e-3, 0b101101, model, rank_all=ra)
            assert np.array_equal(np.isnan(res.pred_all), np.isnan(ref))
            m = ~np.isnan(ref)
            np.testing.assert_allclose(res.pred_all[m], ref[m], rtol=0, atol=1e-8)


def test_duplicated_run_equals_single_run_with_half_lambda():
    # ridge on every pair twice minimises 2 sum (y - b - z.beta)^2 + lam |beta|^2: the single
    # run's fit at lam / 2; pooled statistics over a run and its copy are the run's own
    runs = _small_runs(3, inputs=1, runs=2, feat=12)
    one = synth.take_programs(runs, [0])
    dup = synth.take_programs(runs, [0, 0])
    test = synth.take_programs(runs, [1])
    a = oracle.transfer(dup, test, np.array([0, 2]), lam=2e-2)
    b = oracle.transfer(one, test, np.array([0, 1]), lam=1e-2)
    m = ~np.isnan(b.pred_all)
    np.testing.assert_allclose(a.pred_all[m], b.pred_all[m], rtol=0, atol=1e-9)
    np.testing.assert_array_equal(a.rec_code, b.rec_code)


def test_counts_follow_from_the_masks():
    # all 64 masks in every run: each test program has 64 rows; optimization j is a candidate
    # of the 32 versions without it (all 64 with RANK_ALL) and known for exactly those 32
    runs = _small_runs(5, inputs=2, runs=2, feat=8)
    pr = synth.table2_problems(runs, 5)
    Q = pr.test.n_programs
    for flags, per in ((0, 32), (oracle.RANK_ALL, 64)):
        r = oracle.transfer(pr.train, pr.test, pr.groups, flags=flags, opt_mask=pr.opt_mask)
        assert r.counter("n_rows") == 64 * Q
        assert r.counter("n_pred") == 2 * per * Q
        assert r.counter("n_scored") == 2 * 32 * Q
        assert r.counters[9] == 6 * Q and r.counters[10:13].sum() == 0
        rec = oracle.decode_rec(r.rec_code)
        assert all(set(lst) <= {4, 5} for lst in rec)


def test_counters_rederived_from_predictions():
    runs = _small_runs(11, inputs=2, runs=3, feat=9)
    for e in (2, 4, 6):
        pr = synth.table2_problems(runs, e)
        r = oracle.transfer(pr.train, pr.test, pr.groups, opt_mask=pr.opt_mask, model="ibk")
        rec = oracle.decode_rec(r.rec_code)
        cnt = np.zeros(9, dtype=np.int64)
        row = 0
        for q in range(pr.test.n_programs):
            rows = pr.test.program_rows(q)
            m = pr.test.masks[rows].astype(int)
            lt = pr.test.log_time[rows]
            slot = {int(v): i for i, v in enumerate(m)}
            for t in range(len(m)):
                p = r.pred_all[row]
                act = {j: lt[t] - lt[slot[m[t] | (1 << j)]] for j in range(6)
                       if not np.isnan(p[j]) and not (m[t] >> j) & 1 and (m[t] | (1 << j)) in slot}
                cnt[0] += 1
                cnt[1] += int((~np.isnan(p)).sum())
                cnt[2] += len(act)
                cnt[3] += sum((p[j] > 0) == (a > 0) for j, a in act.items())
                cnt[4] += len(rec[row])
                cnt[5] += sum(j in act for j in rec[row])
                cnt[6] += sum(j in act and act[j] > 0 for j in rec[row])
                if act:
                    cnt[7] += 1
                    cnt[8] += int(max(act, key=lambda j: (p[j], -j)) == max(act, key=lambda j: (act[j], -j)))
                vals = [p[j] for j in rec[row]]
                assert all(vals[i] >= vals[i + 1] for i in range(len(vals) - 1))
                assert all(v >= math.log(1.05) for v in vals) and len(vals) <= 3
                row += 1
        np.testing.assert_array_equal(r.counters[:9].astype(np.int64), cnt)


def test_empty_and_single_pair_fits():
    # one version: no pair (EMPTY, no prediction); two versions one optimization apart: one
    # pair, whose label is every prediction (ridge: alpha = 0, b = y; IBK: the only neighbour)
    X = np.exp(np.random.default_rng(0).normal(size=(3, 4)))
    mk = lambda rows, masks, lt: synth.ProgramBatch(
        X=X[rows].reshape(-1), x_offsets=np.array([0]), row_offsets=np.array([0, len(rows)]),
        feat_width=np.array([4], dtype=np.int32), masks=np.array(masks, dtype=np.uint8),
        log_time=np.array(lt), cycles=None)
    test = mk([0, 1, 2], [0, 1, 2], [0.0, -0.2, 0.1])
    one = mk([0], [0], [0.0])
    pair = mk([0, 1], [0, 1], [0.3, 0.1])
    r = oracle.transfer(one, test)
    assert (r.fit_status == oracle.FIT_EMPTY).all() and np.isnan(r.pred_all).all()
    assert r.counters[10] == 6 and r.counter("n_pred") == 0
    for model in ("ridge", "ibk"):
        r = oracle.transfer(pair, test, model=model)
        assert r.fit_status[0, 0] == oracle.FIT_OK and (r.fit_status[0, 1:] == oracle.FIT_EMPTY).all()
        # candidates for optimization 0: test versions 0 (mask 0) and 2 (mask 2)
        assert r.pred_all[0, 0] == pytest.approx(0.2, abs=1e-15) and r.pred_all[2, 0] == r.pred_all[0, 0]
        assert np.isnan(r.pred_all[1, 0])


@pytest.mark.parametrize("model", ["ibk", "ridge"])
def test_transfer_three_and_four_run_groups_match_numpy(model):
    # groups of three and four runs of all 64 masks pool 96 and 128 training pairs per
    # optimization (Sec. 5: a model trained on every run of an input); the IBK neighbour
    # search then runs over more pairs than one program can hold
    runs = _small_runs(31, inputs=1, runs=4, feat=8)
    idx = {key: p for p, key in enumerate(runs.meta["index"])}
    bh = [idx[("BH", 0, r)] for r in range(4)]
    nb = [idx[("NB", 0, r)] for r in range(4)]
    train = synth.take_programs(runs, bh + bh[:3])
    test = synth.take_programs(runs, [nb[0], nb[1]])
    groups = np.array([0, 4, 7])
    res = oracle.transfer(train, test, groups, model=model)
    ref = _numpy_transfer(train, test, groups, 1e-3, 0x3F, model)
    assert np.array_equal(np.isnan(res.pred_all), np.isnan(ref))
    m = ~np.isnan(ref)
    tol = 1e-12 if model == "ibk" else 1e-8
    np.testing.assert_allclose(res.pred_all[m], ref[m], rtol=0, atol=tol)
