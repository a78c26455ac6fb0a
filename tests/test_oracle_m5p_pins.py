"""Pins of the oracle's M5P model tree (Sec. 3.4 names M5P; the algorithm is the published M5'
description: SDR splits, models on the attributes tested below a node with greedy term
elimination, pruning by estimated error, smoothing with k = 15).  Each pin comes from outside
the oracle's C code: the same description restated here in plain Python (numpy solves the
linear models), closed forms (a linear target is one leaf with the exact model, a constant
target one leaf with that constant), and counts of the transfer protocol."""
import math

import numpy as np
import pytest

import oracle
from paper_1910_07776_gb300 import synth

K_SMOOTH, MIN_SPLIT, MIN_SIDE, SD_FRAC, RIDGE = 15.0, 4, 2, 0.05, 1e-8


def _sd(c, s1, s2):
    v = (s2 - s1 * s1 / c) / c
    return math.sqrt(v) if v > 0 else 0.0


def _lm(Z, y, idx, attrs):
    """Least squares with intercept on the attributes, estimated error (inf if m <= v)."""
    m = len(idx)
    Zs, ys = Z[np.ix_(idx, attrs)] if attrs else np.zeros((m, 0)), y[idx]
    zb, yb = Zs.mean(0), ys.mean()
    Zc = Zs - zb
    w = np.linalg.solve(Zc.T @ Zc + RIDGE * np.eye(len(attrs)), Zc.T @ (ys - yb)) if attrs else np.zeros(0)
    b = yb - float(w @ zb)
    v = len(attrs) + 1
    if m <= v:
        return math.inf, w, b
    e = float(np.mean(np.abs(ys - (b + Zs @ w))))
    return e * (m + v) / (m - v), w, b


def _py_m5p(Z, y):
    """Returns a predict(z) function of the tree grown, modelled, pruned as described."""
    n, F = Z.shape
    s1, s2 = sum(y), sum(v * v for v in y)
    sd_root = _sd(n, s1, s2)

    def grow(idx):
        m = len(idx)
        node = {"idx": idx, "attr": None}
        sd = _sd(m, sum(y[i] for i in idx), sum(y[i] * y[i] for i in idx))
        if m < MIN_SPLIT or sd <= SD_FRAC * sd_root:
            return node
        t1, t2 = sum(y[i] for i in idx), sum(y[i] * y[i] for i in idx)
        best, choice = 0.0, None
        for f in range(F):
            order = sorted(idx, key=lambda i: (Z[i, f], i))
            l1 = l2 = 0.0
            for c in range(1, m):
                yv = y[order[c - 1]]
                l1 += yv
                l2 += yv * yv
                va, vb = Z[order[c - 1], f], Z[order[c], f]
                if not va < vb or c < MIN_SIDE or m - c < MIN_SIDE:
                    continue
                sdr = sd - (c * _sd(c, l1, l2) + (m - c) * _sd(m - c, t1 - l1, t2 - l2)) / m
                if sdr > best:
                    best, choice = sdr, (f, (va + vb) * 0.5)
        if choice is None:
            return node
        f, thr = choice
        node.update(attr=f, thr=thr, left=grow([i for i in idx if Z[i, f] <= thr]),
                    right=grow([i for i in idx if Z[i, f] > thr]))
        return node

    def tested(node, acc):
        if node["attr"] is not None:
            acc.add(node["attr"])
            tested(node["left"], acc)
            tested(node["right"], acc)
        return acc

    def model(node):
        attrs = sorted(tested(node, set()))
        e, w, b = _lm(Z, y, node["idx"], attrs)
        while attrs:
            best, drop = math.inf, None
            for d in range(len(attrs)):
                et = _lm(Z, y, node["idx"], attrs[:d] + attrs[d + 1:])[0]
                if et < best:
                    best, drop = et, d
            if drop is None or not best <= e:
                break
            attrs = attrs[:drop] + attrs[drop + 1:]
            e, w, b = _lm(Z, y, node["idx"], attrs)
        node["model"] = (attrs, w, b)
        return e

    def prune(node):
        sub = 0.0
        if node["attr"] is not None:
            el, er = prune(node["left"]), prune(node["right"])
            ml, mr = len(node["left"]["idx"]), len(node["right"]["idx"])
            sub = (ml * el + mr * er) / len(node["idx"])
        e = model(node)
        if node["attr"] is not None and not e <= sub:
            return sub
        node["attr"] = None
        return e

    root = grow(list(range(n)))
    prune(root)

    def at(node, z):
        attrs, w, b = node["model"]
        return b + sum(w[k] * z[a] for k, a in enumerate(attrs))

    def predict(z):
        path = [root]
        while path[-1]["attr"] is not None:
            nd = path[-1]
            path.append(nd["left"] if z[nd["attr"]] <= nd["thr"] else nd["right"])
        p = at(path[-1], z)
        for child, parent in zip(reversed(path[1:]), reversed(path[:-1])):
            nc = len(child["idx"])
            p = (nc * p + K_SMOOTH * at(parent, z)) / (nc + K_SMOOTH)
        return p

    return predict


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_m5p_matches_python_restatement(seed):
    rng = np.random.default_rng(seed)
    n, F = [(12, 3), (30, 6), (64, 10), (96, 12)][seed]
    Z = rng.normal(size=(n, F))
    y = 0.4 * np.tanh(2 * Z[:, 0]) + 0.2 * Z[:, 1] * (Z[:, 2] > 0) + 0.05 * rng.normal(size=n)
    Zt = rng.normal(size=(20, F))
    got, leaves, nodes = oracle.m5p_fit_predict(Z, y, Zt)
    pred = _py_m5p(Z, y)
    ref = np.array([pred(z) for z in Zt])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)
    assert nodes == 2 * leaves - 1


def test_linear_target_is_one_leaf_with_the_exact_model():
    # y linear in one attribute: the root splits on it, so the root's model has that attribute
    # and fits exactly (estimated error 0, never above the subtree's): all is pruned to one
    # leaf whose model is the target (up to the 1e-8 guard on the normal equations)
    rng = np.random.default_rng(5)
    Z = rng.normal(size=(50, 4))
    y = 2.0 * Z[:, 2] + 1.0
    Zt = rng.normal(size=(10, 4))
    got, leaves, nodes = oracle.m5p_fit_predict(Z, y, Zt)
    assert leaves == 1 and nodes == 1
    np.testing.assert_allclose(got, 2.0 * Zt[:, 2] + 1.0, rtol=0, atol=1e-7)


def test_constant_target_and_tiny_sets():
    rng = np.random.default_rng(6)
    Z = rng.normal(size=(20, 3))
    got, leaves, _ = oracle.m5p_fit_predict(Z, np.full(20, -0.25), Z[:4])
    assert leaves == 1 and np.all(got == -0.25)
    for n in (1, 2, 3):                          # fewer than 4 instances: a leaf, the mean
        y = rng.normal(size=n)
        got, leaves, _ = oracle.m5p_fit_predict(Z[:n], y, Z[:2])
        assert leaves == 1
        np.testing.assert_allclose(got, np.mean(y), rtol=0, atol=1e-15)


def test_step_target_splits_at_the_gap_and_smooths():
    # y is +1 / -1 by the sign of attribute 1 with a wide gap: the root splits there (the
    # largest SDR), both children are constant (sd 0) leaves, and the subtree's error (0) beats
    # the root's linear model, so it stays; a prediction is the leaf's constant blended with
    # the root's model: (n_c * (+-1) + 15 q(z)) / (n_c + 15)
    rng = np.random.default_rng(7)
    Z = rng.normal(size=(40, 3))
    Z[:, 1] = np.where(np.arange(40) < 20, -1.0 - rng.random(40), 1.0 + rng.random(40))
    y = np.where(Z[:, 1] > 0, 1.0, -1.0)
    Zt = np.array([[0.1, -1.5, 0.2], [0.0, 1.7, -0.3]])
    got, leaves, nodes = oracle.m5p_fit_predict(Z, y, Zt)
    assert leaves == 2 and nodes == 3
    e, w, b = _lm(Z, y, list(range(40)), [1])
    q = b + w[0] * Zt[:, 1]
    np.testing.assert_allclose(got, (20 * np.array([-1.0, 1.0]) + 15 * q) / 35, rtol=0, atol=1e-9)


def test_transfer_with_m5p_counts_and_statuses():
    runs = synth.make_runs(codes=(("BH", 2), ("NB", 2)), runs=2, feat=8, seed=3)
    pr = synth.table2_problems(runs, 3)
    r = oracle.transfer(pr.train, pr.test, pr.groups, opt_mask=pr.opt_mask, model="m5p")
    Q = pr.test.n_programs
    assert (r.fit_status == oracle.FIT_OK).all() and r.counters[9] == 6 * Q
    assert r.counter("n_rows") == 64 * Q and r.counter("n_pred") == 6 * 32 * Q
    # the transfer's M5P predictions for problem 0 are those of the same group alone
    tr = synth.take_programs(pr.train, list(range(int(pr.groups[0]), int(pr.groups[1]))))
    ref = oracle.transfer(tr, synth.take_programs(pr.test, [0]), None, model="m5p")
    np.testing.assert_array_equal(ref.pred_all, r.pred_all[:64])
