"""GPU parity: the sm_103a library (through its C ABI) against the FP64 CPU reference, on the
same seeded inputs.  Element-wise at small sizes that still span many chunks, program
changes and ragged tails; sampled at the full batched-CV size in the launch configuration
the benchmark times."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1910_07776_gb300 import synth
from parity import close, compare_counters, compare_rankings

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build
    build.build()
    from paper_1910_07776_gb300 import rs as _rs
    return _rs


@pytest.fixture(scope="module")
def ctx(rs):
    c = rs.Context(0)
    yield c
    c.close()


def _run_both(rs, ctx, batch, splits, lam=1e-3, k=3, tau=1.05, flags=0, form=0, exact_rows=True):
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch if exact_rows else None)
    g = rs.cv_run(ctx, db, ds, lam=lam, k=k, tau=tau, flags=flags, form=form, want_Z=True)
    r = oracle.cv_batch(batch, splits, lam=lam, k=k, tau=tau, flags=flags)
    return g, r


def _check_cv(g, r, k, tau):
    np.testing.assert_array_equal(g["rec_offsets"], r.rec_offsets)
    err = close(g["pred_all"], r.pred_all)
    ndiff, nnear = compare_rankings(g["rec_code"], r.rec_code, r.pred_all, math.log(tau))
    same = g["rec_code"] == r.rec_code
    close(g["rec_pred"][same], r.rec_pred[same])
    compare_counters(g["counters"], r.counters, slack=nnear)
    return err, ndiff


# ------------------------------------------------------------------------------ A1 + A3
@pytest.mark.parametrize("dtype,cycles", [(np.float64, False), (np.float32, True)])
def test_standardize_and_gram(rs, ctx, dtype, cycles):
    batch = synth.make_batch(5, versions=(1, 64), feat_choices=[24, 40, 96, 130], dtype=dtype,
                             seed=21, with_cycles=cycles)
    splits = synth.make_splits(batch, "half", 2, seed=21)
    g, r = _run_both(rs, ctx, batch, splits)
    close(g["Z"], r.Z, rel=1e-12, abs_=1e-12)
    close(g["mu"], r.mu, rel=1e-13, abs_=1e-13)
    close(g["sigma"], r.sigma, rel=1e-12, abs_=1e-14)
    K = g["K"].cpu().numpy().reshape(-1, 64, 64)
    for p in range(batch.n_programs):
        V, F = batch.versions(p), int(batch.feat_width[p])
        o = int(batch.x_offsets[p])
        Zp = r.Z[o:o + V * F].reshape(V, F)
        ref = Zp @ Zp.T
        close(K[p, :V, :V], ref, rel=1e-12, abs_=1e-12 * F)
        np.testing.assert_array_equal(K[p, :V, :V], K[p, :V, :V].T)


@pytest.mark.parametrize("dtype,cycles", [(np.float64, False), (np.float32, True), (np.float64, True)])
def test_standardize_logarithm_accuracy(rs, ctx, dtype, cycles):
    """The standardization's own table-driven logarithm against the FP64 library log.  With one
    version per program the per-feature mean is the log itself, so mu = log(max(x / c, 1e-30))
    element by element.  The device forms q = x * (1 / c); the same two IEEE operations on the
    host give the same q.  Bound: 4 ulp of max(1, |log q|)."""
    rng = np.random.default_rng(23)
    P, F = 24, 512
    if dtype == np.float32:
        x = (10.0 ** rng.uniform(-37, 38, size=(P, F))).astype(np.float32)
        x.flat[:8] = [0.0, 1.0, 2.0, 0.5, 1e-40, 3e38, np.float32(1) + np.float32(2 ** -23), 7.0]
    else:
        x = 10.0 ** rng.uniform(-300, 300, size=(P, F))
        x.flat[:8] = [0.0, 1.0, 2.0, 0.5, 1e-310, 1e300, 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53]
    x[1] = 1.0 + rng.uniform(-1e-3, 1e-3, size=F)         # q near 1: small logs
    c = 10.0 ** rng.uniform(0, 9, size=P) if cycles else None
    batch = synth.ProgramBatch(
        X=x.reshape(-1), x_offsets=np.arange(P, dtype=np.int64) * F,
        row_offsets=np.arange(P + 1, dtype=np.int64), feat_width=np.full(P, F, dtype=np.int32),
        masks=np.zeros(P, dtype=np.uint8), log_time=np.zeros(P), cycles=c)
    db = rs.DeviceBatch.from_host(batch)
    mu = torch.empty(P * F, dtype=torch.float64, device="cuda")
    sg = torch.empty(P * F, dtype=torch.float64, device="cuda")
    ctx.standardize(db, mu=mu, sigma=sg)
    torch.cuda.synchronize()
    got = mu.cpu().numpy().reshape(P, F)
    q = x.astype(np.float64)
    if cycles:
        q = q * (1.0 / c)[:, None]
    ref = np.log(np.maximum(q, 1e-30))
    bound = 4 * 2.0 ** -53 * np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)
    assert np.all(sg.cpu().numpy() == 0)


# ------------------------------------------------------------------------------ A2..A6
@pytest.mark.parametrize("form", [0, 1])
def test_tiny_config_lovo_full(rs, ctx, form):
    # 2 programs x 64 versions (all masks) x 96 FP64 features, leave-one-version-out:
    # 128 fits of 6 ridge regressions, lambda 1e-3, top-3, threshold 1.05, seed 0
    batch = synth.make_batch(2, versions=64, feat=96, dtype=np.float64, seed=0)
    splits = synth.make_splits(batch, "lovo")
    g, r = _run_both(rs, ctx, batch, splits, form=form)
    err, ndiff = _check_cv(g, r, 3, 1.05)
    assert r.counter("fit_ok") == 128 * 6
    assert g["counters"][9] == 128 * 6
    assert ndiff == 0


@pytest.mark.parametrize("kind,k,flags,form,exact", [
    ("half", 3, 0, 0, True), ("frac", 6, 0, 0, False), ("frac", 2, 1, 0, True),
    ("half", 3, 0, 1, True), ("frac", 1, 1, 1, False)])
def test_ragged_batches(rs, ctx, kind, k, flags, form, exact):
    batch = synth.make_batch(9, versions=(1, 64), feat_choices=[8, 33, 64], dtype=np.float32,
                             seed=31 + k)
    splits = synth.make_splits(batch, kind, 37, seed=5 + k)
    g, r = _run_both(rs, ctx, batch, splits, k=k, flags=flags, form=form, exact_rows=exact)
    _check_cv(g, r, k, 1.05)


def test_wrong_size_hints_are_caught(rs, ctx):
    # hints smaller than the data: the kernels' own checks skip the excess and flag RS_EDATA
    batch = synth.make_batch(3, versions=64, feat=16, seed=71)
    splits = synth.make_splits(batch, "half", 9, seed=71)
    db = rs.DeviceBatch.from_host(batch)
    for bad in ("rows", "train"):
        ds = rs.DeviceSplits.from_host(splits, batch=batch)
        if bad == "rows":
            ds.n_test_rows = ds.n_test_rows // 2
        else:
            ds.max_train = 8
        Z = ctx.standardize(db)
        zb = db.with_X(Z)
        K = ctx.gram(zb)
        ro = ctx.rec_offsets(zb, ds)
        R = int(ro[-1])
        out = rs.alloc_outputs(R, ds.n_splits, 3)
        ctx.predict_rank(zb, K, ds, ro, out.rec_code, rec_pred=out.rec_pred, counters=out.counters)
        torch.cuda.synchronize()
        with pytest.raises(rs.RsError) as e:
            ctx.check_device_status()
        assert e.value.status == rs.RS_EDATA


def test_degenerate_splits(rs, ctx):
    batch = synth.make_batch(3, versions=(30, 64), feat=16, seed=41)
    S = 5
    offs = np.arange(4, dtype=np.int64) * S
    tm = []
    for p in range(3):
        V = batch.versions(p)
        full = (1 << V) - 1 if V < 64 else (1 << 64) - 1
        tm += [0, full, full & ~1, 1, 0b11]     # nothing, everything, one out, one, two
    splits = synth.Splits(split_offsets=offs, train_masks=np.array(tm, dtype=np.uint64))
    g, r = _run_both(rs, ctx, batch, splits)
    _check_cv(g, r, 3, 1.05)


def test_fit_batched_coefficients_and_status(rs, ctx):
    batch = synth.make_batch(4, versions=(10, 64), feat=48, seed=51)
    splits = synth.make_splits(batch, "frac", 40, seed=51)
    r = oracle.cv_batch(batch, splits)
    db, ds = rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits)
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    K = ctx.gram(zb)
    S = ds.n_splits
    coef = torch.full((S * 6 * 33,), 7.0, dtype=torch.float64, device="cuda")
    st = torch.full((S * 6,), 9, dtype=torch.uint8, device="cuda")
    ctx.fit_batched(zb, K, ds, 1e-3, 0, coef, st)
    ro = ctx.rec_offsets(zb, ds)
    R = int(ro[-1])
    out_a = rs.alloc_outputs(R, S, 3)
    out_b = rs.alloc_outputs(R, S, 3)
    ctx.predict_rank(zb, K, ds, ro, out_a.rec_code, rec_pred=out_a.rec_pred, pred_all=out_a.pred_all,
                     counters=out_a.counters)
    ctx.predict_rank(zb, K, ds, ro, out_b.rec_code, coef=coef, rec_pred=out_b.rec_pred,
                     pred_all=out_b.pred_all, counters=out_b.counters)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(st.cpu().numpy().reshape(S, 6), r.fit_status)
    # predicting from stored coefficients is the same arithmetic as the fused path
    np.testing.assert_array_equal(out_a.pred_all.cpu().numpy(), out_b.pred_all.cpu().numpy())
    np.testing.assert_array_equal(out_a.rec_code.cpu().numpy(), out_b.rec_code.cpu().numpy())
    cf = coef.cpu().numpy().reshape(S, 6, 33)
    ok = r.fit_status == 0
    assert np.all(np.isnan(cf[~ok][:, 0])) and np.all(cf[~ok][:, 1:] == 0)
    assert np.all(np.isfinite(cf[ok][:, 0]))
    # the dual coefficients of a fit sum to zero (stationarity in the intercept)
    sums = cf[ok][:, 1:].sum(axis=1)
    assert np.abs(sums).max() < 1e-6 * max(1.0, np.abs(cf[ok][:, 1:]).max())


def test_full_batched_cv_size_sampled(rs, ctx):
    # 64 programs x U{16..64} versions x 256 FP32 features, 4096 random half splits each,
    # through rs_cv_step (the single-call path the benchmark times); sampled splits are
    # recomputed by the reference and compared row by row.
    batch = synth.make_batch(64, versions=(16, 64), feat=256, dtype=np.float32, seed=0)
    splits = synth.make_half_splits_fast(batch, 4096, seed=0)
    db, ds = rs.DeviceBatch.from_host(batch), rs.DeviceSplits.from_host(splits, batch=batch)
    ro = ctx.rec_offsets(db, ds)
    R = int(ro[-1])
    out = rs.alloc_outputs(R, ds.n_splits, 3)
    ws = torch.empty(ctx.cv_workspace_bytes(db, ds), dtype=torch.uint8, device="cuda")
    ctx.cv_step(db, ds, ws, out.rec_offsets, out.rec_code, rec_pred=out.rec_pred,
                pred_all=out.pred_all, counters=out.counters)
    torch.cuda.synchronize()
    ctx.check_device_status()
    gro = out.rec_offsets.cpu().numpy()
    ref_ro = oracle.rec_offsets(batch, splits)
    np.testing.assert_array_equal(gro, ref_ro)
    cnt = out.counters.cpu().numpy()
    assert cnt[0] == R and cnt[9] + cnt[10] + cnt[11] + cnt[12] == 6 * ds.n_splits
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(ds.n_splits, size=48, replace=False))
    prog = np.searchsorted(splits.split_offsets, pick, side="right") - 1
    sub_off = np.zeros(batch.n_programs + 1, dtype=np.int64)
    for p in prog:
        sub_off[p + 1:] += 1
    sub = synth.Splits(split_offsets=sub_off, train_masks=splits.train_masks[pick])
    r = oracle.cv_batch(batch, sub)
    rows = np.concatenate([np.arange(gro[i], gro[i + 1]) for i in pick])
    pa = out.pred_all.cpu().numpy().reshape(R, 6)[rows]
    code = out.rec_code.cpu().numpy().view(np.uint32)[rows]
    close(pa, r.pred_all)
    compare_rankings(code, r.rec_code, r.pred_all, math.log(1.05))


def test_bad_program_size_is_reported(rs, ctx):
    # a program with 65 rows: every kernel's own check skips it and flags RS_EDATA
    batch = synth.make_batch(2, versions=64, feat=8, seed=61)
    db = rs.DeviceBatch.from_host(batch)
    db.row_offsets = torch.tensor([0, 65, 128], dtype=torch.int64, device="cuda")
    ctx.standardize(db)
    torch.cuda.synchronize()
    with pytest.raises(rs.RsError) as e:
        ctx.check_device_status()
    assert e.value.status == rs.RS_EDATA
    ctx.check_device_status()   # cleared


def test_argument_errors(rs, ctx):
    batch = synth.make_batch(1, versions=8, feat=8, seed=62)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(synth.make_splits(batch, "half", 2))
    Z = ctx.standardize(db)
    zb = db.with_X(Z)
    K = ctx.gram(zb)
    ro = ctx.rec_offsets(zb, ds)
    code = torch.empty(int(ro[-1]), dtype=torch.int32, device="cuda")
    for kw in (dict(k=0), dict(k=7), dict(tau=0.0), dict(lam=-1.0), dict(flags=64), dict(form=3)):
        with pytest.raises(rs.RsError) as e:
            ctx.predict_rank(zb, K, ds, ro, code, **kw)
        assert e.value.status == rs.RS_EINVAL


@pytest.mark.parametrize("flags,k", [(0, 3), (4, 3), (4, 6), (0, 1)])
def test_packed_predictions_equal_the_dense_lists(rs, ctx, flags, k):
    # RS_PACK_PRED: the reported predictions back to back in row order, no padding; the same
    # values as the dense rec_pred without its NaN slots, and as many as counter 4 says
    batch = synth.make_batch(12, versions=(1, 64), feat=48, dtype=np.float32, seed=321)
    splits = synth.make_splits(batch, "half", 200, seed=321)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    R = ds.n_test_rows
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    dense = rs.alloc_outputs(R, ds.n_splits, k, "cuda")
    ctx.cv_step(db, ds, ws, dense.rec_offsets, dense.rec_code, k=k, flags=flags, rec_pred=dense.rec_pred,
                counters=dense.counters)
    packed = rs.alloc_outputs(R, ds.n_splits, k, "cuda")
    packed.rec_pred.fill_(7.0)
    ctx.cv_step(db, ds, ws, packed.rec_offsets, packed.rec_code, k=k, flags=flags | rs.RS_PACK_PRED,
                rec_pred=packed.rec_pred, counters=packed.counters)
    torch.cuda.synchronize()
    ctx.check_device_status()
    assert torch.equal(dense.rec_code, packed.rec_code) and torch.equal(dense.counters, packed.counters)
    d = dense.rec_pred.cpu().numpy().reshape(R, k)
    want = d[~np.isnan(d)]                      # row order, then list order
    total = int(packed.counters[4].item())
    got = packed.rec_pred.cpu().numpy()
    assert total == want.size
    np.testing.assert_array_equal(got[:total], want)
    assert np.all(got[total:] == 7.0)           # nothing written past the packed lists


# ------------------------------------------------------------------------------ failed fits
@pytest.mark.parametrize("kind", ["half", "frac"])
def test_failed_fits_leave_their_optimization_out(rs, ctx, kind):
    """A version with an infinite log time gives its pairs infinite labels: every fit with one
    of them in training is non-finite (RS_FIT_NONFINITE), in each solver's size range (the
    frac splits make fits of 1 to 32 pairs).  The failed fit's optimization leaves its split's
    rows (the row records carry the failure); rankings and counters equal the oracle's."""
    batch = synth.make_batch(6, versions=(24, 64), feat=24, dtype=np.float64, seed=77)
    lt = batch.log_time.copy()
    for p in (1, 4):
        lt[int(batch.row_offsets[p]) + 3] = np.inf
    batch.log_time = lt
    splits = synth.make_splits(batch, kind, 40, seed=78)
    g, r = _run_both(rs, ctx, batch, splits)
    assert r.counter("fit_nonfinite") > 0
    _check_cv(g, r, 3, 1.05)


def test_rank_outputs_with_unaligned_rec_pred(rs, ctx):
    """rec_pred 16-byte aligned (a warp's values go through shared memory as 16-byte stores)
    and only 8-byte aligned (each lane stores its own values): the same outputs, and nothing
    written outside the view."""
    batch = synth.make_batch(7, versions=(20, 64), feat=32, dtype=np.float64, seed=91)
    splits = synth.make_splits(batch, "half", 50, seed=91)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    zb = db.with_X(ctx.standardize(db))
    K = ctx.gram(zb, rs.RS_GRAM_F64)
    ro = ctx.rec_offsets(zb, ds)
    R = int(ro[-1].item())
    got = []
    for off in (0, 1):
        buf = torch.full((R * 3 + 2,), 7.0, dtype=torch.float64, device="cuda")
        rp = buf[off:off + R * 3]
        code = torch.empty(R, dtype=torch.int32, device="cuda")
        ctx.predict_rank(zb, K, ds, ro, code, lam=1e-3, k=3, tau=1.05, rec_pred=rp)
        torch.cuda.synchronize()
        ctx.check_device_status()
        got.append((code.cpu().numpy(), rp.cpu().numpy(), buf.cpu().numpy()))
    np.testing.assert_array_equal(got[0][0], got[1][0])
    np.testing.assert_array_equal(got[0][1], got[1][1])
    assert got[0][2][-2] == 7.0 and got[0][2][-1] == 7.0
    assert got[1][2][0] == 7.0 and got[1][2][-1] == 7.0


# ------------------------------------------------------------------------------ slot order
def _shuffled(batch, seed):
    """The batch with each program's versions in a random slot order, so that its masks no
    longer ascend over the slots (the pair masks then take the bit-by-bit path)."""
    rng = np.random.default_rng(seed)
    X, masks, lt = batch.X.copy(), batch.masks.copy(), batch.log_time.copy()
    cyc = None if batch.cycles is None else batch.cycles.copy()
    for p in range(batch.n_programs):
        r0, V = int(batch.row_offsets[p]), batch.versions(p)
        F, xo = int(batch.feat_width[p]), int(batch.x_offsets[p])
        perm = rng.permutation(V)
        masks[r0:r0 + V] = batch.masks[r0:r0 + V][perm]
        lt[r0:r0 + V] = batch.log_time[r0:r0 + V][perm]
        if cyc is not None:
            cyc[r0:r0 + V] = batch.cycles[r0:r0 + V][perm]
        X[xo:xo + V * F] = batch.X[xo:xo + V * F].reshape(V, F)[perm].reshape(-1)
    return synth.ProgramBatch(X=X, x_offsets=batch.x_offsets.copy(), row_offsets=batch.row_offsets.copy(),
                              feat_width=batch.feat_width.copy(), masks=masks, log_time=lt, cycles=cyc)


@pytest.mark.parametrize("kind", ["half", "frac", "lovo"])
def test_versions_in_any_slot_order(rs, ctx, kind):
    # programs whose masks do not ascend over their slots, beside the sorted layout of every
    # other test: the same parity with the oracle
    batch = _shuffled(synth.make_batch(8, versions=(12, 64), feat=40, dtype=np.float32, seed=93), 93)
    unsorted = sum(not np.all(np.diff(batch.masks[batch.program_rows(p)].astype(int)) > 0)
                   for p in range(batch.n_programs))
    assert unsorted >= 7
    splits = synth.make_splits(batch, kind, 60, seed=94)
    g, r = _run_both(rs, ctx, batch, splits)
    _check_cv(g, r, 3, 1.05)
