"""The plain predictor as the surrogate's fallback (rs_surrogate_fallback): rows that the
surrogate flags out of distribution take the plain pass's ranking of their version bit for
bit, every other row keeps the surrogate's, and only the programs with a flagged row are
refitted.  Out-of-distribution rows are made by scaling all counters of a few versions of
some programs (their standardized features become extreme)."""
import numpy as np
import pytest
import torch

from paper_1910_07776_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_1910_07776_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    yield rs, ctx
    ctx.close()


def _outlier_batch(P, seed):
    b = synth.make_batch(P, versions=64, feat=256, dtype=np.float32, seed=seed)
    out, progs = synth.with_anomalous_versions(b, 1 / 3, per_program=3, seed=seed)
    return out, set(int(p) for p in progs)


@pytest.mark.parametrize("k", [3, 6])
def test_flagged_rows_take_the_plain_ranking(env, k):
    rs, ctx = env
    batch, shifted = _outlier_batch(9, seed=5)
    splits = synth.make_complementary_halves(batch, seed=5)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    n = batch.n_rows
    Z = ctx.standardize(db)
    Zm = Z.view(n, 256)
    sur = rs.Surrogate(ctx, 64, infer_chunk=64)
    sur.load(synth.init_mlp_params(5))
    Y = torch.zeros(n, 6, dtype=torch.float64, device="cuda")
    sur.train(Zm, Y, steps=0)                  # feature statistics and BF16 weights only
    code = torch.empty(n, dtype=torch.int32, device="cuda")
    rp = torch.empty(n * k, dtype=torch.float64, device="cuda")
    _, score, fb = sur.infer(Zm, ood_threshold=3.0, want_ood=True, masks=db.masks, k=k, rec_code=code,
                             rec_pred=rp, want_pred=False)
    torch.cuda.synchronize()
    code_s, rp_s, flag = code.cpu().numpy().copy(), rp.cpu().numpy().reshape(n, k).copy(), fb.cpu().numpy()
    assert 0 < flag.sum() < n // 4
    progs = {p for p in range(batch.n_programs) if flag[batch.program_rows(p)].any()}
    assert progs & shifted
    refit = ctx.surrogate_fallback(db, ds, fb, code, rp, k=k)
    torch.cuda.synchronize()
    ctx.check_device_status()
    assert refit == (len(progs), 64 * len(progs))
    code_f, rp_f = code.cpu().numpy(), rp.cpu().numpy().reshape(n, k)
    # the plain pass over the whole batch, and the row of each version in it
    R = ds.n_test_rows
    out = rs.alloc_outputs(R, ds.n_splits, k)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ctx.cv_step(db, ds, ws, out.rec_offsets, out.rec_code, k=k, rec_pred=out.rec_pred)
    torch.cuda.synchronize()
    pc = out.rec_code.cpu().numpy()
    pp = out.rec_pred.cpu().numpy().reshape(R, k)
    ro = out.rec_offsets.cpu().numpy()
    for p in range(batch.n_programs):
        for v in range(64):
            i = int(batch.row_offsets[p]) + v
            if flag[i]:
                for s in range(int(splits.split_offsets[p]), int(splits.split_offsets[p + 1])):
                    T = int(splits.train_masks[s])
                    if not (T >> v) & 1:
                        r = int(ro[s]) + bin(~T & ((1 << 64) - 1) & ((1 << v) - 1)).count("1")
                        assert code_f[i] == pc[r]
                        np.testing.assert_array_equal(rp_f[i], pp[r])
                        break
            else:
                assert code_f[i] == code_s[i]
                np.testing.assert_array_equal(rp_f[i], rp_s[i])


def test_no_flagged_row_changes_nothing(env):
    rs, ctx = env
    batch = synth.make_batch(3, versions=64, feat=256, dtype=np.float32, seed=6)
    splits = synth.make_complementary_halves(batch, seed=6)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    n = batch.n_rows
    fb = torch.zeros(n, dtype=torch.uint8, device="cuda")
    code = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
    rp = torch.full((n * 3,), 2.5, dtype=torch.float64, device="cuda")
    assert ctx.surrogate_fallback(db, ds, fb, code, rp) == (0, 0)
    torch.cuda.synchronize()
    assert (code.cpu().numpy() == 12345).all() and (rp.cpu().numpy() == 2.5).all()
