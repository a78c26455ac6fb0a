"""rs_cv_step_static: the whole step with its scratch in the library's fixed device array,
for callers that cannot allocate device memory.  Called through the C ABI twice in a row on
the same inputs and compared with rs_cv_step (which takes a caller-allocated workspace)."""
import ctypes as C

import numpy as np
import pytest
import torch

from parity import close

pytestmark = pytest.mark.gpu


def _static_call(rs, lib, db, ds, outs, dev_status, k=3, tau=1.05, lam=1e-3):
    bc, sc = db.c(), ds.c()
    err = C.create_string_buffer(256)
    st = lib.rs_cv_step_static(
        C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(bc), C.byref(sc), lam, k, tau, 0,
        rs._ptr(outs.rec_offsets), rs._ptr(outs.rec_code), rs._ptr(outs.rec_pred),
        rs._ptr(outs.pred_all), rs._ptr(outs.counters), rs._ptr(dev_status), err, 256)
    return st, err.value.decode()


def test_static_scratch_step_matches_workspace_step_twice():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build, rs, synth
    build.build()
    lib = rs.load()
    batch = synth.make_batch(6, versions=(12, 64), feat_choices=[24, 96], dtype=np.float32, seed=90)
    splits = synth.make_splits(batch, "half", 50, seed=90)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    R = ds.n_test_rows
    ctx = rs.Context(0)
    ref = rs.alloc_outputs(R, ds.n_splits, 3)
    ws = ctx.workspace(ctx.cv_workspace_bytes(db, ds))
    ctx.cv_step(db, ds, ws, ref.rec_offsets, ref.rec_code, rec_pred=ref.rec_pred,
                pred_all=ref.pred_all, counters=ref.counters)
    torch.cuda.synchronize()
    ctx.check_device_status()
    want = {k: getattr(ref, k).cpu().numpy() for k in ("rec_offsets", "rec_code", "rec_pred", "pred_all", "counters")}
    dev_status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        outs = rs.alloc_outputs(R, ds.n_splits, 3)
        outs.rec_code.fill_(-1)
        outs.pred_all.fill_(7.0)
        st, msg = _static_call(rs, lib, db, ds, outs, dev_status)
        assert st == rs.RS_OK, msg
        torch.cuda.synchronize()
        assert int(dev_status.item()) == 0
        np.testing.assert_array_equal(outs.rec_offsets.cpu().numpy(), want["rec_offsets"])
        np.testing.assert_array_equal(outs.rec_code.cpu().numpy(), want["rec_code"])
        close(outs.pred_all.cpu().numpy(), want["pred_all"])
        close(outs.rec_pred.cpu().numpy(), want["rec_pred"])
        np.testing.assert_array_equal(outs.counters.cpu().numpy(), want["counters"])
    ctx.close()


def test_static_scratch_rejects_batches_beyond_its_size():
    from paper_1910_07776_gb300 import build, rs, synth
    build.build()
    lib = rs.load()
    batch = synth.make_batch(2, versions=64, feat=8, seed=91)
    splits = synth.make_splits(batch, "half", 4, seed=91)
    db = rs.DeviceBatch.from_host(batch)
    ds = rs.DeviceSplits.from_host(splits, batch=batch)
    db.x_elems = 64 << 20          # claims a Z larger than the whole static scratch
    outs = rs.alloc_outputs(ds.n_test_rows, ds.n_splits, 3)
    st, msg = _static_call(rs, lib, db, ds, outs, None)
    assert st == rs.RS_ENOMEM and "static scratch" in msg
