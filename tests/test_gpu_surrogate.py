"""The surrogate's tensor-core kernels (forward, backward, AdamW) through the C ABI against the
FP64 reference, on the same BF16-rounded inputs and weights."""
import numpy as np
import pytest
import torch

from oracle import mlp

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def env():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build, rs
    build.build()
    ctx = rs.Context(0)
    yield rs, ctx
    ctx.close()


def data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 256))
    Y = 0.3 * rng.normal(size=(n, 6))
    return X, Y, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()


def ref_params(p):
    """The weights the GPU multiplies with: BF16 copies of W, FP32 biases."""
    return {k: (bf16(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64)) for k, v in p.items()}


def cos_rel(a, b):
    a, b = a.ravel(), b.ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)), float(np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300))


def test_gradients_and_loss_match_reference(env):
    rs, ctx = env
    X, Y, Xd, Yd = data(512, 1)
    p = mlp.init_params(1)
    sur = rs.Surrogate(ctx, 512)
    sur.load(p)
    lc = torch.zeros(1, dtype=torch.float32, device="cuda")
    sur.train(Xd, Yd, steps=1, lr=0.0, use_graph=False, loss_curve=lc)
    torch.cuda.synchronize()
    ctx.check_device_status()
    loss, g = mlp.loss_and_grads(ref_params(p), bf16(X), Y)
    assert abs(float(lc[0]) - loss) <= 2e-2 * loss
    for k in mlp.NAMES:
        gg = sur.view(k, "grad").cpu().numpy().astype(np.float64)
        if k in ("W3", "b3"):
            assert np.all(gg[6:] == 0)
            gg = gg[:6]
        c, r = cos_rel(gg, g[k])
        assert c >= 0.999 and r <= 3e-2, (k, c, r)
    # lr = 0: the master weights are unchanged
    np.testing.assert_array_equal(sur.view("W2").cpu().numpy(), np.asarray(p["W2"], np.float32))


def test_forward_matches_reference_on_ragged_chunks(env):
    rs, ctx = env
    X, Y, Xd, Yd = data(300, 2)
    p = mlp.init_params(2)
    sur = rs.Surrogate(ctx, 128)
    sur.load(p)
    sur.train(Xd[:128], Yd[:128], steps=0)          # prepares the BF16 copies and statistics only
    pred, _, _ = sur.infer(Xd, chunk_rows=128)
    torch.cuda.synchronize()
    out, _ = mlp.forward(ref_params(p), bf16(X))
    err = np.abs(pred.cpu().numpy() - out).max() / np.abs(out).max()
    assert err < 2e-2, err


def test_first_adamw_step_closed_form(env):
    rs, ctx = env
    X, Y, Xd, Yd = data(256, 3)
    p = mlp.init_params(3)
    sur = rs.Surrogate(ctx, 256)
    sur.load(p)
    lr, wd = 1e-3, 0.01
    sur.train(Xd, Yd, steps=1, lr=lr, weight_decay=wd, use_graph=False)
    torch.cuda.synchronize()
    for k in mlp.NAMES:
        g = sur.view(k, "grad").cpu().numpy().astype(np.float64)
        w1 = sur.view(k).cpu().numpy().astype(np.float64)
        w0 = np.zeros_like(w1)
        src = np.asarray(p[k], np.float32).astype(np.float64)
        w0[:src.shape[0]] = src
        # after one step mhat = g, vhat = g^2: w1 = w0 - lr (g / (|g| + eps) + wd w0)
        want = w0 - lr * (g / (np.abs(g) + 1e-8) + wd * w0)
        assert np.abs(w1 - want).max() <= 1e-6, k


def test_graph_replay_equals_eager_steps(env):
    rs, ctx = env
    X, Y, Xd, Yd = data(1024, 4)
    p = mlp.init_params(4)
    a, b = rs.Surrogate(ctx, 256), rs.Surrogate(ctx, 256)
    a.load(p)
    b.load(p)
    la = torch.zeros(6, device="cuda")
    lb = torch.zeros(6, device="cuda")
    a.train(Xd, Yd, steps=6, lr=1e-3, use_graph=True, loss_curve=la)
    b.train(Xd, Yd, steps=6, lr=1e-3, use_graph=False, loss_curve=lb)
    torch.cuda.synchronize()
    for k in mlp.NAMES:
        assert torch.equal(a.view(k), b.view(k)), k
    assert torch.allclose(la, lb, rtol=1e-5, atol=0)


def test_training_learns_and_ood_flags_shifted_rows(env):
    rs, ctx = env
    rng = np.random.default_rng(5)
    n = 8192
    X = rng.normal(size=(n, 256))
    W = rng.normal(size=(256, 6)) / 16.0
    Y = np.tanh(X @ W)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    sur = rs.Surrogate(ctx, 1024)
    sur.load(mlp.init_params(5))
    steps = 400
    lc = torch.zeros(steps, device="cuda")
    sur.train(Xd, Yd, steps=steps, lr=1e-3, use_graph=True, loss_curve=lc)
    torch.cuda.synchronize()
    curve = lc.cpu().numpy()
    assert curve[-20:].mean() < 0.2 * curve[:5].mean()
    Xs = np.concatenate([X[:512], 4.0 * X[:512]])
    pred, score, fb = sur.infer(torch.from_numpy(Xs).cuda(), ood_threshold=3.0, want_ood=True)
    torch.cuda.synchronize()
    fb = fb.cpu().numpy()
    assert fb[:512].mean() < 0.01 and fb[512:].mean() > 0.99
    s = score.cpu().numpy()
    ref = mlp.ood_score(Xs, X.mean(0), X.std(0))
    np.testing.assert_allclose(s, ref, rtol=1e-4)


def test_inference_ranking_matches_reference_ranking(env):
    rs, ctx = env
    import math
    import oracle
    X, Y, Xd, Yd = data(700, 6)
    p = mlp.init_params(6)
    p["b3"] = np.array([0.05, -0.02, 0.1, 0.049, 0.3, 0.0])       # spread the outputs around log 1.05
    sur = rs.Surrogate(ctx, 256)
    sur.load(p)
    sur.train(Xd[:256], Yd[:256], steps=0)
    masks = torch.from_numpy(np.random.default_rng(6).integers(0, 64, size=700).astype(np.uint8)).cuda()
    code = torch.empty(700, dtype=torch.int32, device="cuda")
    rp = torch.empty(700 * 3, dtype=torch.float64, device="cuda")
    pred, _, _ = sur.infer(Xd, masks=masks, k=3, tau=1.05, rec_code=code, rec_pred=rp, chunk_rows=256)
    torch.cuda.synchronize()
    P = pred.cpu().numpy().astype(np.float64)
    m = masks.cpu().numpy()
    lt = float(np.float32(math.log(1.05)))
    got = oracle.decode_rec(code.cpu().numpy().view(np.uint32))
    for r in range(700):
        valid = np.array([not (m[r] >> j) & 1 for j in range(6)], dtype=np.int32)
        want = list(oracle.rank(P[r], valid, 3, lt))
        assert got[r] == want, (r, got[r], want, P[r])
        np.testing.assert_array_equal(rp.cpu().numpy().reshape(700, 3)[r, :len(want)], P[r, want])


def test_checkpoint_resume_continues_the_run(env, tmp_path):
    # 3 steps, a checkpoint, a restore into a fresh state and 7 more steps give the weights and
    # Adam moments of 10 steps in one run (4 minibatches of 256 rows: the run wraps around)
    rs, ctx = env
    X, Y, Xd, Yd = data(1024, 6)
    p = mlp.init_params(6)
    a = rs.Surrogate(ctx, 256)
    a.load(p)
    a.train(Xd, Yd, steps=10, lr=1e-3)
    b = rs.Surrogate(ctx, 256)
    b.load(p)
    b.train(Xd, Yd, steps=3, lr=1e-3)
    path = str(tmp_path / "surrogate.ckpt")
    assert b.save(path) == 3
    c = rs.Surrogate(ctx, 256)
    c.restore(path)
    c.train(Xd, Yd, steps=7, lr=1e-3)
    torch.cuda.synchronize()
    for k in mlp.NAMES:
        assert torch.equal(a.view(k), c.view(k)), k
        assert torch.equal(a.view(k, "m"), c.view(k, "m")) and torch.equal(a.view(k, "v"), c.view(k, "v")), k
    # a damaged or truncated checkpoint is refused
    raw = bytearray(open(path, "rb").read())
    for bad in (bytes([raw[0] ^ 1]) + bytes(raw[1:]), bytes(raw[:1000])):
        f = tmp_path / "bad.ckpt"
        f.write_bytes(bad)
        with pytest.raises(rs.RsError) as e:
            c.restore(str(f))
        assert e.value.status == rs.RS_EINVAL
