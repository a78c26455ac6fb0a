"""The tcgen05 BF16 GEMM core (TMA-fed, FP32 accumulation in tensor memory) through the C ABI,
against a plain FP32 matrix product of the same BF16 values."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1910_07776_gb300 import build, rs
    build.build()
    c = rs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 128, 512), (300, 200, 320), (1000, 512, 256),
                                   (4096, 256, 512), (77, 16, 512), (513, 6, 64), (64, 64, 1024)])
def test_gemm_bf16_matches_fp32_product(ctx, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    ldb = max(8, (K + 7) // 8 * 8)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = ctx.gemm_bf16(A, B)
    torch.cuda.synchronize()
    ctx.check_device_status()
    ref = A.float() @ B.float().T
    scale = (A.float().abs() @ B.float().abs().T)
    err = (D - ref).abs() / (scale + 1e-30)
    assert float(err.max()) < 2e-6, float(err.max())


def test_gemm_bf16_padded_leading_dimensions(ctx):
    M, N, K = 200, 48, 100
    Ab = torch.randn(M, 128, device="cuda").to(torch.bfloat16)
    Bb = torch.randn(N, 104, device="cuda").to(torch.bfloat16)
    A, B = Ab[:, :K], Bb[:, :K]
    D = torch.full((M, 64), 3.0, device="cuda")
    from paper_1910_07776_gb300 import rs
    ctx._check(ctx.L.rs_gemm_bf16(ctx.h, rs._ptr(Ab), 128, rs._ptr(Bb), 104, rs._ptr(D), 64, M, N, K))
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T
    assert torch.allclose(D[:, :N], ref, rtol=1e-5, atol=1e-4)
    assert torch.all(D[:, N:] == 3.0)          # columns beyond N untouched
