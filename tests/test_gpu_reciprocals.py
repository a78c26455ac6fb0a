"""The solvers' FP64 reciprocal (an FP32 seed and a truncated series in three FMAs) and
reciprocal square root (an FP32 seed and two Newton steps), which take the pivots of every
LDL^T and Cholesky factorisation of the ridge fits (Sec. 3.4), against CUDA's correctly
rounded division and square root and against exact decimal arithmetic, over a log-uniform
sweep of 2^-100 .. 2^100 plus the edges of that range and values outside it."""
from decimal import Decimal, getcontext

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _ulp_diff(a, b):
    """Distance in units in the last place between positive doubles."""
    return np.abs(a.view(np.int64) - b.view(np.int64))


def _inputs():
    rng = np.random.default_rng(5)
    e = rng.uniform(-100, 100, size=200_000)
    d = np.ldexp(rng.uniform(1.0, 2.0, size=e.size), np.floor(e).astype(int))
    edges = np.array([2.0 ** -100, np.nextafter(2.0 ** -100, 1), 2.0 ** 100, np.nextafter(2.0 ** 100, 0),
                      1.0, np.nextafter(1.0, 2), np.nextafter(2.0, 1), 3.0, 1e-3, 1e-300, 1e300, 5e-324,
                      np.finfo(np.float64).max, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52])
    # mantissas near the FP32 seed's truncation boundaries
    m = 1.0 + np.arange(1, 4097) * 2.0 ** -12 - 2.0 ** -40
    return np.concatenate([d, edges, m, m * 2.0 ** 37])


def test_reciprocal_and_rsqrt_within_one_ulp_of_cuda_and_exact():
    from paper_1910_07776_gb300 import build, rs
    build.build()
    d = _inputs()
    out = rs.check_reciprocals(torch.from_numpy(d).cuda()).cpu().numpy()
    rcp, div, rsq, ref_rsq = out[:, 0], out[:, 1], out[:, 2], out[:, 3]
    # CUDA's 1.0 / d is correctly rounded: the host's IEEE division gives the same bits
    with np.errstate(over="ignore", divide="ignore"):
        np.testing.assert_array_equal(div, 1.0 / d)
    assert _ulp_diff(rcp, div).max() <= 1
    # 1.0 / sqrt(d) rounds twice, so it may itself be an ulp off the true value
    assert _ulp_diff(rsq, ref_rsq).max() <= 2
    # against exact decimal arithmetic on a sample: both within one ulp of the true value
    getcontext().prec = 50
    for x, r, q in zip(d[::97], rcp[::97], rsq[::97]):
        t_r = float(Decimal(1) / Decimal(float(x)))
        t_q = float(Decimal(1) / Decimal(float(x)).sqrt())
        assert _ulp_diff(np.array([r]), np.array([t_r]))[0] <= 1
        assert _ulp_diff(np.array([q]), np.array([t_q]))[0] <= 1
