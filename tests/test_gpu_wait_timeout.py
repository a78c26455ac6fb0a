"""Failure detection without a GPU fault: the bounded wait used by the rank pass's TMA ring and
by the tensor-core GEMM's pipeline gives up on an mbarrier that nothing ever arrives at (no
copy is in flight), reports RS_ETIMEOUT with its site through the device status word, and
leaves the context usable for the next launch."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_a_status():
    from paper_1910_07776_gb300 import build, rs
    build.build()
    lib = rs.load()
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    done = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.rs_check_wait_timeout(rs._ptr(status), rs._ptr(done), 2_000_000, stream)   # 2 ms
    assert st == rs.RS_OK
    torch.cuda.synchronize()
    assert int(done.item()) == 0                       # the wait gave up
    assert status.cpu().tolist() == [rs.RS_ETIMEOUT, 99]
    # the context still runs kernels afterwards
    d = torch.tensor([2.0, 4.0], dtype=torch.float64, device="cuda")
    out = rs.check_reciprocals(d).cpu().numpy()
    np.testing.assert_array_equal(out[:, 1], [0.5, 0.25])
    assert lib.rs_check_wait_timeout(None, None, 2_000_000, stream) == rs.RS_EINVAL
