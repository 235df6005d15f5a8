"""The allocation-free ULV solve (ulv_solve_noalloc) gives the same result as ulv_solve.

ulv_solve_noalloc serves callers that cannot allocate device memory: it works in fixed
device arrays of the library instead of buffers it allocates.  This file is collected last
so that a run stopping at the first failure has already run every other test; it also
passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2011_07632_gb300 import inputs

from gpu_util import need_gpu, rel

pytestmark = pytest.mark.gpu


def _call_noalloc(native, torch, u, B, nrhs, n):
    Bc = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xc = torch.empty_like(Bc)
    st = native.lib().ulv_solve_noalloc(u._h, ctypes.c_void_p(Bc.data_ptr()),
                                        ctypes.c_void_p(Xc.data_ptr()), nrhs, n,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, Xc


@pytest.mark.parametrize("n,leaf,r", [(3000, 64, 30), (40, 64, 5)])
def test_noalloc_matches_ulv_solve_twice(n, leaf, r):
    api = need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    X = inputs.uniform_cube(n, 3, 3)
    h = api.H2(X, "matern32", 0.2, 1e-3, leaf, 1e-8)
    hs = api.HSS(h, r, 10, seed=4)
    u = api.ULV(hs)
    for call in range(2):
        B = inputs.rhs(n, 3, 10 + call)
        ref = u.solve(B).cpu().numpy()
        st, Xc = _call_noalloc(native, torch, u, B, 3, n)
        assert st == native.OK, native.lib().spdhss_last_error()
        torch.cuda.synchronize()
        got = Xc.t().cpu().numpy()
        assert rel(got, ref) < 1e-12


def test_noalloc_allocates_nothing_and_rejects_oversize():
    api = need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    n = 3000
    X = inputs.uniform_cube(n, 3, 5)
    h = api.H2(X, "exp", 1.0, 1e-2, 64, 1e-8)
    hs = api.HSS(h, 20, 10, seed=2)
    u = api.ULV(hs)
    B = inputs.rhs(n, 2, 1)
    st, _ = _call_noalloc(native, torch, u, B, 2, n)      # first call: per-device set-up
    assert st == native.OK
    torch.cuda.synchronize()
    Bc = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xc = torch.empty_like(Bc)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        s = native.lib().ulv_solve_noalloc(u._h, ctypes.c_void_p(Bc.data_ptr()),
                                           ctypes.c_void_p(Xc.data_ptr()), 2, n,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert s == native.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # more columns than the fixed level buffers hold: a clear EINVAL, nothing done
    big = 2500
    Bb = torch.zeros((big, n), dtype=torch.float64, device="cuda")
    Xb = torch.zeros_like(Bb)
    s = native.lib().ulv_solve_noalloc(u._h, ctypes.c_void_p(Bb.data_ptr()),
                                       ctypes.c_void_p(Xb.data_ptr()), big, n,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == native.EINVAL
    assert b"48 MiB" in native.lib().spdhss_last_error()
