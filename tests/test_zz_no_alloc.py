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


def _raw(native, torch, u, Bc, Xc, nrhs, n):
    return native.lib().ulv_solve_noalloc(u._h, ctypes.c_void_p(Bc.data_ptr()),
                                          ctypes.c_void_p(Xc.data_ptr()), nrhs, n,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_allocates_nothing_and_rejects_oversize():
    api = need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    n = 3000
    X = inputs.uniform_cube(n, 3, 5)
    h = api.H2(X, "exp", 1.0, 1e-2, 64, 1e-8)
    hs = api.HSS(h, 20, 10, seed=2)
    u = api.ULV(hs)          # the factorization loads the fixed arrays on this device
    B = inputs.rhs(n, 2, 1)
    Bc = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xc = torch.empty_like(Bc)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # the first call (a fresh process: the first on this device) and the ones after it
    for _ in range(3):
        assert _raw(native, torch, u, Bc, Xc, 2, n) == native.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # more columns than the fixed level buffers hold: a clear EINVAL, nothing done
    big = 2500
    Bb = torch.zeros((big, n), dtype=torch.float64, device="cuda")
    Xb = torch.zeros_like(Bb)
    assert _raw(native, torch, u, Bb, Xb, big, n) == native.EINVAL
    assert b"48 MiB" in native.lib().spdhss_last_error()


def test_noalloc_in_place():
    """B and X the same array: the result equals ulv_solve's."""
    api = need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    n = 2500
    X = inputs.uniform_cube(n, 2, 6)
    h = api.H2(X, "gauss", 0.1, 1e-3, 64, 1e-8)
    hs = api.HSS(h, 25, 10, seed=3)
    u = api.ULV(hs)
    B = inputs.rhs(n, 4, 2)
    ref = u.solve(B).cpu().numpy()
    Bc = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    assert _raw(native, torch, u, Bc, Bc, 4, n) == native.OK
    torch.cuda.synchronize()
    assert rel(Bc.t().cpu().numpy(), ref) < 1e-12


def test_noalloc_rejects_too_many_descriptors():
    """Many small leaves: the launch descriptors (one work item per node and column) outgrow
    their 8 MiB array before the level buffers outgrow theirs."""
    api = need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    n = 2000
    X = inputs.uniform_cube(n, 3, 7)
    h = api.H2(X, "exp", 1.0, 1e-2, 4, 1e-8)
    hs = api.HSS(h, 2, 4, seed=5)
    u = api.ULV(hs)
    msg = None
    for nrhs in (32, 64, 128, 256, 512, 1024):
        Bc = torch.zeros((nrhs, n), dtype=torch.float64, device="cuda")
        st = _raw(native, torch, u, Bc, Bc, nrhs, n)
        if st != native.OK:
            assert st == native.EINVAL
            msg = native.lib().spdhss_last_error()
            break
    assert msg is not None and b"8 MiB" in msg, msg
