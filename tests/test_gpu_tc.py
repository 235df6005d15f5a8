"""Tensor-core FP32 GEMM (tcgen05.mma kind::tf32) against an FP64 product of the same FP32
operands: 3xTF32 to FP32 accuracy, plain TF32 to TF32 accuracy, over ragged sizes that
span several 128 x 64 / 128 x 128 tiles and K chunks, every transpose combination and
alpha / beta."""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

# (M, N, K, tA, tB): one tile, ragged tails in every dimension, several tiles and chunks,
# K = 0 (beta C only), a single row / column
CASES = [(128, 64, 32, 0, 0), (100, 60, 77, 0, 0), (300, 130, 257, 1, 0),
         (257, 200, 65, 0, 1), (64, 256, 512, 1, 1), (1, 1, 1, 0, 0), (129, 65, 0, 0, 0),
         (513, 33, 1000, 0, 0)]
# bounds relative to |A| |B| (row/column norms): FP32 rounding over K terms for 3xTF32 and
# the CUDA cores, TF32's 2^-11 for plain TF32
TOL = {0: 2e-6, 1: 3e-3, 2: 2e-6}


def _run(torch, native, M, N, K, tA, tB, mode, alpha, beta, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((K, M) if tA else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if tB else (K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    dA = torch.from_numpy(np.asfortranarray(A).T.copy()).cuda()   # column-major storage
    dB = torch.from_numpy(np.asfortranarray(B).T.copy()).cuda()
    dC = torch.from_numpy(np.asfortranarray(C0).T.copy()).cuda()
    lda = A.shape[0]
    ldb = B.shape[0]
    st = native.lib().spdhss_gemm_f32(
        M, N, K, ctypes.c_void_p(dA.data_ptr()), max(lda, 1), tA, ctypes.c_void_p(dB.data_ptr()),
        max(ldb, 1), tB, ctypes.c_void_p(dC.data_ptr()), M, ctypes.c_float(alpha),
        ctypes.c_float(beta), mode, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == native.OK, native.lib().spdhss_last_error()
    got = dC.cpu().numpy().T
    opA = (A.T if tA else A).astype(np.float64)
    opB = (B.T if tB else B).astype(np.float64)
    ref = alpha * (opA @ opB) + beta * C0.astype(np.float64)
    scale = alpha * np.outer(np.linalg.norm(opA, axis=1), np.linalg.norm(opB, axis=0)) + \
        abs(beta) * np.abs(C0) + 1e-30
    return float(np.max(np.abs(got - ref) / scale))


@pytest.mark.parametrize("M,N,K,tA,tB", CASES)
@pytest.mark.parametrize("mode", [2, 1, 0])
def test_tensor_core_gemm(M, N, K, tA, tB, mode):
    need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    err = _run(torch, native, M, N, K, tA, tB, mode, 1.0, 0.0, M + 7 * N + K)
    assert err < TOL[mode], err
    err = _run(torch, native, M, N, K, tA, tB, mode, -0.5, 2.0, M + N + 3 * K)
    assert err < TOL[mode], err


def test_bounded_wait_expires_and_the_context_stays_usable():
    """Mode 3 issues no MMA, so the kernel's mbarrier waits cannot complete: each gives up
    after about a second, the kernel records the failure, frees its tensor memory and
    returns, and the call reports TIMEOUT.  The next product on the same context is right."""
    need_gpu()
    import torch
    from paper_2011_07632_gb300 import native
    A = torch.ones((64, 64), dtype=torch.float32, device="cuda")
    C = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    st = native.lib().spdhss_gemm_f32(64, 64, 64, ctypes.c_void_p(A.data_ptr()), 64, 0,
                                      ctypes.c_void_p(A.data_ptr()), 64, 0,
                                      ctypes.c_void_p(C.data_ptr()), 64, ctypes.c_float(1.0),
                                      ctypes.c_float(0.0), 3,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == native.TIMEOUT
    assert b"gave up" in native.lib().spdhss_last_error()
    err = _run(torch, native, 100, 60, 77, 0, 0, 2, 1.0, 0.0, 5)
    assert err < TOL[2]
