"""Pins of the oracle's precision-mode PCG (oracle.pcg.pcg_mixed): it reduces to the textbook
PCG when its FP32 product is exact and no refresh runs, and on kernel systems whose FP32
product error is large relative to the residual it shows why the refresh restarts and the
switch to FP64 products are there.  The FP32 product is emulated as an FP32 kernel
evaluation: entries from FP32 coordinates in FP32 arithmetic, FP32 accumulation."""
import numpy as np
import pytest

from oracle import kernels as K
from oracle import pcg as P
from oracle import spdhss as S
from oracle import tree as T
from oracle import ulv as U
from paper_2011_07632_gb300 import inputs


def _gauss_f32(X, ell, sigma):
    """Gaussian kernel matrix evaluated in FP32 (FP32 coordinates, differences, squares,
    exponential), + sigma on the diagonal."""
    X32 = X.astype(np.float32)
    d2 = np.zeros((X.shape[0], X.shape[0]), np.float32)
    for k in range(X.shape[1]):
        diff = X32[:, None, k] - X32[None, :, k]
        d2 += diff * diff
    A = np.exp(-d2 / np.float32(ell * ell)).astype(np.float32)
    A[np.diag_indices_from(A)] += np.float32(sigma)
    return A


def _system(n, ell, sigma, rank=30, seed=7):
    X = inputs.uniform_cube(n, 2, seed)
    tr = T.build_tree(X, 64)
    Xs = X[tr.perm]
    A = K.dense_matrix(K.GAUSS, ell, sigma, Xs)
    A32 = _gauss_f32(Xs, ell, sigma)
    hss = S.build_spdhss(tr, A, inputs.sketch(n, rank + 10, 3)[tr.perm], rank)
    M = U.ULV(hss).solve
    b = inputs.rhs(n, 2, 4)[tr.perm]
    f64 = lambda v: A @ v
    f32 = lambda v: (A32 @ v.astype(np.float32)).astype(np.float64)
    return A, f64, f32, M, b


def _true_relres(A, x, b):
    return np.linalg.norm(b - A @ x, axis=0) / np.linalg.norm(b, axis=0)


def test_exact_product_without_refresh_is_the_textbook_pcg():
    """apply_A32 = apply_A and refresh = 0: the same iterates as oracle.pcg.pcg, bit for bit."""
    n = 600
    X = inputs.uniform_cube(n, 3, 1)
    tr = T.build_tree(X, 32)
    A = K.dense_matrix(K.EXP, 1.0, 1e-2, X[tr.perm])
    hss = S.build_spdhss(tr, A, inputs.sketch(n, 20, 2), 10)
    M = U.ULV(hss).solve
    b = inputs.rhs(n, 3, 5)
    f = lambda v: A @ v
    x0, it0, rr0 = P.pcg(f, M, b, 1e-8, 500)
    x1, it1, rr1, sw = P.pcg_mixed(f, f, M, b, 1e-8, 500, refresh=0)
    assert sw is None
    assert np.array_equal(it0, it1) and np.array_equal(rr0, rr1) and np.array_equal(x0, x1)


def test_exact_product_with_refresh_keeps_the_iteration_count():
    """An exact product and refreshes every 10 iterations: the refreshed residual equals the
    recursive one up to rounding, so nothing restarts or switches, and the count stays that
    of pcg within the spread that rounding alone gives CG (3%, at least 2)."""
    n = 600
    X = inputs.uniform_cube(n, 2, 3)
    tr = T.build_tree(X, 32)
    A = K.dense_matrix(K.MATERN32, 0.2, 1e-3, X[tr.perm])
    hss = S.build_spdhss(tr, A, inputs.sketch(n, 20, 4), 10)
    M = U.ULV(hss).solve
    b = inputs.rhs(n, 2, 6)
    f = lambda v: A @ v
    _, it0, _ = P.pcg(f, M, b, 1e-8, 2000)
    x1, it1, rr1, sw = P.pcg_mixed(f, f, M, b, 1e-8, 2000, refresh=10)
    assert np.max(it0) > 20
    assert sw is None
    assert np.all(np.abs(it1 - it0) <= np.maximum(2, np.ceil(0.03 * it0)))
    assert np.all(_true_relres(A, x1, b) <= 1e-8)


def test_restarts_are_needed_when_the_fp32_recursion_drifts():
    """Gaussian l = 0.2 in 2D, sigma = 1e-3: x = A^-1 b is dominated by the eigenvectors of
    the smallest eigenvalues, so the FP32 product's error is large relative to the residual.
    Plain residual replacement (no restart) stalls far above the tolerance; with the
    restarts the solve reaches it within twice the FP64 iteration count."""
    A, f64, f32, M, b = _system(2000, 0.2, 1e-3)
    _, it64, rr64 = P.pcg(f64, M, b, 1e-6, 3000)
    assert np.all(rr64 <= 1e-6)
    x0, it0, rr0, _ = P.pcg_mixed(f64, f32, M, b, 1e-6, 600, restarts=False, switch=False)
    assert np.all(it0 == 600) and np.all(rr0 > 1e-4)
    x1, it1, rr1, sw = P.pcg_mixed(f64, f32, M, b, 1e-6, 3000)
    assert np.all(_true_relres(A, x1, b) <= 1e-6) and np.all(rr1 <= 1e-6)
    assert np.all(it1 <= 2 * it64)


def test_switch_to_fp64_products_when_a_block_makes_no_progress():
    """Gaussian l = 0.2 in 2D, sigma = 1e-4: the refinement contracts too slowly on FP32
    products; the switch to FP64 products (after the first block without progress) brings the
    count close to the FP64 one, where restarts alone take nearly three times as many
    iterations."""
    A, f64, f32, M, b = _system(2000, 0.2, 1e-4)
    _, it64, rr64 = P.pcg(f64, M, b, 1e-6, 3000)
    assert np.all(rr64 <= 1e-6)
    _, it0, rr0, sw0 = P.pcg_mixed(f64, f32, M, b, 1e-6, 3000, switch=False)
    x1, it1, rr1, sw = P.pcg_mixed(f64, f32, M, b, 1e-6, 3000)
    assert sw is not None and sw % 50 == 0
    assert np.all(_true_relres(A, x1, b) <= 1e-6)
    assert np.all(it1 <= 1.5 * it64)
    assert np.max(it0) > 2 * np.max(it1)
