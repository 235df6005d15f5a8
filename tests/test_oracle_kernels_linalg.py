"""Pins of the oracle kernels (Sec. 6) and of its column-pivoted QR (Alg. 5.1 step 3)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import kernels as K
from oracle.linalg import pivoted_qr


def test_kernel_closed_forms():
    ell = 0.3
    r2 = np.array([0.0, ell * ell, ell * ell / 3.0])
    assert np.allclose(K.kernel_of_r2(K.EXP, r2[:2], ell), [1.0, np.exp(-1.0)], rtol=1e-15)
    assert np.allclose(K.kernel_of_r2(K.GAUSS, r2[:2], ell), [1.0, np.exp(-1.0)], rtol=1e-15)
    # Matern-3/2 at sqrt(3) r / ell = 1: (1 + 1) e^{-1}
    assert np.allclose(K.kernel_of_r2(K.MATERN32, r2[[0, 2]], ell), [1.0, 2.0 * np.exp(-1.0)], rtol=1e-15)
    assert np.allclose(K.kernel_of_r2(K.IMQ, r2[:2], ell), [1.0, 1.0 / np.sqrt(2.0)], rtol=1e-15)


@pytest.mark.parametrize("kind", [K.EXP, K.GAUSS, K.MATERN32, K.IMQ])
def test_shifted_kernel_matrix_is_spd(kind):
    X = np.random.default_rng(0).random((300, 3))
    A = K.dense_matrix(kind, 0.2, 1e-3, X)
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 1e-3 * (1 - 1e-6)


@pytest.mark.parametrize("m,n,seed", [(40, 25, 0), (25, 40, 1), (110, 60, 2), (64, 64, 3)])
def test_pivoted_qr_matches_lapack(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * np.logspace(0, -6, n)[None, rng.permutation(n)]
    k, piv, R, Q = pivoted_qr(A, min(m, n), 0.0)
    Rl, pl = sla.qr(A, mode="r", pivoting=True)
    assert k == min(m, n)
    assert (piv[:k] == pl[:k]).all()
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)[:k]), rtol=1e-10)
    assert np.abs(A[:, piv[:k]] - Q @ R[:, :k]).max() < 1e-13 * np.abs(A).max()
    assert np.abs(Q.T @ Q - np.eye(k)).max() < 1e-14
    d = np.abs(np.diag(R))
    assert np.all(d[1:] <= d[:-1] * (1 + 1e-12))


def test_pivoted_qr_rank_and_cap():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((50, 7)) @ rng.standard_normal((7, 30))
    k, piv, R, Q = pivoted_qr(A, 30, 1e-12)
    assert k == 7
    assert np.abs(A - Q @ (Q.T @ A)).max() < 1e-12 * np.abs(A).max()
    k2, _, _, Q2 = pivoted_qr(A, 4, 0.0)
    assert k2 == 4 and Q2.shape == (50, 4)


def test_pivoted_qr_tie_lowest_index_and_sign():
    A = np.zeros((4, 3))
    A[:, 0] = [1, 0, 0, 0]
    A[:, 1] = [0, 2, 0, 0]
    A[:, 2] = [0, 0, 2, 0]
    k, piv, R, Q = pivoted_qr(A, 3, 0.0)
    assert piv[:2].tolist() == [1, 2]
    # x_0 = 0 takes sign +: beta = -|x|
    assert R[0, 0] == -2.0
