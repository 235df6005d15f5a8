"""Pins of the oracle's deterministic Alg. 4.1 (bases from truncated SVDs of the scaled
block rows C_ii^c and E_ii^c, Eq. minimization), and what the sketch of Sec. 5.2.1 costs
against it.  The mode is not a GPU parity target."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import kernels as K
from oracle import pcg as P
from oracle import spdhss as S
from oracle import tree as T
from oracle import ulv as U
from paper_2011_07632_gb300 import inputs


def _setup(n, leaf, kind, ell, sigma, seed=0):
    X = inputs.uniform_cube(n, 3, seed)
    tr = T.build_tree(X, leaf)
    return tr, K.dense_matrix(kind, ell, sigma, X[tr.perm])


def _resid(C, V):
    return np.linalg.norm(C - V @ (V.T @ C))


@pytest.mark.parametrize("kind,ell,sigma", [(K.EXP, 1.0, 1e-6), (K.GAUSS, 0.3, 1e-5)])
def test_deterministic_hss_is_spd(kind, ell, sigma):
    tr, M = _setup(512, 32, kind, ell, sigma, seed=1)
    H = S.assemble_dense(S.build_spdhss_deterministic(tr, M, 6))
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() > 0.0


def test_deterministic_full_rank_is_exact():
    tr, M = _setup(600, 40, K.MATERN32, 0.3, 1e-3, seed=2)
    H = S.assemble_dense(S.build_spdhss_deterministic(tr, M, 600))
    assert np.abs(H - M).max() <= 1e-12 * np.abs(M).max()


def test_deterministic_bases_minimize_the_scaled_residual():
    """Eckart-Young: no orthonormal r-column basis leaves a smaller residual of C_ii^c
    (leaves) or E_ii^c (above) than the one chosen, in particular not the randomized
    basis of Alg. 5.3 (leaves, same C) nor the pivoted-QR basis of the target itself;
    and the chosen columns lie in col(target)."""
    r = 10
    tr, M = _setup(1024, 32, K.EXP, 1.0, 1e-2, seed=3)
    hd = S.build_spdhss_deterministic(tr, M, r, keep=True)
    hr = S.build_spdhss(tr, M, inputs.sketch(1024, r + 10, 2)[tr.perm], r)
    leaves = set(tr.nodes_at_level(1))
    for i, C in hd.target.items():
        V = hd.Vbar[i]
        best = _resid(C, V)
        slack = 1e-13 * np.linalg.norm(C)      # full-rank nodes: both residuals are rounding
        Q, _, _ = sla.qr(C, mode="economic", pivoting=True)
        assert best <= _resid(C, Q[:, :V.shape[1]]) + slack
        if i in leaves:
            assert best <= _resid(C, hr.Vbar[i]) + slack
        Z = np.linalg.lstsq(C, V, rcond=None)[0]
        assert np.linalg.norm(C @ Z - V) <= 1e-8
        assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)


def test_cost_of_the_sketch():
    """The sketch of Sec. 5.2.1 approximates col(S_i^{-1} A_ii^c) instead of
    col(C_ii^c): its leaf bases leave a larger scaled residual than the optimal ones (by
    a median factor of about 1.7 here) and its preconditioner needs more PCG iterations
    (25 against 18 for this matrix)."""
    r = 20
    tr, M = _setup(2048, 64, K.EXP, 1.0, 1e-2, seed=0)
    hd = S.build_spdhss_deterministic(tr, M, r, keep=True)
    hr = S.build_spdhss(tr, M, inputs.sketch(2048, r + 10, 2)[tr.perm], r)
    ratio = [_resid(hd.target[i], hr.Vbar[i]) / _resid(hd.target[i], hd.Vbar[i])
             for i in tr.nodes_at_level(1)]
    assert min(ratio) >= 1.0 - 1e-12
    assert 1.2 < np.median(ratio) < 3.0
    b = inputs.rhs_uniform(2048, 1, 1)[tr.perm]
    its = []
    for h in (hd, hr):
        u = U.ULV(h)
        _, it, rr = P.pcg(lambda v: M @ v, u.solve, b, 1e-6, 3000)
        assert rr[0] <= 1e-6
        its.append(int(it[0]))
    assert its[0] < its[1]
