"""Pins of the oracle SPD-HSS construction (Sec. 3-5), ULV solve and PCG (Sec. 6)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import h2 as H
from oracle import kernels as K
from oracle import pcg as P
from oracle import spdhss as S
from oracle import tree as T
from oracle import ulv as U
from paper_2011_07632_gb300 import inputs


def _problem(n, dim, leaf, kind, ell, sigma, seed=0):
    X = inputs.uniform_cube(n, dim, seed)
    tr = T.build_tree(X, leaf)
    M = K.dense_matrix(kind, ell, sigma, X[tr.perm])
    return X, tr, M


@pytest.mark.parametrize("kind,ell,sigma,r", [(K.EXP, 1.0, 1e-2, 8), (K.GAUSS, 0.2, 1e-6, 5),
                                              (K.MATERN32, 0.1, 1e-4, 12), (K.IMQ, 0.5, 1e-5, 3)])
def test_hss_is_spd(kind, ell, sigma, r):
    """Sec. 3.2: the scaling-and-compression HSS approximation is SPD whatever r."""
    X, tr, M = _problem(512, 3, 16, kind, ell, sigma, seed=1)
    Om = inputs.sketch(512, r + 10, 7)
    hss = S.build_spdhss(tr, M, Om, r)
    Hd = S.assemble_dense(hss)
    assert np.allclose(Hd, Hd.T, atol=1e-12 * np.abs(Hd).max())
    assert np.linalg.eigvalsh(Hd).min() > 0.0


@pytest.mark.parametrize("n,dim,leaf", [(400, 3, 16), (300, 2, 8)])
def test_full_rank_hss_is_exact(n, dim, leaf):
    """With r >= every block dimension the projections are identities: HSS = M."""
    X, tr, M = _problem(n, dim, leaf, K.EXP, 0.5, 1e-2, seed=2)
    Om = inputs.sketch(n, n + 10, 8)
    hss = S.build_spdhss(tr, M, Om, n)
    assert np.abs(S.assemble_dense(hss) - M).max() <= 1e-13 * np.abs(M).max() * 10


def _explicit_recursion(tr, M, hss):
    """Literal scaling-and-compression (Eq. no_w, Eq. recursion) with the explicit large
    S_i (Eq. Si, Eq. Si0) and V_i (Eq. Vi) of every level; returns A^(L-1)."""
    Sbig, Vbig = {}, {}
    A_prev = M.copy()
    for k in range(1, tr.L):
        nodes = list(tr.nodes_at_level(k))
        for i in nodes:
            b, e = tr.begin[i], tr.end[i]
            if k == 1:
                Sbig[i], Vbig[i] = hss.S[i], hss.Vbar[i]
            else:
                kids = [int(c) for c in tr.children(i)]
                Sd = sla.block_diag(*[Sbig[c] for c in kids])
                Vd = sla.block_diag(*[Vbig[c] for c in kids])
                F = hss.Fhalf[i]
                Sbar = np.eye(e - b) + Vd @ (F - np.eye(F.shape[0])) @ Vd.T
                Sbig[i] = Sd @ Sbar
                Vbig[i] = Vd @ hss.Vbar[i]
            # Eq. Aii0 / Eq. Si: S_i S_i^T reproduces the diagonal block
            assert np.abs(Sbig[i] @ Sbig[i].T - A_prev[b:e, b:e]).max() < 1e-11 * np.abs(M).max()
            # Eq. R: U_i = S_i V_i equals the nested form diag(U_children) R_i
            assert np.abs(Sbig[i] @ Vbig[i] - S.explicit_U(hss, i)).max() < 1e-10 * np.abs(M).max()
        A_k = A_prev.copy()
        for i in nodes:
            bi, ei = tr.begin[i], tr.end[i]
            Pi = Sbig[i] @ Vbig[i] @ Vbig[i].T
            for j in nodes:
                if i == j:
                    continue
                bj, ej = tr.begin[j], tr.end[j]
                C = np.linalg.solve(Sbig[i], A_prev[bi:ei, bj:ej])
                C = np.linalg.solve(Sbig[j], C.T).T
                Pj = Sbig[j] @ Vbig[j] @ Vbig[j].T
                A_k[bi:ei, bj:ej] = Pi @ C @ Pj.T
        assert np.linalg.eigvalsh(A_k).min() > 0.0       # Sec. 3.2, every level
        A_prev = A_k
    return A_prev


@pytest.mark.parametrize("factor", ["eig", "chol"])
def test_generators_equal_literal_recursion(factor):
    X, tr, M = _problem(400, 2, 6, K.MATERN32, 0.3, 1e-3, seed=3)
    assert tr.L >= 5
    Om = inputs.sketch(400, 16, 9)
    hss = S.build_spdhss(tr, M, Om, 6, factor=factor)
    Ak = _explicit_recursion(tr, M, hss)
    Hd = S.assemble_dense(hss)
    assert np.abs(Ak - Hd).max() < 1e-10 * np.abs(M).max()


def test_eig_and_cholesky_factor_agree():
    """(I + bold B)^{1/2} and its Cholesky factor give the same HSS matrix."""
    X, tr, M = _problem(1024, 3, 32, K.EXP, 1.0, 1e-2, seed=4)
    Om = inputs.sketch(1024, 30, 10)
    H1 = S.assemble_dense(S.build_spdhss(tr, M, Om, 20, "eig"))
    H2_ = S.assemble_dense(S.build_spdhss(tr, M, Om, 20, "chol"))
    assert np.linalg.norm(H1 - H2_) / np.linalg.norm(H1) < 1e-12


def test_bij_recursion_matches_phi_form():
    """Eq. Mijk (from the children's B) equals Eq. bij_hss (Phi_i A_ij Phi_j^T)."""
    X, tr, M = _problem(600, 3, 16, K.GAUSS, 0.3, 1e-3, seed=5)
    Om = inputs.sketch(600, 18, 11)
    hss = S.build_spdhss(tr, M, Om, 8)
    for k in range(2, tr.L):
        nodes = list(tr.nodes_at_level(k))
        for i in nodes:
            for j in nodes:
                if i == j:
                    continue
                ki = [int(c) for c in tr.children(i)]
                kj = [int(c) for c in tr.children(j)]
                Bij = np.block([[hss.B[(a, b)] for b in kj] for a in ki])
                Fi = np.linalg.inv(S._sym_power(hss.Bbold[i], 0.5))
                Fj = np.linalg.inv(S._sym_power(hss.Bbold[j], 0.5))
                rec = hss.Vbar[i].T @ Fi @ Bij @ Fj @ hss.Vbar[j]
                assert np.abs(rec - hss.B[(i, j)]).max() < 1e-11 * max(1.0, np.abs(hss.B[(i, j)]).max())


def test_type3_shortcut_on_h2_input():
    """Eq. type3_Mij: for a Type-3 pair B_ij = (Phi_i U_i^H2) B_ij^H2 (Phi_j U_j^H2)^T, with
    Phi U^H2 from the nested recursion of Sec. 5.2.2."""
    X = inputs.uniform_cube(1024, 3, 6)
    tr = T.build_tree(X, 16)
    h = H.build_h2(tr, X, K.EXP, 1.0, 1e-2, 1e-5)
    M = H.dense(h)
    Om = inputs.sketch(1024, 20, 12)
    hss = S.build_spdhss(tr, M, Om, 10)
    PhiU = {}
    for k in range(1, tr.L):
        for i in tr.nodes_at_level(k):
            if k == 1:
                PhiU[i] = hss.Phi[i] @ h.U[i]
            else:
                kids = [int(c) for c in tr.children(i)]
                Dg = sla.block_diag(*[PhiU[c] for c in kids])
                Fm = np.linalg.inv(S._sym_power(hss.Bbold[i], 0.5))
                PhiU[i] = hss.Vbar[i].T @ Fm @ Dg @ h.U[i]
            if PhiU[i].size:
                assert np.abs(PhiU[i] - hss.Phi[i] @ H.explicit_basis(h, i)).max() < 1e-9
    checked = 0
    for (i, j), Bh in h.B.items():
        if tr.depth(i) == 0 or (i, j) not in hss.B:
            continue
        sc = PhiU[i] @ Bh @ PhiU[j].T
        assert np.abs(sc - hss.B[(i, j)]).max() < 1e-9 * max(1.0, np.abs(hss.B[(i, j)]).max())
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("n,leaf,r", [(1024, 32, 10), (40, 64, 5), (700, 16, 30)])
def test_ulv_solves_hss_exactly(n, leaf, r):
    X, tr, M = _problem(n, 3, leaf, K.EXP, 0.7, 1e-2, seed=7)
    Om = inputs.sketch(n, r + 10, 13)
    hss = S.build_spdhss(tr, M, Om, r)
    Hd = S.assemble_dense(hss)
    b = inputs.rhs(n, 3, 14)
    x = U.ULV(hss).solve(b)
    xd = U.dense_solve(Hd, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12
    assert np.linalg.norm(Hd @ x - b) / np.linalg.norm(b) < 1e-12


def test_pcg_pins():
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    lam = np.repeat([1.0, 3.0, 10.0, 40.0], 15)
    A = (Q * lam) @ Q.T
    b = rng.standard_normal((60, 2))
    # CG terminates in at most (number of distinct eigenvalues) steps in exact arithmetic
    x, it, rel = P.pcg(lambda v: A @ v, lambda v: v, b, 1e-10, 100)
    assert it.max() <= 5 and rel.max() <= 1e-10
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-8)
    # the exact inverse as preconditioner converges in one step
    Ainv = np.linalg.inv(A)
    x, it, rel = P.pcg(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-10, 100)
    assert it.max() == 1


def test_spdhss_preconditioner_reduces_iterations():
    X, tr, M = _problem(2048, 3, 32, K.EXP, 1.0, 1e-2, seed=8)
    Om = inputs.sketch(2048, 30, 15)
    hss = S.build_spdhss(tr, M, Om, 20)
    u = U.ULV(hss)
    b = inputs.rhs(2048, 1, 16)
    _, it_p, rel_p = P.pcg(lambda v: M @ v, u.solve, b, 1e-6, 3000)
    _, it_c, rel_c = P.pcg(lambda v: M @ v, lambda v: v, b, 1e-6, 3000)
    assert rel_p.max() <= 1e-6 and rel_c.max() <= 1e-6
    assert it_p.max() * 5 < it_c.max()


@pytest.mark.parametrize("tau", [1e-1, 1e-2, 1e-4])
def test_tolerance_truncation_leaf_ranks_match_lapack(tau):
    """Tolerance-driven bases: the leaf rank is the number of |R_kk| > tau |R_00| in
    LAPACK's column-pivoted QR (scipy) of the scaled sample S_i^{-1} Y_i^(1), capped at r."""
    n, r = 512, 40
    X, tr, M = _problem(n, 3, 32, K.GAUSS, 0.3, 1e-4, seed=3)
    Om = inputs.sketch(n, r + 10, 9)
    hss = S.build_spdhss(tr, M, Om, r, rtol=tau)
    Y = S.sample_products(tr, M, Om)
    for i in tr.nodes_at_level(1):
        b, e = tr.begin[i], tr.end[i]
        lam = sla.solve_triangular(np.linalg.cholesky(M[b:e, b:e]), Y[1][b:e], lower=True)
        R = sla.qr(lam, mode="r", pivoting=True)[0]
        d = np.abs(np.diag(R))
        want = min(r, int(np.sum(d > tau * d[0])))
        assert hss.rank[i] == want


def test_tolerance_truncation_monotone_and_spd():
    """Larger tau: ranks never grow, the approximation error grows, and the HSS stays SPD
    (Sec. 3.2 holds for any truncation)."""
    n, r = 512, 40
    X, tr, M = _problem(n, 3, 32, K.EXP, 0.5, 1e-3, seed=4)
    Om = inputs.sketch(n, r + 10, 10)
    prev_rank, prev_err = None, None
    for tau in (1e-14, 1e-6, 1e-2, 1e-1):
        hss = S.build_spdhss(tr, M, Om, r, rtol=tau)
        Hd = S.assemble_dense(hss)
        assert np.linalg.eigvalsh(Hd).min() > 0.0
        ranks = np.array([hss.rank[i] for i in sorted(hss.rank)])
        err = np.linalg.norm(Hd - M) / np.linalg.norm(M)
        if prev_rank is not None:
            assert np.all(ranks <= prev_rank)
            assert err >= prev_err * (1 - 1e-12)
        prev_rank, prev_err = ranks, err
    assert prev_rank.sum() < np.array([S.build_spdhss(tr, M, Om, r).rank[i] for i in sorted(hss.rank)]).sum()


def test_rank_zero_is_block_jacobi():
    """r = 0: every basis is empty and the SPD-HSS matrix is the block diagonal of the leaf
    blocks, the block-Jacobi preconditioner of the paper's comparisons, exactly."""
    X, tr, M = _problem(400, 3, 16, K.EXP, 0.5, 1e-2, seed=1)
    hss = S.build_spdhss(tr, M, inputs.sketch(400, 10, 3), 0)
    B = np.zeros_like(M)
    for i in tr.nodes_at_level(1):
        b, e = tr.begin[i], tr.end[i]
        B[b:e, b:e] = M[b:e, b:e]
    assert np.array_equal(S.assemble_dense(hss), B)


def test_adaptive_sketch_grows_until_ranks_fit():
    """Tolerance-driven construction with a growing sketch: the sketch doubles from 8
    columns (+ p) until every basis rank is below the attempt's cap; the result is the
    construction with that sketch, whose ranks are all below it."""
    n, p = 512, 10
    X, tr, M = _problem(n, 3, 64, K.MATERN32, 0.3, 1e-2, seed=6)
    Om = inputs.sketch(n, 200 + p, 11)
    hss = S.build_spdhss_adaptive(tr, M, Om, 200, p, 1e-3, r0=8)
    r = hss.sketch_rank
    assert r > 8 and r in (16, 32, 64, 128, 200)
    assert max(hss.rank.values()) < r
    ref = S.build_spdhss(tr, M, Om[:, :r + p], r, rtol=1e-3)
    assert ref.rank == hss.rank
    # the previous attempt was limited by its sketch
    rp = 128 if r == 200 else r // 2
    prev = S.build_spdhss(tr, M, Om[:, :rp + p], rp, rtol=1e-3)
    assert max(prev.rank.values()) == rp
