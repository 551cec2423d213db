"""Pins for the oracle's determinant ratio (Sec. 1 Eq. 2; Sec. 3 Eqs. 11-13) and the
standard explicit-inverse / Sherman-Morrison algorithm (Sec. 1)."""
import itertools
import math

import numpy as np
import pytest


def _perm_sign(p):
    s, p = 1, list(p)
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            s = -s
    return s


def test_leibniz_closed_forms(orc):
    assert orc.leibniz_det(np.array([[2.0, 3.0], [5.0, 7.0]])) == 2 * 7 - 3 * 5
    T = np.triu(np.arange(1, 26, dtype=float).reshape(5, 5))
    assert orc.leibniz_det(T) == pytest.approx(np.prod(np.diag(T)), rel=1e-14)
    for p in [(1, 0, 2, 3), (3, 2, 1, 0), (1, 2, 3, 0), (0, 1, 2, 3)]:
        P = np.eye(4)[list(p)]
        assert orc.leibniz_det(P) == _perm_sign(p)
    # linear in one row, zero for two equal rows
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 6))
    A2 = A.copy(); A2[2] = A2[4]
    assert abs(orc.leibniz_det(A2)) < 1e-12
    A3 = A.copy(); A3[1] *= 3.0
    assert orc.leibniz_det(A3) == pytest.approx(3.0 * orc.leibniz_det(A), rel=1e-12)


def test_lu_det_matches_leibniz(orc):
    rng = np.random.default_rng(2)
    for n in (1, 2, 3, 5, 8):
        A = rng.standard_normal((n, n))
        LU, piv, sign = orc.lu(A)
        det = sign * np.prod(np.diag(LU))
        assert det == pytest.approx(orc.leibniz_det(A), rel=1e-11)


@pytest.mark.parametrize("n", [3, 6, 8])
def test_ratio_is_det_ratio_random(orc, n):
    """Matrix determinant lemma: det(A + e_i u^T) / det A = 1 + u^T A^{-1} e_i."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 2 * np.eye(n)
    for i in range(n):
        a_new = rng.standard_normal(n)
        A2 = A.copy(); A2[i] = a_new
        exact = orc.leibniz_det(A2) / orc.leibniz_det(A)
        r, rl = orc.ratio_dense(A, i, a_new)
        assert r == pytest.approx(exact, rel=1e-11, abs=1e-12)
        assert rl == pytest.approx(exact, rel=1e-11, abs=1e-12)


def test_ratio_on_tiny_slater_system(orc):
    """n = 8 simple-cubic system (K = 2) with r_c < L/2: ratio equals the Leibniz ratio."""
    s = orc.system(2, 0, 1.0, 0.7, 0.95)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 5, 0.15)
    A = orc.slater_dense(s, Z, R)
    assert (A != 0).sum() > 8          # some off-diagonal coupling
    d0 = orc.leibniz_det(A)
    for i in range(8):
        r_new = orc.propose(s, 5, 0, i, 0.3, R[i])
        a_new = orc.row_dense(s, Z, r_new)
        A2 = A.copy(); A2[i] = a_new
        exact = orc.leibniz_det(A2) / d0
        r, _ = orc.ratio_dense(A, i, a_new)
        assert r == pytest.approx(exact, rel=1e-11, abs=1e-13)


def test_null_move_ratio_is_exactly_one(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 1, 0.1)
    A = orc.slater_dense(s, Z, R)
    for i in (0, 17, 215):
        r, rl = orc.ratio_dense(A, i, A[i])
        assert r == 1.0
        assert rl == pytest.approx(1.0, abs=1e-12)
    # a proposal with sigma = 0 is a null move
    _, ratios, acc, _ = orc.chain(s, 1, 0.0, R, 1, max_steps=30, solver=orc.SOLVER_DENSE_LU)
    assert np.all(ratios == 1.0) and np.all(acc)


def test_reverse_move_gives_reciprocal(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 3, 0.1)
    A = orc.slater_dense(s, Z, R)
    for i in (4, 100, 200):
        r_new = orc.propose(s, 3, 0, i, 0.2, R[i])
        a_new = orc.row_dense(s, Z, r_new)
        fwd, _ = orc.ratio_dense(A, i, a_new)
        A2 = A.copy(); A2[i] = a_new
        back, _ = orc.ratio_dense(A2, i, A[i])
        assert fwd * back == pytest.approx(1.0, abs=1e-12)


def test_ratio_invariant_under_reordering(orc):
    """Simultaneous row and column permutations leave |det| ratios unchanged (Sec. 2.1)."""
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 4, 0.1)
    A = orc.slater_dense(s, Z, R)
    rng = np.random.default_rng(4)
    P = rng.permutation(A.shape[0])
    Q = rng.permutation(A.shape[0])
    Ap = A[P][:, Q]
    pos = np.argsort(P)
    for i in (0, 50, 150):
        a_new = orc.row_dense(s, Z, orc.propose(s, 4, 0, i, 0.2, R[i]))
        r0, _ = orc.ratio_dense(A, i, a_new)
        r1, _ = orc.ratio_dense(Ap, int(pos[i]), a_new[Q])
        assert r1 == pytest.approx(r0, rel=1e-12)


def test_sherman_morrison_tracks_fresh_inverse(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 6, 0.1)
    A = orc.slater_dense(s, Z, R)
    B = orc.inverse(A)
    assert np.abs(A @ B - np.eye(A.shape[0])).max() < 1e-12
    for step in range(60):
        i = step % A.shape[0]
        a_new = orc.row_dense(s, Z, orc.propose(s, 6, 0, i, 0.2, R[i]))
        u = a_new - A[i]
        r_sm = orc.sm_ratio(B, i, u)
        r_lu, _ = orc.ratio_dense(A, i, a_new)
        assert r_sm == pytest.approx(r_lu, rel=1e-11)
        if r_sm * r_sm > 0.3:
            orc.sm_update(B, i, u, r_sm)
            A[i] = a_new
    assert np.abs(B - orc.inverse(A)).max() < 1e-10


def test_gmres_reference_matches_dense_solve(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 8, 0.1)
    A = orc.slater_dense(s, Z, R)
    rp, ci, cv = orc.slater_csr(s, Z, R)
    LU, piv, _ = orc.lu(A)
    for i in (0, 99):
        e = np.zeros(A.shape[0]); e[i] = 1.0
        x, its = orc.gmres(rp, ci, cv, e, tol=1e-14)
        assert its > 0
        assert np.abs(x - orc.lu_solve(LU, piv, e)).max() < 1e-12


def test_coincident_electrons_make_the_determinant_vanish(orc):
    """Two electrons at one position give two equal rows of A (Eq. 1), so the determinant is zero:
    the oracle's LU reports the matrix singular, and moving electron i onto electron j gives the
    ratio 1 + (a_j - a_i)^T A^{-1} e_i = 1 + delta_ij - 1 = 0 (Eq. 13) from every ratio solver."""
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 9, 0.1)
    A = orc.slater_dense(s, Z, R)
    B = orc.inverse(A)
    rp, ci, cv = orc.slater_csr(s, Z, R)
    for i, j in ((3, 4), (100, 7), (215, 214)):
        a_new = orc.row_dense(s, Z, R[j])
        assert np.array_equal(a_new, A[j])
        r, rl = orc.ratio_dense(A, i, a_new)
        assert abs(r) < 1e-12
        assert rl == 0.0                      # A' itself is exactly singular
        assert abs(orc.sm_ratio(B, i, a_new - A[i])) < 1e-12
        e = np.zeros(A.shape[0]); e[i] = 1.0
        z, _ = orc.gmres(rp, ci, cv, e, tol=1e-14)
        assert abs(1.0 + (a_new - A[i]) @ z) < 1e-11
        R2 = R.copy(); R2[i] = R[j]
        with pytest.raises(np.linalg.LinAlgError):
            orc.lu(orc.slater_dense(s, Z, R2))
    # exactly zero for a small system by the Leibniz sum as well
    s8 = orc.system(2, 0, 1.0, 0.7, 0.95)
    Z8 = orc.sites(s8)
    R8 = orc.initial_positions(s8, 5, 0.15)
    R8[6] = R8[1]
    assert abs(orc.leibniz_det(orc.slater_dense(s8, Z8, R8))) < 1e-15


@pytest.mark.parametrize("kappa,r_c", [(2.0, 1.5), (1.0, 2.0)])
def test_gmres_reference_at_n_1728(orc, kappa, r_c):
    """The restarted GMRES that the oracle uses above n = 1000 (Sec. 3.2; x0 = 0, so the
    relative residual is the absolute one) against dense LU at n = 12^3, for both orbital
    widths of the configured workloads; the residual is recomputed here with numpy."""
    s = orc.system(12, 0, 1.0, kappa, r_c)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 3, 0.1)
    A = orc.slater_dense(s, Z, R)
    rp, ci, cv = orc.slater_csr(s, Z, R)
    LU, piv, _ = orc.lu(A)
    for i in (0, 777, 1727):
        e = np.zeros(A.shape[0]); e[i] = 1.0
        x, its = orc.gmres(rp, ci, cv, e, tol=1e-14)
        assert its > 0
        assert np.linalg.norm(A @ x - e) <= 1e-13
        assert np.abs(x - orc.lu_solve(LU, piv, e)).max() <= 1e-12
