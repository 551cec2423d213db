"""GPU checks of the preconditioner pieces: ILUTP exactness without dropping, the
preconditioner apply against dense triangular solves, the paper's identity for the
updated preconditioner (Sec. 3.2), the greedy reordering against the oracle's
(Sec. 3.1), and one-iteration convergence with an exact factorisation."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmc():
    import torch

    assert torch.cuda.is_available()
    from paper_1008_5113_gb300.build import build_library

    build_library()
    O.build()
    from paper_1008_5113_gb300 import vmc as v

    return v


def _colour_order(K):
    """Orbital columns: sites sorted by (x mod 3, y mod 3, z mod 3), then index."""
    idx = np.arange(K ** 3)
    x, y, z = idx % K, (idx // K) % K, idx // (K * K)
    colour = (x % 3) + 3 * (y % 3) + 9 * (z % 3)
    return np.lexsort((idx, colour))


@pytest.mark.parametrize("prec", [0, 1])
def test_ilutp_without_dropping_is_exact_lu(vmc, prec):
    K = 3
    s = O.system(K, 0, 1.0, 2.0, 1.45)
    R = O.initial_positions(s, 4, 0.15)
    ctx = vmc.vmc_create([(K, 0, 1.0, 2.0, 1.45)], vmc.params(precision=prec, drop_tol=0.0, lfil_extra=27))
    try:
        vmc.vmc_set_positions(ctx, 0, R)
        A, por, ooc = vmc.vmc_get_matrix(ctx, 0)
        L, U, perm = vmc.vmc_get_factors(ctx, 0)
        assert np.allclose(np.tril(L, -1) + np.eye(27), L) and np.allclose(np.triu(U), U)
        # the mixed engine eliminates in FP32 (its factors are FP32), the FP64 engine in FP64
        assert np.abs(A[:, perm] - L @ U).max() < (1e-13 if prec == 0 else 1e-6)
        st0 = vmc.vmc_get_stats(ctx, 0)
        r_new = O.propose(s, 4, 0, 11, 0.2, R[11])
        vmc.vmc_ratio(ctx, 0, 11, r_new)
        st = vmc.vmc_get_stats(ctx, 0)
        assert st["first_pass_iterations"] - st0["first_pass_iterations"] == 1
        assert st["N_max_seen"] < (1e-12 if prec == 0 else 1e-5)
    finally:
        vmc.vmc_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_preconditioner_apply_matches_dense_solves(vmc, prec):
    K = 6
    s = O.system(K)
    R = O.initial_positions(s, 9, 0.1)
    ctx = vmc.vmc_create([(K, 0, 1.0, 2.0, 1.5)], vmc.params(precision=prec))
    try:
        vmc.vmc_set_positions(ctx, 0, R)
        L, U, perm = vmc.vmc_get_factors(ctx, 0)
        rng = np.random.default_rng(1)
        for _ in range(3):
            v = rng.standard_normal(216)
            z = vmc.vmc_apply_preconditioner(ctx, 0, v)
            y = np.linalg.solve(U, np.linalg.solve(L, v))
            ref = np.zeros(216)
            ref[perm] = y
            tol = 1e-12 if prec == 0 else 1e-5
            assert np.abs(z - ref).max() <= tol * np.abs(ref).max()
    finally:
        vmc.vmc_destroy(ctx)


def test_updated_preconditioner_keeps_AM_fixed(vmc):
    """A_{k+1} M_{k+1} = A_k M_k + r_k u_k^T M_k / (1 + u_k^T z_k) (Sec. 3.2): with an FP64
    solve the residual term is ~1e-12, so A M v must not move after accepted moves."""
    K = 6
    s = O.system(K)
    R = O.initial_positions(s, 2, 0.1)
    ctx = vmc.vmc_create([(K, 0, 1.0, 2.0, 1.5)], vmc.params(precision=0, max_updates=64))
    try:
        vmc.vmc_set_positions(ctx, 0, R)
        rng = np.random.default_rng(5)
        v = rng.standard_normal(216)
        A0, _, _ = vmc.vmc_get_matrix(ctx, 0)
        amv0 = A0 @ vmc.vmc_apply_preconditioner(ctx, 0, v)
        moved = 0
        for step, k in enumerate([3, 50, 120, 77, 200, 9]):
            r_new = O.propose(s, 2, 1, k, 0.2, R[k])
            ratio = vmc.vmc_ratio(ctx, 0, k, r_new)
            if ratio * ratio > 0.05:
                vmc.vmc_accept(ctx, 0)
                R[k] = r_new
                moved += 1
        st = vmc.vmc_get_stats(ctx, 0)
        assert moved >= 3 and st["n_updates"] == moved and st["reorders"] == 0
        A1, _, _ = vmc.vmc_get_matrix(ctx, 0)
        assert np.abs(A1 - A0).max() > 1e-3          # the matrix did change
        amv1 = A1 @ vmc.vmc_apply_preconditioner(ctx, 0, v)
        assert np.abs(amv1 - amv0).max() <= 1e-9 * np.abs(amv0).max()
    finally:
        vmc.vmc_destroy(ctx)


@pytest.mark.parametrize("K,jitter", [(6, 0.1), (6, 0.3), (10, 0.2)])
def test_reordering_matches_oracle_greedy_rule(vmc, K, jitter):
    s = O.system(K)
    Z = O.sites(s)
    R = O.initial_positions(s, 11, jitter)
    ctx = vmc.vmc_create([(K, 0, 1.0, 2.0, 1.5)], vmc.params(precision=1))
    try:
        vmc.vmc_set_positions(ctx, 0, R)
        _, por, ooc = vmc.vmc_get_matrix(ctx, 0)
    finally:
        vmc.vmc_destroy(ctx)
    cols = _colour_order(K)
    assert np.array_equal(ooc, cols)
    P0 = cols.astype(np.int32)            # start: particle i paired with orbital i
    P, Q = O.greedy_pairing(s, R, Z, P0, cols.astype(np.int32))
    partner = np.empty(K ** 3, dtype=np.int64)
    partner[Q] = P                         # orbital -> particle
    assert np.array_equal(por, partner[ooc])


@pytest.fixture(scope="module")
def hard_positions():
    """n = 1000 positions after 20 Sherman-Morrison sweeps (hard, pivoting matrices)."""
    s = O.system(10, 0, 1.0, 2.0, 1.5)
    R0 = O.initial_positions(s, 3, 0.1)
    return O.chain(s, 3, 0.2, R0, 20, solver=O.SOLVER_SHERMAN_MORRISON)[0]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_shared_memory_ilutp_gives_the_dense_row_factors(vmc, hard_positions, prec):
    """The shared-memory ILUTP (hashed working row) performs the elimination, drop, lfil
    and pivot steps of the dense-working-row variant in the same order: the factors, the
    permutation and a partial sweep's logs agree bit for bit."""
    R = hard_positions
    out = []
    for variant in (2, 1):
        ctx = vmc.vmc_create([(10, 0, 1.0, 2.0, 1.5)], vmc.params(precision=prec, ilutp_variant=variant,
                                                                 sweep_moves=200))
        try:
            vmc.vmc_set_positions(ctx, 0, R)
            L, U, perm = vmc.vmc_get_factors(ctx, 0)
            st = vmc.vmc_get_stats(ctx, 0)
            vmc.vmc_set_sweep_count(ctx, 20)
            acc, rat = vmc.vmc_sweep(ctx, 1, 0.2, [3])
            out.append((L, U, perm, st["pivots"], acc[:200].copy(), rat[:200].copy()))
        finally:
            vmc.vmc_destroy(ctx)
    (L0, U0, p0, v0, a0, r0), (L1, U1, p1, v1, a1, r1) = out
    assert np.array_equal(p0, p1) and v0 == v1
    assert np.array_equal(L0.view(np.uint64), L1.view(np.uint64))
    assert np.array_equal(U0.view(np.uint64), U1.view(np.uint64))
    assert np.array_equal(a0, a1) and np.array_equal(r0.view(np.uint64), r1.view(np.uint64))


@pytest.mark.parametrize("prec", [0, 1])
def test_grouped_triangular_solves_apply_the_same_preconditioner(vmc, hard_positions, prec):
    """The grouped (partitioned-inverse) triangular solves apply the operator of the
    level-by-level substitution: same factors, results equal to rounding, far fewer
    synchronisation steps."""
    R = hard_positions
    rng = np.random.default_rng(5)
    v = rng.standard_normal(1000)
    out = {}
    # (levels a group, expanded-row cap, entries a lane); the last two cases size the lane
    # groups differently (level by level and grouped)
    cases = ((1, 0, 0), (8, 0, 0), (16, 400, 0), (1, 0, 16), (8, 0, 1))
    for case in cases:
        group, row_cap, lane_entries = case
        ctx = vmc.vmc_create([(10, 0, 1.0, 2.0, 1.5)], vmc.params(precision=prec, trisolve_group=group,
                                                                  trisolve_row_cap=row_cap,
                                                                  trisolve_lane_entries=lane_entries))
        try:
            vmc.vmc_set_positions(ctx, 0, R)
            L, U, perm = vmc.vmc_get_factors(ctx, 0)
            out[case] = (vmc.vmc_apply_preconditioner(ctx, 0, v), L, U, vmc.vmc_get_stats(ctx, 0))
        finally:
            vmc.vmc_destroy(ctx)
    z1, L1, U1, s1 = out[cases[0]]
    tol = 1e-12 if prec == 0 else 1e-5
    assert s1["groups_L"] == s1["levels_L"] and s1["groups_U"] == s1["levels_U"]
    for case in cases[1:]:
        zg, Lg, Ug, sg = out[case]
        assert np.array_equal(L1, Lg) and np.array_equal(U1, Ug)
        assert np.abs(zg - z1).max() <= tol * np.abs(z1).max()
        if case[0] > 1:
            assert sg["groups_L"] < sg["levels_L"] and sg["groups_U"] < sg["levels_U"]
            assert sg["stream_bytes"] > s1["stream_bytes"]  # the expanded rows are longer
    # longer expanded rows and more levels a group: fewer groups
    s16, s8 = out[cases[2]][3], out[cases[1]][3]
    assert s16["groups_L"] + s16["groups_U"] < s8["groups_L"] + s8["groups_U"]
