"""Parity in the regime the benchmark times and at the sizes of the large configurations.

- n = 1000 (FP64 and mixed; background and in-line refactorisation): two walkers are
  taken through 20 sweeps by the oracle's Sherman-Morrison chain (the paper discards 20
  sweeps, Sec. 4), their positions are restored on the device (vmc_set_positions_all,
  vmc_set_sweep_count) and sweep 20 -- the sweep bench.py times, from an equilibrated
  state where the Slater matrices are far harder than at the start -- is compared move
  by move with the oracle's own sweep 20 from the same state.
- uneven batch of 158 walkers (n = 512 x 156, 4096, 8000; more walkers than SMs, so the
  walker CTAs share SMs and the n = 8000 walker's ILUTP working row lives in global
  memory), mixed precision, a chain of at most 4 updates so that in-line
  refactorisations happen within the bounded partial sweep (sweep_moves): the first 60
  moves of the large walkers and of two small ones against the oracle's chains (GMRES
  above n = 1000)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

RTOL, ATOL, TIE = 1e-10, 1e-13, 1e-9
S_EQ = 20


@pytest.fixture(scope="module")
def vmc():
    import torch

    assert torch.cuda.is_available()
    from paper_1008_5113_gb300.build import build_library

    build_library()
    O.build()
    from paper_1008_5113_gb300 import vmc as v

    return v


def _compare(rat, acc, r_ref, a_ref, u_ref, min_len):
    bad = np.nonzero(acc != a_ref)[0]
    upto = int(bad[0]) if len(bad) else len(acc)
    if upto < len(acc):
        assert abs(r_ref[upto] ** 2 - u_ref[upto]) < TIE, f"decision differs at {upto} away from a tie"
    lim = np.where(np.abs(r_ref[:upto]) >= 1e-3, RTOL * np.abs(r_ref[:upto]), ATOL)
    err = np.abs(rat[:upto] - r_ref[:upto])
    assert np.all(err <= lim), f"worst ratio error {np.max(err / np.maximum(lim, 1e-300))} x tolerance"
    assert upto >= min_len
    return upto


@pytest.fixture(scope="module")
def equilibrated():
    """Two walkers (seeds 1, 2) of n = 1000 after S_EQ oracle sweeps, and the oracle's
    sweep S_EQ from there (ratios, decisions, uniforms)."""
    s = O.system(10, 0, 1.0, 2.0, 1.5)
    seeds = [1, 2]
    R0 = np.stack([O.initial_positions(s, w, 0.1) for w in seeds])
    R, _, _ = O.chains(s, seeds, 0.2, R0, S_EQ, solver=O.SOLVER_SHERMAN_MORRISON)
    ref = [O.chain(s, w, 0.2, R[i], 1, first_sweep=S_EQ, solver=O.SOLVER_SHERMAN_MORRISON, refresh=100)
           for i, w in enumerate(seeds)]
    return R, ref


@pytest.mark.parametrize("prec,lag,moves", [(0, -1, 0), (1, -1, 0), (0, 0, 300), (1, 0, 300)])
def test_equilibrated_sweep_matches_oracle(vmc, equilibrated, prec, lag, moves):
    """Full sweeps with background refactorisation (the benchmark's mapping), partial
    sweeps (the first 300 moves) with in-line refactorisation."""
    R, ref = equilibrated
    ctx = vmc.vmc_create([(10, 0, 1.0, 2.0, 1.5)] * 2, vmc.params(precision=prec, refactor_lag=lag,
                                                                  sweep_moves=moves))
    try:
        vmc.vmc_set_positions_all(ctx, [R[0], R[1]])
        vmc.vmc_set_sweep_count(ctx, S_EQ)
        acc, rat = vmc.vmc_sweep(ctx, 1, 0.2, [1, 2])
        st = [vmc.vmc_get_stats(ctx, w) for w in range(2)]
    finally:
        vmc.vmc_destroy(ctx)
    assert st[0]["async_lag"] == (32 if lag == -1 else 0)
    m = moves or 1000
    for w in range(2):
        _, r_ref, a_ref, u_ref = ref[w]
        _compare(rat[w * 1000:w * 1000 + m], acc[w * 1000:w * 1000 + m], r_ref[:m], a_ref[:m], u_ref[:m], 150)
    # the equilibrated matrices are hard: the controller acts during the sweep
    assert sum(s["factorizations"] + s["refactors_async"] for s in st) > 2
    assert all(s["status"] == 0 for s in st)


def test_restore_makes_identical_sweeps(vmc, equilibrated):
    """Restoring the same state and sweep index gives the same sweep bit for bit (the
    benchmark's timed steps are identical work)."""
    R, _ = equilibrated
    ctx = vmc.vmc_create([(10, 0, 1.0, 2.0, 1.5)] * 2, vmc.params(precision=1, sweep_moves=300))
    try:
        logs = []
        for _ in range(2):
            vmc.vmc_set_positions_all(ctx, [R[0], R[1]])
            vmc.vmc_set_sweep_count(ctx, S_EQ)
            acc, rat = vmc.vmc_sweep(ctx, 1, 0.2, [1, 2])
            logs.append((acc.reshape(2, 1000)[:, :300].copy(), rat.reshape(2, 1000)[:, :300].copy()))
            assert vmc.vmc_get_stats(ctx, 0)["proposals"] == 300
    finally:
        vmc.vmc_destroy(ctx)
    assert np.array_equal(logs[0][0], logs[1][0])
    assert np.array_equal(logs[0][1].view(np.uint64), logs[1][1].view(np.uint64))


def test_uneven_partial_sweep_with_inline_refactors_matches_oracle(vmc):
    Ks = [8] * 156 + [16, 20]
    systems = [(K, 0, 1.0, 2.0, 1.5) for K in Ks]
    seeds = list(range(1, len(Ks) + 1))
    moves = 60
    ctx = vmc.vmc_create(systems, vmc.params(precision=1, max_updates=4, refactor_lag=0, sweep_moves=moves))
    try:
        vmc.vmc_init_positions(ctx, seeds, 0.1)
        acc, rat = vmc.vmc_sweep(ctx, 1, 0.2, seeds)
        stats = {w: vmc.vmc_get_stats(ctx, w) for w in (0, 155, 156, 157)}
    finally:
        vmc.vmc_destroy(ctx)
    base = np.concatenate([[0], np.cumsum([K ** 3 for K in Ks])])
    for w in (0, 155, 156, 157):
        K = Ks[w]
        s = O.system(K, 0, 1.0, 2.0, 1.5)
        R0 = O.initial_positions(s, seeds[w], 0.1)
        solver = O.SOLVER_SHERMAN_MORRISON if K ** 3 <= 1000 else O.SOLVER_GMRES
        _, r_ref, a_ref, u_ref = O.chain(s, seeds[w], 0.2, R0, 1, max_steps=moves, solver=solver)
        lo = base[w]
        _compare(rat[lo:lo + moves], acc[lo:lo + moves], r_ref, a_ref, u_ref, moves // 2)
        st = stats[w]
        assert st["proposals"] == moves and st["status"] == 0
        assert st["refactors_updates"] >= 2, st["refactors_updates"]   # in-line refactorisations happened
