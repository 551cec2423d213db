"""Parity at the workloads' full sizes.

- n = 1000, 64 walkers, FP64, persistent engine (the launch configuration bench.py
  times): one sweep of every walker; sampled walkers compared move by move with the
  oracle's chain.  The dense explicit-inverse engine likewise.
- uneven batch (walkers of different n in one launch): every walker's trajectory is
  the one it has when run alone.
- n = 4096 (256 walkers, mixed), n = 1000..8000 (uneven, mixed) and n = 32768
  (kappa = 1, r_c = 2, step 0.25, 32 walkers, mixed): the oracle drives the chain
  (its proposals and decisions) and the device computes each move's ratio through
  the single-move API in a context of the full size; ratios compared one by one."""
import numpy as np
import pytest

import oracle as O
from paper_1008_5113_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

RTOL, ATOL, TIE = 1e-10, 1e-13, 1e-9


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


@pytest.mark.parametrize("engine", ["persistent", "dense"])
def test_batch_1000_sweep_matches_oracle(vmc, engine):
    wl = WL.BATCH_1000
    eng = vmc.ENGINE_PERSISTENT if engine == "persistent" else vmc.ENGINE_DENSE_SM
    ctx = vmc.vmc_create(wl.systems(), vmc.params(precision=0, engine=eng))
    try:
        vmc.vmc_init_positions(ctx, wl.seeds(), wl.jitter)
        acc, rat = vmc.vmc_sweep(ctx, 1, wl.sigma, wl.seeds())
        st = [vmc.vmc_get_stats(ctx, w) for w in (0, 63)]
    finally:
        vmc.vmc_destroy(ctx)
    n = 1000
    s = O.system(10, 0, wl.a, wl.kappa, wl.r_c)
    for w in (0, 63):
        seed = wl.seeds()[w]
        R0 = O.initial_positions(s, seed, wl.jitter)
        _, r_ref, a_ref, u_ref = O.chain(s, seed, wl.sigma, R0, 1, solver=O.SOLVER_SHERMAN_MORRISON)
        _compare(rat[w * n:(w + 1) * n], acc[w * n:(w + 1) * n], r_ref, a_ref, u_ref, 300)
    assert all(x["status"] == 0 and x["proposals"] == n for x in st)


def test_uneven_batch_walkers_equal_their_solo_runs(vmc):
    systems = [(6, 0, 1.0, 2.0, 1.5), (8, 0, 1.0, 2.0, 1.5), (7, 0, 1.0, 2.0, 1.5)]
    seeds = [11, 12, 13]
    ctx = vmc.vmc_create(systems, vmc.params(precision=1))
    try:
        vmc.vmc_init_positions(ctx, seeds, 0.1)
        acc, rat = vmc.vmc_sweep(ctx, 1, 0.2, seeds)
    finally:
        vmc.vmc_destroy(ctx)
    off = 0
    for sysw, seed in zip(systems, seeds):
        n = sysw[0] ** 3
        c1 = vmc.vmc_create([sysw], vmc.params(precision=1))
        try:
            vmc.vmc_init_positions(c1, [seed], 0.1)
            a1, r1 = vmc.vmc_sweep(c1, 1, 0.2, [seed])
        finally:
            vmc.vmc_destroy(c1)
        assert np.array_equal(acc[off:off + n], a1) and np.array_equal(rat[off:off + n], r1)
        off += n


def _driven(vmc, systems, walker, kappa, r_c, sigma, steps, solver):
    """The oracle's chain (proposals, ratios, decisions) for `steps` moves of walker
    `walker`; the device computes each ratio through vmc_ratio in a context holding
    all `systems`, accepting whenever the oracle accepts."""
    K = systems[walker][0]
    s = O.system(K, 0, 1.0, kappa, r_c)
    seed = walker + 1
    R0 = O.initial_positions(s, seed, 0.1)
    _, r_ref, a_ref, u_ref = O.chain(s, seed, sigma, R0, 1, max_steps=steps, solver=solver)
    ctx = vmc.vmc_create(systems, vmc.params(precision=1))
    got = np.zeros(steps)
    try:
        vmc.vmc_set_positions(ctx, walker, R0)
        R = R0.copy()
        for k in range(steps):
            r_new = O.propose(s, seed, 0, k, sigma, R[k])
            got[k] = vmc.vmc_ratio(ctx, walker, k, r_new)
            if a_ref[k]:
                vmc.vmc_accept(ctx, walker)
                R[k] = r_new
        assert np.array_equal(vmc.vmc_get_positions(ctx, walker), R)
    finally:
        vmc.vmc_destroy(ctx)
    lim = np.where(np.abs(r_ref) >= 1e-3, RTOL * np.abs(r_ref), ATOL)
    err = np.abs(got - r_ref)
    assert np.all(err <= lim), f"worst ratio error {np.max(err / lim)} x tolerance"


def test_mixed_4096_sampled(vmc):
    wl = WL.MIXED_4096
    _driven(vmc, wl.systems(), 0, wl.kappa, wl.r_c, wl.sigma, 60, O.SOLVER_GMRES)


def test_uneven_320_sampled(vmc):
    wl = WL.UNEVEN_320
    systems = wl.systems()
    for w in (64 * 1, 64 * 4):                     # n = 1000 and n = 8000 walkers of the 320
        _driven(vmc, systems, w, wl.kappa, wl.r_c, wl.sigma, 25, O.SOLVER_GMRES)


def test_large_32768_sampled(vmc):
    wl = WL.LARGE_32768
    _driven(vmc, wl.systems(), 0, wl.kappa, wl.r_c, wl.sigma, 8, O.SOLVER_GMRES)
