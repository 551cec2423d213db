"""GPU checks of the budgeted advance (vmc_advance): the batch makes a total number of
moves claimed dynamically by the walkers; every walker's chain must be the oracle's
chain of the moves that walker made, and the move counts must add up to the budget."""
import numpy as np
import pytest

import oracle as O
from paper_1008_5113_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TIE = 1e-9


@pytest.fixture(scope="module")
def vmc():
    import torch

    assert torch.cuda.is_available()
    from paper_1008_5113_gb300.build import build_library

    build_library()
    O.build()
    from paper_1008_5113_gb300 import vmc as v

    return v


def _moves(vmc, ctx, w, n, sweep0):
    sw, k = vmc.vmc_get_progress(ctx, w)
    return (sw - sweep0) * n + k


@pytest.mark.parametrize("prec,lag", [(0, -1), (1, -1), (1, 0)])
def test_advance_walkers_follow_their_chains(vmc, prec, lag):
    wl = WL.PLAIN_216
    nw, n = 4, 216
    seeds = [1, 2, 3, 4]
    ctx = vmc.vmc_create(wl.systems() * nw, vmc.params(precision=prec, refactor_lag=lag))
    s = O.system(6, 0, wl.a, wl.kappa, wl.r_c)
    try:
        vmc.vmc_init_positions(ctx, seeds, wl.jitter)
        total = 0
        for budget in (nw * 300, nw * 250):
            acc = vmc.vmc_advance(ctx, budget, wl.sigma, seeds)
            total += budget
            m = [_moves(vmc, ctx, w, n, 0) for w in range(nw)]
            assert sum(m) == total and all(x > 0 for x in m)
            st = [vmc.vmc_get_stats(ctx, w) for w in range(nw)]
            assert [x["proposals"] for x in st] == m and list(acc) == [x["accepts"] for x in st]
            for w in range(nw):
                R0 = O.initial_positions(s, seeds[w], wl.jitter)
                R_ref, r_ref, a_ref, u_ref = O.chain(s, seeds[w], wl.sigma, R0, (m[w] + n - 1) // n,
                                                     max_steps=m[w], solver=O.SOLVER_SHERMAN_MORRISON)
                if np.any(np.abs(r_ref ** 2 - u_ref) < TIE):
                    continue  # a tie: the chains may legitimately part
                assert np.abs(vmc.vmc_get_positions(ctx, w) - R_ref).max() <= 1e-13
                assert int(np.sum(a_ref)) == acc[w]
        # a fixed sweep starts every walker at particle 0 of the context's sweep counter again
        vmc.vmc_sweep(ctx, 1, wl.sigma, seeds, logs=False)
        assert all(vmc.vmc_get_progress(ctx, w) == (1, 0) for w in range(nw))
    finally:
        vmc.vmc_destroy(ctx)


def test_advance_needs_the_persistent_engine(vmc):
    wl = WL.PLAIN_216
    ctx = vmc.vmc_create(wl.systems(), vmc.params(precision=1, engine=vmc.ENGINE_STEP))
    try:
        vmc.vmc_init_positions(ctx, [1], wl.jitter)
        with pytest.raises(vmc.VmcError) as e:
            vmc.vmc_advance(ctx, 10, wl.sigma, [1])
        assert e.value.status == 1
    finally:
        vmc.vmc_destroy(ctx)
