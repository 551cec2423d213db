"""GPU checks of background refactorisation (persistent engine, a factor CTA per walker).

The factor CTA factors a snapshot of A while the solver steps; the solver adopts the new
factors a fixed number of accepts later and re-roots the update chain on them (Sec. 3.2
Eqs. 16-18 hold for any root).  The ratios must stay the oracle's, the runs must be
reproducible bit for bit (the adoption points do not depend on timing), and stale
requests (a reorder in between) must be dropped cleanly."""
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


@pytest.fixture(scope="module")
def reference():
    s = O.system(6)
    R0 = O.initial_positions(s, 1, 0.1)
    _, r, a, u = O.chain(s, 1, 0.2, R0, 2, solver=O.SOLVER_SHERMAN_MORRISON)
    return r, a, u


def _check(rat, acc, ref, min_len):
    r_ref, a_ref, u_ref = ref
    bad = np.nonzero(acc != a_ref)[0]
    upto = int(bad[0]) if len(bad) else len(acc)
    if upto < len(acc):
        assert abs(r_ref[upto] ** 2 - u_ref[upto]) < TIE, f"decision differs at step {upto} away from a tie"
    lim = np.where(np.abs(r_ref[:upto]) >= 1e-3, RTOL * np.abs(r_ref[:upto]), ATOL)
    err = np.abs(rat[:upto] - r_ref[:upto])
    assert np.all(err <= lim), f"ratio mismatch at step {int(np.argmax(err - lim))}"
    assert upto >= min_len


def _run(vmc, walkers=1, sweeps=2, calls=1, **kw):
    wl = WL.PLAIN_216
    seeds = list(range(1, walkers + 1))
    ctx = vmc.vmc_create(wl.systems() * walkers, vmc.params(engine=vmc.ENGINE_PERSISTENT, **kw))
    try:
        vmc.vmc_init_positions(ctx, seeds, wl.jitter)
        logs = [vmc.vmc_sweep(ctx, sweeps // calls, wl.sigma, seeds) for _ in range(calls)]
        acc = np.concatenate([a.reshape(walkers, -1) for a, _ in logs], axis=1)
        rat = np.concatenate([r.reshape(walkers, -1) for _, r in logs], axis=1)
        st = [vmc.vmc_get_stats(ctx, w) for w in range(walkers)]
        z = vmc.vmc_apply_preconditioner(ctx, 0, np.ones(216))
        assert np.all(np.isfinite(z))
        return acc, rat, st
    finally:
        vmc.vmc_destroy(ctx)


@pytest.mark.parametrize("reorder", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_pair_matches_oracle(vmc, reference, prec, reorder):
    """With and without re-pairing rows in the background (the chain is invariant under
    a new row order, so either root is valid)."""
    acc, rat, st = _run(vmc, precision=prec, max_updates=8, refactor_lag=4, refactor_reorder=reorder)
    _check(rat[0], acc[0], reference, 300)
    s = st[0]
    assert s["status"] == 0 and s["async_lag"] == 4
    # every 4 accepts past the first 4 a new factorisation is adopted
    assert s["refactors_async"] >= s["accepts"] // 4 - 3
    assert s["refactors_updates"] == 0 and s["n_updates"] <= 8


def test_pair_is_reproducible_and_launch_independent(vmc):
    """Two identical runs agree bit for bit, and so does the same work split over
    two launches (the factor CTA of each launch finishes its request before leaving)."""
    a1, r1, _ = _run(vmc, walkers=2, precision=1, max_updates=4, refactor_lag=2)
    a2, r2, _ = _run(vmc, walkers=2, precision=1, max_updates=4, refactor_lag=2)
    a3, r3, st = _run(vmc, walkers=2, calls=2, precision=1, max_updates=4, refactor_lag=2)
    assert np.array_equal(a1, a2) and np.array_equal(r1, r2)
    assert np.array_equal(a1, a3) and np.array_equal(r1, r3)
    assert all(s["status"] == 0 and s["refactors_async"] > 20 for s in st)


def test_pair_every_accept(vmc, reference):
    """refactor_lag 1: a snapshot at every accept, adopted at the next one."""
    acc, rat, st = _run(vmc, precision=1, max_updates=2, refactor_lag=1)
    _check(rat[0], acc[0], reference, 300)
    assert st[0]["status"] == 0 and st[0]["refactors_async"] >= st[0]["accepts"] - 3


def test_pair_drops_stale_requests(vmc, reference):
    """A monitor threshold that forces frequent reorders makes requests stale; they are
    dropped and the ratios stay the oracle's."""
    _, _, st0 = _run(vmc, precision=1, max_updates=8, refactor_lag=2)
    mean_N = st0[0]["N_sum"] / st0[0]["solves"]
    thr = 0.5 * (mean_N + st0[0]["N_max_seen"])  # only the larger N values trigger
    acc, rat, st = _run(vmc, precision=1, max_updates=8, refactor_lag=2, N_max=thr)
    _check(rat[0], acc[0], reference, 150)
    s = st[0]
    assert s["status"] == 0 and s["reorder_monitor"] > 5 and s["refactors_async"] > 0


def test_auto_lag(vmc):
    wl = WL.PLAIN_216
    ctx = vmc.vmc_create(wl.systems(), vmc.params())
    try:
        st = vmc.vmc_get_stats(ctx, 0)  # one walker: pairs fit; chain 64, adopted every 32 accepts
        assert st["async_lag"] == 32 and st["max_updates"] == 64
    finally:
        vmc.vmc_destroy(ctx)
    ctx = vmc.vmc_create(wl.systems(), vmc.params(engine=vmc.ENGINE_STEP))
    try:
        st = vmc.vmc_get_stats(ctx, 0)  # in-line refactorisation: the longer default chain
        assert st["async_lag"] == 0 and st["max_updates"] == 128
    finally:
        vmc.vmc_destroy(ctx)
