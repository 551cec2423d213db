"""GPU checks of the reorder/refactor controller (Sec. 4) and of failure reporting.

Each trigger is forced through the solver parameters; the ratios must stay those of
the oracle (the controller changes the cost of a solve, never its result)."""
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
    _, r, a, u = O.chain(s, 1, 0.2, R0, 1, solver=O.SOLVER_SHERMAN_MORRISON)
    return r, a, u


def _run(vmc, **kw):
    wl = WL.PLAIN_216
    ctx = vmc.vmc_create(wl.systems(), vmc.params(**kw))
    try:
        vmc.vmc_init_positions(ctx, wl.seeds(), wl.jitter)
        acc, rat = vmc.vmc_sweep(ctx, 1, wl.sigma, wl.seeds())
        return acc, rat, vmc.vmc_get_stats(ctx, 0)
    finally:
        vmc.vmc_destroy(ctx)


def _check(rat, acc, ref):
    r_ref, a_ref, u_ref = ref
    bad = np.nonzero(acc != a_ref)[0]
    upto = int(bad[0]) if len(bad) else len(acc)
    if upto < len(acc):
        assert abs(r_ref[upto] ** 2 - u_ref[upto]) < TIE
    lim = np.where(np.abs(r_ref[:upto]) >= 1e-3, RTOL * np.abs(r_ref[:upto]), ATOL)
    assert np.all(np.abs(rat[:upto] - r_ref[:upto]) <= lim)
    assert upto > 100


@pytest.mark.parametrize("prec", [0, 1])
def test_monitor_trigger_reorders(vmc, reference, prec):
    acc, rat, st = _run(vmc, precision=prec, N_max=1e-9)
    _check(rat, acc, reference)
    assert st["reorder_monitor"] > 50 and st["reorders"] == st["reorder_monitor"] + st["reorder_noconv"] + \
        st["reorder_slow"] + st["reorder_breakdown"]


def test_nonconvergence_trigger_and_restarts(vmc, reference):
    """GMRES(3) needs many restarts; a tolerance of 1e-12 to be reached within 3 iterations
    makes every solve count as not converged (reorder + refactor for the next moves)."""
    acc, rat, st = _run(vmc, precision=0, gmres_m=3, max_restarts=40, trigger_rtol=1e-12, trigger_its=3)
    _check(rat, acc, reference)
    assert st["reorder_noconv"] > 10 and st["outer_passes"] > 2 * st["proposals"]
    assert st["trigger_iterations"] > 3 * st["proposals"]


def test_slow_convergence_trigger(vmc, reference):
    acc, rat, st = _run(vmc, precision=1, slow_factor=0.5)
    _check(rat, acc, reference)
    assert st["reorder_slow"] > 10


def test_refactor_after_every_update(vmc, reference):
    acc, rat, st = _run(vmc, precision=1, max_updates=0)
    _check(rat, acc, reference)
    assert st["refactors_updates"] == st["accepts"] and st["n_updates"] == 0


def test_unreachable_tolerance_reports_noconv_cleanly(vmc):
    wl = WL.PLAIN_216
    ctx = vmc.vmc_create(wl.systems(), vmc.params(precision=0, gmres_m=1, max_restarts=0, ratio_tol=1e-300))
    try:
        vmc.vmc_init_positions(ctx, wl.seeds(), wl.jitter)
        with pytest.raises(vmc.VmcError) as e:
            vmc.vmc_sweep(ctx, 1, wl.sigma, wl.seeds())
        assert e.value.status == 4
        st = vmc.vmc_get_stats(ctx, 0)
        assert st["status"] == 4 and st["proposals"] >= 1
    finally:
        vmc.vmc_destroy(ctx)


def test_bounded_wait_reports_timeout_and_context_survives(vmc):
    wl = WL.PLAIN_216
    ctx = vmc.vmc_create(wl.systems(), vmc.params(precision=1))
    try:
        vmc.vmc_init_positions(ctx, wl.seeds(), wl.jitter)
        assert vmc.vmc_check_wait_timeout(ctx) == 6
        acc, rat = vmc.vmc_sweep(ctx, 1, wl.sigma, wl.seeds())   # still usable
        assert np.all(np.isfinite(rat)) and vmc.vmc_get_stats(ctx, 0)["status"] == 0
    finally:
        vmc.vmc_destroy(ctx)
