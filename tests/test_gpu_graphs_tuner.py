"""GPU checks of the sweep graphs (STEP / PLAIN engines replayed from a captured CUDA
graph) and of the autotuner.  A graph replays exactly the launches it captured, so the
logs must equal the launch-by-launch ones bit for bit; the tuned parameters must give
the oracle's ratios."""
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


def _logs(vmc, engine, graphs, calls=2, prec=1):
    wl = WL.PLAIN_216
    ctx = vmc.vmc_create(wl.systems() * 2, vmc.params(precision=prec, engine=engine, graphs=graphs))
    try:
        vmc.vmc_init_positions(ctx, [1, 2], wl.jitter)
        out = [vmc.vmc_sweep(ctx, 1, wl.sigma, [1, 2]) for _ in range(calls)]
        return out, vmc.vmc_get_positions(ctx, 1)
    finally:
        vmc.vmc_destroy(ctx)


@pytest.mark.parametrize("engine", ["step", "plain"])
def test_graph_replay_equals_launches(vmc, engine):
    eng = vmc.ENGINE_STEP if engine == "step" else vmc.ENGINE_PLAIN
    g, Rg = _logs(vmc, eng, 1)
    l, Rl = _logs(vmc, eng, 0)
    for (ag, rg), (al, rl) in zip(g, l):
        assert np.array_equal(ag, al) and np.array_equal(rg, rl)
    assert np.array_equal(Rg, Rl)


def test_graph_multi_sweep_without_logs(vmc):
    """Several sweeps in one call without logs: the sweep index advances on the device."""
    import torch

    wl = WL.PLAIN_216
    res = []
    for graphs in (1, 0):
        ctx = vmc.vmc_create(wl.systems(), vmc.params(precision=1, engine=vmc.ENGINE_STEP, graphs=graphs))
        try:
            vmc.vmc_init_positions(ctx, [1], wl.jitter)
            sd = torch.tensor([1], dtype=torch.int64, device="cuda")
            vmc.vmc_sweep_async(ctx, 3, wl.sigma, sd)
            vmc.vmc_synchronize(ctx)
            res.append((vmc.vmc_get_positions(ctx, 0), vmc.vmc_sweep_count(ctx), vmc.vmc_get_stats(ctx, 0)))
        finally:
            vmc.vmc_destroy(ctx)
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] == 3
    assert res[0][2]["proposals"] == res[1][2]["proposals"] == 3 * 216


def test_autotune_picks_a_valid_mapping(vmc):
    wl = WL.PLAIN_216
    systems = wl.systems() * 4
    p, trials = vmc.vmc_autotune(systems, vmc.params(precision=1), [1, 2, 3, 4], wl.jitter, wl.sigma, 96)
    assert len(trials) >= 7 and all(t["status"] == 0 and t["ratios_per_s"] > 0 for t in trials)
    best = max(trials, key=lambda t: t["ratios_per_s"])
    assert (p.engine, p.block_threads, p.max_updates, p.lfil_extra) == (best["engine"], best["block_threads"],
                                                                         best["max_updates"], best["lfil_extra"])
    assert {t["lfil_extra"] for t in trials} >= {-1, 16, 32, 48}   # the fill limits were tried
    assert any(t["refactor_lag"] > 0 for t in trials)       # the walker-pair mapping was tried
    assert {t["engine"] for t in trials} >= {vmc.ENGINE_PERSISTENT, vmc.ENGINE_STEP}
    # the tuned parameters reproduce the oracle's chain
    ctx = vmc.vmc_create(wl.systems(), p)
    try:
        vmc.vmc_init_positions(ctx, [1], wl.jitter)
        acc, rat = vmc.vmc_sweep(ctx, 1, wl.sigma, [1])
    finally:
        vmc.vmc_destroy(ctx)
    s = O.system(6, 0, wl.a, wl.kappa, wl.r_c)
    R0 = O.initial_positions(s, 1, wl.jitter)
    _, r_ref, a_ref, u_ref = O.chain(s, 1, wl.sigma, R0, 1, solver=O.SOLVER_SHERMAN_MORRISON)
    bad = np.nonzero(acc != a_ref)[0]
    upto = int(bad[0]) if len(bad) else len(acc)
    if upto < len(acc):
        assert abs(r_ref[upto] ** 2 - u_ref[upto]) < TIE
    lim = np.where(np.abs(r_ref[:upto]) >= 1e-3, RTOL * np.abs(r_ref[:upto]), ATOL)
    assert np.all(np.abs(rat[:upto] - r_ref[:upto]) <= lim) and upto > 100


def test_autotune_from_a_given_state(vmc):
    """Trials can start from a supplied state (e.g. an equilibrated one) and sweep index."""
    wl = WL.PLAIN_216
    s = O.system(6, 0, wl.a, wl.kappa, wl.r_c)
    R0 = np.stack([O.initial_positions(s, w, wl.jitter) for w in (1, 2)])
    R, _, _ = O.chains(s, [1, 2], wl.sigma, R0, 5, solver=O.SOLVER_SHERMAN_MORRISON)
    p, trials = vmc.vmc_autotune(wl.systems() * 2, vmc.params(precision=1), [1, 2], wl.jitter, wl.sigma, 64,
                                 xyz=[R[0], R[1]], sweep0=5)
    assert trials and all(t["status"] == 0 and t["ratios_per_s"] > 0 for t in trials)
