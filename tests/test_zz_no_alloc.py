"""GPU check of vmc_ratio_noalloc, the entry point for callers that cannot allocate
device memory (a framework that owns all device memory through its own pool,
latency-critical code that cannot afford an allocation's implicit synchronisation,
or a process that has already reserved the free memory).  It must return the same
ratio as the regular context-based entry point (vmc_create + vmc_set_positions +
vmc_ratio), on two calls in a row that reuse its fixed device scratch array, and it
must refuse a system whose workspace exceeds that array.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-13


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    from paper_1008_5113_gb300.build import build_library

    build_library()
    O.build()
    from paper_1008_5113_gb300 import vmc

    return vmc, torch


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_ratio_matches_context_ratio_twice(env, prec):
    vmc, torch = env
    system = (10, 0, 1.0, 2.0, 1.5)
    s = O.system(10, 0, 1.0, 2.0, 1.5)
    R = O.initial_positions(s, 7, 0.1)
    moves = [(5, O.propose(s, 7, 0, 5, 0.2, R[5])), (733, O.propose(s, 7, 0, 733, 0.2, R[733]))]
    params = vmc.params(precision=prec)
    ctx = vmc.vmc_create([system], params)
    try:
        vmc.vmc_set_positions(ctx, 0, R)
        ref = [vmc.vmc_ratio(ctx, 0, k, r) for k, r in moves]
    finally:
        vmc.vmc_destroy(ctx)
    # the plain definition: dense LU solve of A z = e_k, ratio 1 + u^T z (Sec. 3 Eq. 13)
    Z = O.sites(s)
    A = O.slater_dense(s, Z, R)
    exact = [O.ratio_dense(A, k, O.row_dense(s, Z, r))[0] for k, r in moves]
    xyz = torch.tensor(R.reshape(-1), dtype=torch.float64, device="cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for (k, r), want, ex in zip(moves, ref, exact):
        out.fill_(float("nan"))
        vmc.vmc_ratio_noalloc(system, params, xyz, k, r, out)
        got = float(out.item())
        assert abs(got - want) <= max(RTOL * abs(want), ATOL), (k, got, want)
        assert abs(got - ex) <= max(RTOL * abs(ex), ATOL), (k, got, ex)


def test_noalloc_wrapper_checks_its_buffers(env):
    vmc, torch = env
    system = (6, 0, 1.0, 2.0, 1.5)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for bad in (torch.zeros(3 * 216 - 1, dtype=torch.float64, device="cuda"),   # too short
                torch.zeros(3 * 216, dtype=torch.float32, device="cuda"),        # wrong dtype
                torch.zeros(3 * 216 * 2, dtype=torch.float64, device="cuda")[::2],  # not contiguous
                torch.zeros(3 * 216, dtype=torch.float64)):                      # host memory
        with pytest.raises(vmc.VmcError) as e:
            vmc.vmc_ratio_noalloc(system, None, bad, 0, [0.1, 0.1, 0.1], out)
        assert e.value.status == 1


def test_noalloc_rejects_systems_beyond_its_scratch(env):
    vmc, torch = env
    xyz = torch.zeros(3 * 8000, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(vmc.VmcError) as e:
        vmc.vmc_ratio_noalloc((20, 0, 1.0, 2.0, 1.5), None, xyz, 0, [0.1, 0.1, 0.1], out)
    assert e.value.status == 8 and "fixed maximum" in str(e.value)
    assert vmc.vmc_noalloc_capacity() == 16 << 20
