"""Pins for the oracle's Metropolis chain (Sec. 2.2) and kinetic energy (Eq. 21, Sec. 4)."""
import math

import numpy as np
import pytest


def test_three_ratio_solvers_agree_on_a_chain(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    R0 = orc.initial_positions(s, 1, 0.1)
    Rd, rd, ad, ud = orc.chain(s, 1, 0.2, R0, 1, solver=orc.SOLVER_DENSE_LU)
    Rs, rs, as_, us = orc.chain(s, 1, 0.2, R0, 1, solver=orc.SOLVER_SHERMAN_MORRISON, refresh=50)
    Rg, rg, ag, ug = orc.chain(s, 1, 0.2, R0, 1, solver=orc.SOLVER_GMRES)
    assert len(rd) == 216
    assert np.abs(rs - rd).max() < 1e-11 and np.abs(rg - rd).max() < 1e-11
    assert np.array_equal(ad, as_) and np.array_equal(ad, ag)
    assert np.array_equal(Rd, Rs) and np.array_equal(Rd, Rg)


def test_accept_rule_is_strict_ratio_squared_above_uniform(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    R0 = orc.initial_positions(s, 2, 0.1)
    R, r, a, u = orc.chain(s, 2, 0.2, R0, 2, solver=orc.SOLVER_SHERMAN_MORRISON)
    assert np.array_equal(a, r * r > u)
    for k in range(len(u)):
        sweep, p = divmod(k, 216)
        assert u[k] == orc.accept_uniform(2, sweep, p)
    assert 0.3 < a.mean() < 0.9
    # positions change exactly for accepted moves
    R1, _, a1, _ = orc.chain(s, 2, 0.2, R0, 1, solver=orc.SOLVER_SHERMAN_MORRISON)
    moved = np.any(R1 != R0, axis=1)
    assert np.array_equal(moved, a1[:216])


def test_chain_resumes_across_sweeps(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    R0 = orc.initial_positions(s, 3, 0.1)
    R2, r2, a2, _ = orc.chain(s, 3, 0.2, R0, 2, solver=orc.SOLVER_SHERMAN_MORRISON)
    Ra, ra, aa, _ = orc.chain(s, 3, 0.2, R0, 1, solver=orc.SOLVER_SHERMAN_MORRISON)
    Rb, rb, ab, _ = orc.chain(s, 3, 0.2, Ra, 1, first_sweep=1, solver=orc.SOLVER_SHERMAN_MORRISON)
    assert np.array_equal(np.concatenate([aa, ab]), a2)
    assert np.abs(np.concatenate([ra, rb]) - r2).max() < 1e-12
    assert np.array_equal(Rb, R2)


def test_multi_walker_chains_equal_single_chains(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    seeds = [1, 2, 3]
    R0 = np.stack([orc.initial_positions(s, w, 0.1) for w in seeds])
    R, rl, al = orc.chains(s, seeds, 0.2, R0, 1, solver=orc.SOLVER_SHERMAN_MORRISON, threads=2)
    for k, w in enumerate(seeds):
        Rw, rw, aw, _ = orc.chain(s, w, 0.2, R0[k], 1, solver=orc.SOLVER_SHERMAN_MORRISON)
        assert np.array_equal(aw, al[k]) and np.array_equal(R[k], Rw)


def test_kinetic_energy_isolated_orbitals(orc):
    """With r_c < a/2 every electron sees at most one orbital, A is a scaled permutation
    and Eq. 21 reduces to (1/2n) sum_p (6k - 4k^2 d_p^2); at the sites it is 3k."""
    kappa = 1.3
    s = orc.system(4, 0, 1.0, kappa, 0.45)
    Z = orc.sites(s)
    assert orc.kinetic_energy(s, Z, Z) == pytest.approx(3 * kappa, rel=1e-13)
    rng = np.random.default_rng(0)
    delta = rng.uniform(-0.2, 0.2, size=Z.shape)
    R = np.mod(Z + delta, 4.0)
    d2 = (delta ** 2).sum(axis=1)
    expect = np.sum(6 * kappa - 4 * kappa ** 2 * d2) / (2 * len(Z))
    assert orc.kinetic_energy(s, Z, R) == pytest.approx(expect, rel=1e-12)
