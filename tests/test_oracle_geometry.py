"""Pins for the oracle's lattice, orbitals and Slater matrix (Sec. 2.1 Eqs. 2-3; Sec. 4)."""
import itertools
import math

import numpy as np
import pytest

from conftest import read_golden


def _count_vectors(lattice, a, rc):
    """Brute-force count of lattice vectors within rc (independent of the oracle)."""
    basis = [(0.0, 0.0, 0.0)] if lattice == "sc" else [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)]
    m = int(math.ceil(rc / a)) + 1
    c = 0
    for i, j, k in itertools.product(range(-m, m + 1), repeat=3):
        for b in basis:
            v = (a * (i + b[0]), a * (j + b[1]), a * (k + b[2]))
            if v[0] ** 2 + v[1] ** 2 + v[2] ** 2 <= rc * rc:
                c += 1
    return c


@pytest.mark.parametrize("row", read_golden("lattice_shell_counts.txt"))
def test_row_count_at_sites_matches_shell_count(orc, row):
    lat, a, rc, count = row[0], float(row[1]), float(row[2]), int(row[3])
    assert _count_vectors(lat, a, rc) == count
    K = 6 if lat == "sc" else 4
    s = orc.system(K, 0 if lat == "sc" else 1, a, 1.0, rc)
    Z = orc.sites(s)
    A = orc.slater_dense(s, Z, Z)
    assert np.all((A != 0).sum(axis=1) == count)


def test_sites_are_the_lattice(orc):
    s = orc.system(4, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    assert Z.shape == (64, 3)
    assert np.array_equal(Z[1], [1, 0, 0]) and np.array_equal(Z[4], [0, 1, 0]) and np.array_equal(Z[16], [0, 0, 1])
    b = orc.system(4, 1, 2.0, 1.0, 3.0)
    Zb = orc.sites(b)
    assert Zb.shape == (128, 3)
    assert np.array_equal(Zb[0], [0, 0, 0]) and np.array_equal(Zb[1], [1, 1, 1]) and np.array_equal(Zb[2], [2, 0, 0])


def test_orbital_values_closed_form(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    r = Z[0].copy()
    row = orc.row_dense(s, Z, r)
    assert row[0] == 1.0
    assert row[1] == pytest.approx(math.exp(-2.0), rel=1e-15)        # |d| = 1
    assert row[1 + 6] == pytest.approx(math.exp(-4.0), rel=1e-15)    # |d| = sqrt 2
    assert row[1 + 6 + 36] == 0.0                                    # |d| = sqrt 3 > r_c
    # minimum image across the periodic boundary: x = L - 0.1 is 0.1 from site 0
    r2 = np.array([6.0 - 0.1, 0.0, 0.0])
    row2 = orc.row_dense(s, Z, r2)
    assert row2[0] == pytest.approx(math.exp(-2.0 * 0.01), rel=1e-14)
    assert row2[5] == pytest.approx(math.exp(-2.0 * 0.81), rel=1e-14)
    # the cutoff keeps d == r_c (zeroed only beyond r_c)
    r3 = np.array([1.5, 0.0, 0.0])
    row3 = orc.row_dense(s, Z, r3)
    assert row3[0] == pytest.approx(math.exp(-2.0 * 2.25), rel=1e-15)


@pytest.mark.parametrize("lat,K,a,rc", [("sc", 10, 1.0, 1.5), ("sc", 10, 1.0, 2.0), ("bcc", 6, 2.031, 3.393)])
def test_mean_row_count_for_uniform_positions(orc, lat, K, a, rc):
    """For uniformly random electrons the expected number of orbitals per row is the
    site density times the ball volume (every site is in the ball with probability
    vol(ball)/vol(box))."""
    s = orc.system(K, 0 if lat == "sc" else 1, a, 1.0, rc)
    n = orc.n_of(s)
    Z = orc.sites(s)
    L = K * a
    rng = np.random.default_rng(0)
    R = rng.uniform(0, L, size=(n, 3))
    A = orc.slater_dense(s, Z, R)
    mean = (A != 0).sum() / n
    expect = n / L ** 3 * 4.0 / 3.0 * math.pi * rc ** 3
    sd = math.sqrt(expect / n)  # Poisson-like spread of the mean
    assert abs(mean - expect) < 6 * sd


def test_initial_positions_and_proposals_stay_in_box(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 1, 0.1)
    assert np.all((R >= 0) & (R < 6.0))
    d = R - Z
    d -= 6.0 * np.round(d / 6.0)
    assert 0.05 < np.sqrt((d ** 2).mean() / 3) < 0.15          # jitter 0.1 per coordinate
    for p in range(20):
        r1 = orc.propose(s, 1, 0, p, 0.2, R[p])
        assert np.all((r1 >= 0) & (r1 < 6.0))
        dd = r1 - R[p]
        dd -= 6.0 * np.round(dd / 6.0)
        assert np.all(np.abs(dd) < 0.2 * 7)
    # sigma = 0 proposes the same point
    assert np.array_equal(orc.propose(s, 1, 0, 3, 0.0, R[3]), R[3])


def test_csr_matches_dense(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    R = orc.initial_positions(s, 2, 0.1)
    A = orc.slater_dense(s, Z, R)
    rp, ci, cv = orc.slater_csr(s, Z, R)
    B = np.zeros_like(A)
    for i in range(A.shape[0]):
        B[i, ci[rp[i]:rp[i + 1]]] = cv[rp[i]:rp[i + 1]]
    assert np.array_equal(A, B)
