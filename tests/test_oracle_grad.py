"""Pins of the oracle's gradient and Laplacian at a proposed position (Sec. 2.2: the
drift and local-energy quantities): finite differences of the separately pinned dense
ratio, and the closed form of isolated orbitals."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


def _support(s, Z, r):
    return np.nonzero(O.row_dense(s, Z, r))[0].tolist()


def test_gradient_and_laplacian_match_finite_differences_of_the_ratio():
    s = O.system(4, 0, 1.0, 2.0, 1.5)
    Z = O.sites(s)
    R = O.initial_positions(s, 7, 0.1)
    A = O.slater_dense(s, Z, R)
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(40):
        i = int(rng.integers(0, 64))
        r_new = (R[i] + rng.normal(0.0, 0.2, 3)) % 4.0
        h = 1e-4
        pts = [r_new + h * np.eye(3)[d] * sgn for d in range(3) for sgn in (1, -1)]
        if any(_support(s, Z, p) != _support(s, Z, r_new) for p in pts):
            continue  # an orbital's cutoff lies within h: the ratio is not smooth there
        ratio, grad, lap = O.ratio_grad_lap(s, Z, R, i, r_new)
        f = lambda r: O.ratio_dense(A, i, O.row_dense(s, Z, r))[0]
        f0 = f(r_new)
        assert abs(ratio - f0) <= 1e-12 * max(1.0, abs(f0))
        fd_grad = np.array([(f(r_new + h * np.eye(3)[d]) - f(r_new - h * np.eye(3)[d])) / (2 * h) for d in range(3)])
        fd_lap = sum((f(r_new + h * np.eye(3)[d]) - 2 * f0 + f(r_new - h * np.eye(3)[d])) / h ** 2 for d in range(3))
        scale = max(1.0, np.abs(fd_grad).max())
        assert np.abs(grad * ratio - fd_grad).max() <= 1e-6 * scale
        assert abs(lap * ratio - fd_lap) <= 1e-3 * max(1.0, abs(fd_lap))
        checked += 1
    assert checked >= 20


def test_isolated_orbitals_closed_form():
    """r_c below half the spacing and small displacements: every electron sees only its
    own orbital, A is diagonal, and grad = -2 kappa (r' - Z_i), lap = 4 kappa^2 d^2 - 6 kappa."""
    kappa = 3.0
    s = O.system(3, 0, 1.0, kappa, 0.45)
    Z = O.sites(s)
    R = O.initial_positions(s, 11, 0.05)
    A = O.slater_dense(s, Z, R)
    assert np.count_nonzero(A - np.diag(np.diag(A))) == 0
    for i in (0, 5, 26):
        r_new = Z[i] + np.array([0.1, -0.07, 0.05])
        ratio, grad, lap = O.ratio_grad_lap(s, Z, R, i, r_new)
        d = r_new - Z[i]
        assert abs(ratio - np.exp(-kappa * d @ d) / A[i, i]) <= 1e-13
        assert np.allclose(grad, -2 * kappa * d, rtol=0, atol=1e-12)
        assert abs(lap - (4 * kappa ** 2 * (d @ d) - 6 * kappa)) <= 1e-11


def test_kinetic_energy_equals_minus_half_mean_laplacian_ratio():
    """Eq. 21 is -(1/2n) sum_p lap_p det A / det A; the oracle's kinetic energy (explicit
    inverse) and its Laplacian at the unmoved positions (LU solves, ratio 1) must agree."""
    for sysw, seed in (((4, 0, 1.0, 2.0, 1.5), 3), ((3, 1, 2.031, 1.0, 2.9), 5)):
        s = O.system(*sysw)
        Z = O.sites(s)
        R = O.initial_positions(s, seed, 0.1)
        n = len(R)
        lap_sum = 0.0
        for p in range(n):
            ratio, _, lap = O.ratio_grad_lap(s, Z, R, p, R[p])
            assert abs(ratio - 1.0) < 1e-12
            lap_sum += lap
        assert abs(O.kinetic_energy(s, Z, R) - (-lap_sum / (2 * n))) <= 1e-10 * max(1.0, abs(lap_sum / n))
