"""Pins for the oracle's greedy particle/orbital reordering (Sec. 3.1)."""
import numpy as np


def _d2(s_K, a, r, z):
    L = s_K * a
    d = r - z
    d -= L * np.round(d / L)
    return float((d * d).sum())


def test_electrons_at_sites_pair_with_their_sites_whatever_the_labels(orc):
    s = orc.system(4, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    n = len(Z)
    rng = np.random.default_rng(0)
    perm = rng.permutation(n)
    R = Z[perm]                          # particle p sits on site perm[p]
    P = rng.permutation(n).astype(np.int32)
    Q = rng.permutation(n).astype(np.int32)
    P2, Q2 = orc.greedy_pairing(s, R, Z, P, Q)
    assert sorted(P2) == list(range(n)) and sorted(Q2) == list(range(n))
    assert np.array_equal(perm[P2], Q2)  # every position pairs a particle with its own site


def test_greedy_rule_by_brute_force(orc):
    """Literal transcription of the rule in numpy, on small jittered systems."""
    s = orc.system(3, 0, 1.0, 2.0, 1.45)
    Z = orc.sites(s)
    n = len(Z)
    for seed in range(4):
        R = orc.initial_positions(s, seed + 1, 0.35)
        rng = np.random.default_rng(seed)
        P = rng.permutation(n).astype(np.int32)
        Q = rng.permutation(n).astype(np.int32)
        P2, Q2 = orc.greedy_pairing(s, R, Z, P, Q)
        P, Q = list(P), list(Q)
        for i in range(n - 1):
            ds = [_d2(3, 1.0, R[P[i]], Z[Q[j]]) for j in range(i, n)]
            j = i + int(np.argmin(ds))
            if j != i:
                Q[i], Q[j] = Q[j], Q[i]
            else:
                ds = [_d2(3, 1.0, R[P[k]], Z[Q[i]]) for k in range(i, n)]
                k = i + int(np.argmin(ds))
                if k != i:
                    P[i], P[k] = P[k], P[i]
        assert np.array_equal(P2, P) and np.array_equal(Q2, Q)


def test_greedy_makes_the_diagonal_large(orc):
    s = orc.system(6, 0, 1.0, 2.0, 1.5)
    Z = orc.sites(s)
    n = len(Z)
    R = orc.initial_positions(s, 3, 0.1)
    rng = np.random.default_rng(3)
    P, Q = orc.greedy_pairing(s, R, Z, rng.permutation(n), rng.permutation(n))
    A = orc.slater_dense(s, Z, R)
    nearest = np.argmax(A, axis=1)            # each particle's nearest site
    assert np.mean(nearest[P] == Q) > 0.95    # nearly all pairs are (particle, its nearest site)
    assert np.all(A[P, Q] > 0.0)              # every pair within the cutoff
