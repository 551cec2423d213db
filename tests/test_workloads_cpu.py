"""The synthetic workload parameter sets: sizes, walker counts and laws of the five
configured workloads, and the reading of the paper's drop rule for its own model."""
import math

from paper_1008_5113_gb300 import workloads as WL


def test_configured_workloads():
    plain, batch, mixed, uneven, large = WL.PLAIN_216, WL.BATCH_1000, WL.MIXED_4096, WL.UNEVEN_320, WL.LARGE_32768
    assert plain.n_of(6) == 216 and plain.n_walkers == 1 and plain.sweeps == 10
    assert batch.n_of(10) == 1000 and batch.n_walkers == 64 and batch.seeds() == list(range(1, 65))
    assert mixed.n_of(16) == 4096 and mixed.n_walkers == 256 and mixed.precision == "mixed"
    assert sorted({uneven.n_of(K) for K in uneven.Ks}) == [512, 1000, 1728, 4096, 8000]
    assert uneven.n_walkers == 320 and uneven.walkers_per_K == 64
    assert large.n_of(32) == 32768 and large.n_walkers == 32
    assert (large.kappa, large.r_c, large.sigma) == (1.0, 2.0, 0.25)
    for wl in (plain, batch, mixed, uneven):
        assert (wl.kappa, wl.r_c, wl.a, wl.jitter, wl.sigma) == (2.0, 1.5, 1.0, 0.1, 0.2)
        systems = wl.systems()
        assert len(systems) == wl.n_walkers and all(len(s) == 5 for s in systems)


def test_paper_workload_reading():
    """Entries below 1e-5 of the largest (1, at a site) dropped <=> hard cutoff at r_c."""
    wl = WL.PAPER_BCC
    assert wl.lattice == 1 and wl.a == 2.031 and wl.kappa == 1.0
    assert math.isclose(math.exp(-wl.kappa * wl.r_c ** 2), 1e-5, rel_tol=1e-12)
    assert wl.n_of(7) == 686                      # the paper's smallest size
    assert math.isclose(wl.jitter, 0.1 * wl.a) and math.isclose(wl.sigma, 0.2 * wl.a)
    assert WL.PAPER_SOLVER == dict(drop_tol=0.01, permtol=0.05, gmres_m=40, inner_rtol=1e-6)
