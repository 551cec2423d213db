"""Synthetic workloads: parameter sets only (no arithmetic of the method).

Each configuration is a simple-cubic lattice of spacing a with Gaussian orbitals
exp(-kappa |r - Z_j|^2) cut at r_c (Sec. 2.1 Eq. 3), electrons started at the sites
plus N(0, jitter^2) per coordinate, Metropolis steps N(0, sigma^2) per coordinate
(Sec. 2.2), walker w seeded with seed w + 1.  Both the CUDA path and the oracle take
their inputs from these parameters; neither imports the other.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    Ks: tuple            # lattice size K per walker group (n = K^3 for sc)
    walkers_per_K: int
    sweeps: int
    kappa: float = 2.0
    r_c: float = 1.5
    a: float = 1.0
    lattice: int = 0
    jitter: float = 0.1
    sigma: float = 0.2
    precision: str = "fp64"   # "fp64" or "mixed"

    @property
    def n_walkers(self) -> int:
        return len(self.Ks) * self.walkers_per_K

    def systems(self):
        out = []
        for K in self.Ks:
            out += [(K, self.lattice, self.a, self.kappa, self.r_c)] * self.walkers_per_K
        return out

    def seeds(self):
        return [w + 1 for w in range(self.n_walkers)]

    def n_of(self, K: int) -> int:
        return K ** 3 * (2 if self.lattice == 1 else 1)


# n = 216, one walker, 10 sweeps, plain FP64 (the small parity case)
PLAIN_216 = Workload("sc6_n216_w1_fp64", (6,), 1, 10)
# n = 1000, 64 walkers (seeds 1..64), 20 sweeps, FP64 batched
BATCH_1000 = Workload("sc10_n1000_w64_fp64", (10,), 64, 20)
# n = 4096, 256 walkers, 10 sweeps, mixed precision
MIXED_4096 = Workload("sc16_n4096_w256_mixed", (16,), 256, 10, precision="mixed")
# uneven batch: n in {512, 1000, 1728, 4096, 8000}, 64 walkers each, mixed
UNEVEN_320 = Workload("sc8-20_uneven_w320_mixed", (8, 10, 12, 16, 20), 64, 10, precision="mixed")
# n = 32768, kappa = 1, r_c = 2, step 0.25, 32 walkers, 5 sweeps, mixed
LARGE_32768 = Workload("sc32_n32768_k1_rc2_w32_mixed", (32,), 32, 5, kappa=1.0, r_c=2.0, sigma=0.25,
                       precision="mixed")

# The paper's own model system (Sec. 4): body-centred cubic lattice of cube side 2.031,
# kappa = 1, matrix entries below 1e-5 of the largest (1, at a site) dropped -- read as the
# cutoff r_c = sqrt(5 ln 10 / kappa) -- n = 2 K^3 (K = 7: n = 686, the paper's smallest);
# start jitter and step scale with the cube side (0.1 a, 0.2 a)
PAPER_BCC = Workload("bcc_a2.031_k1_n686_paper", (7,), 1, 10, kappa=1.0, r_c=math.sqrt(5.0 * math.log(10.0)),
                     a=2.031, lattice=1, jitter=0.2031, sigma=0.4062)
# the paper's solver settings (Sec. 4): ILUTP drop 0.01, column-pivot tolerance 0.05,
# lfil half the average row count (the default), GMRES up to 40 iterations to 1e-6
PAPER_SOLVER = dict(drop_tol=0.01, permtol=0.05, gmres_m=40, inner_rtol=1e-6)

ALL = [PLAIN_216, BATCH_1000, MIXED_4096, UNEVEN_320, LARGE_32768, PAPER_BCC]
