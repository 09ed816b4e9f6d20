"""Seeded synthetic workloads: run parameters and random inputs.

This module holds no arithmetic of the method.  It defines the lattice sizes,
couplings, measurement schedules, separations and probe sets of the
workloads below, and draws seeded random inputs (start configurations, gauge
transformations, batch and request mixes) with numpy's PCG64 generator.

The paper simulates 24^3 x N_t lattices, N_t in {4, 8, 12, 24}, near beta = 1
(Section II; Section III.B), with fields measured on the mediator plane of the
static charges.  The workloads restate that setting at nearby sizes.
"""

from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

COMP_ALL = 0x3F       # Ex, Ey, Ez, Bx, By, Bz
COMP_EX = 0x01
COMP_EX_BX = 0x09


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    Nt: int
    beta: float
    seed: int
    fp64: bool
    n_therm: int
    slab: int
    n_sub: int
    n_meas: int
    r: tuple
    rf: tuple
    probes: tuple
    comp_mask: int
    outer_slab: int = 0
    n_sub_outer: int = 0
    k_between: int = 10
    n_or: int = 3
    extra: dict = field(default_factory=dict)

    @property
    def V(self) -> int:
        return self.L ** 3 * self.Nt

    @property
    def links(self) -> int:
        return 4 * self.V

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _probes_y(dmax: int) -> tuple:
    return tuple((d, 0) for d in range(dmax + 1))


# 8^3 x 4, beta 0.9, FP64, 50 thermalisation sweeps, slabs of 2 with 20
# sub-updates, 5 measurements, P(r) r = 1..4, Ex/Bx at r = 2, 4, offsets 0..3.
SMALL_FP64 = Workload("plain-8x8x8x4-fp64", L=8, Nt=4, beta=0.9, seed=1, fp64=True, n_therm=50, slab=2,
                      n_sub=20, n_meas=5, r=(1, 2, 3, 4), rf=(2, 4), probes=_probes_y(3),
                      comp_mask=COMP_EX_BX)

# 24^3 x 8, beta 0.98, FP32 angles, 200 thermalisation sweeps, slabs of 2 with
# 100 sub-updates, 20 measurements, P(r) r = 2..12, all six components on the
# mid-plane at offsets 0..8 for every r of the list.
SINGLE_24 = Workload("single-24x24x24x8-fp32", L=24, Nt=8, beta=0.98, seed=1, fp64=False, n_therm=200,
                     slab=2, n_sub=100, n_meas=20, r=tuple(range(2, 13)), rf=tuple(range(2, 13)),
                     probes=_probes_y(8), comp_mask=COMP_ALL)

# 48^3 x 16, beta 0.99, FP32, two levels (outer 4 with n4 = 20, inner 2 with
# n2 = 200), P(r) r = 2..24, six components at r = 8, 16, 24, offsets 0..12.
LARGE_48 = Workload("two-level-48x48x48x16-fp32", L=48, Nt=16, beta=0.99, seed=1, fp64=False, n_therm=200,
                    slab=2, n_sub=200, n_meas=1, r=tuple(range(2, 25)), rf=(8, 16, 24),
                    probes=_probes_y(12), comp_mask=COMP_ALL, outer_slab=4, n_sub_outer=20)

WORKLOADS = {w.name: w for w in (SMALL_FP64, SINGLE_24, LARGE_48)}


# ----------------------------------------------------------------------------- random inputs
def random_angles(L: int, Nt: int, seed: int) -> np.ndarray:
    """Uniform angles in [-pi, pi), canonical layout [4][V] (float64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=(4, L ** 3 * Nt))


def random_gauge(L: int, Nt: int, seed: int) -> np.ndarray:
    """Uniform gauge angles lambda(x) in [-pi, pi) at every site (float64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=L ** 3 * Nt)


def batch_mix(n: int = 64, master_seed: int = 2024):
    """(L, Nt, beta, seed) of ``n`` independent lattices: L from {12,16,20,24},
    N_t from {4,6,8,10,12}, beta uniform in [0.94, 0.99]."""
    rng = np.random.default_rng(master_seed)
    Ls = rng.choice([12, 16, 20, 24], size=n)
    Nts = rng.choice([4, 6, 8, 10, 12], size=n)
    betas = rng.uniform(0.94, 0.99, size=n)
    return [(int(Ls[b]), int(Nts[b]), float(betas[b]), master_seed * 1000 + b) for b in range(n)]


def request_stream(n: int, rate_per_s: float, seed: int = 7):
    """Poisson arrivals of ``n`` requests: (t_arrival_s, L, Nt, beta, seed);
    L from {12,...,32}, N_t from {4,...,12}, beta uniform in [0.94, 0.99]."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    t = np.cumsum(gaps)
    Ls = rng.choice([12, 16, 20, 24, 28, 32], size=n)
    Nts = rng.choice([4, 6, 8, 10, 12], size=n)
    betas = rng.uniform(0.94, 0.99, size=n)
    return [(float(t[i]), int(Ls[i]), int(Nts[i]), float(betas[i]), i) for i in range(n)]
