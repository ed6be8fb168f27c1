"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This module only describes inputs (model, lattice size, number of chains, seed,
schedules, beta grids, fixed weights).  It holds none of the method's arithmetic and
imports neither the CUDA library nor the oracle.

The paper's workloads are themselves synthetic spin systems (Sec. 3: 2D Ising and
8-state Potts on periodic square lattices, started at infinite temperature), so no
external data set is involved.
"""
import numpy as np

ISING, POTTS = 0, 1

# beta_0 of the two models, Sec. 3: ln(1+sqrt 2)/2 (Ising), ln(1+sqrt 8) (8-Potts)
ISING_BETA0 = 0.4406867935097715
POTTS8_BETA0 = 1.3424540464535260

WORKLOADS = {
    # correctness workload: checked against the exact 8x8 density of states
    "ising_L8_p8": dict(model=ISING, L=8, q=2, p=8, seed=1, iterations=30, sweeps=2000,
                        production=0, betas=None),
    # plain GPU form: 40 x 1000 sweeps, 10^4 production sweeps, 512 betas
    "ising_L64_p1024": dict(model=ISING, L=64, q=2, p=1024, seed=1, iterations=40,
                            sweeps=1000, production=10000, betas=(0.3, 0.6, 512)),
    # 8-Potts: 60 x 500 sweeps, 2x10^4 production sweeps, 1024 betas
    "potts8_L32_p4096": dict(model=POTTS, L=32, q=8, p=4096, seed=1, iterations=60,
                             sweeps=500, production=20000, betas=(1.2, 1.4, 1024)),
    # large lattices at fixed ln W = -beta_0 E, 10^3 production sweeps, 4096 betas
    "ising_L256_p8192": dict(model=ISING, L=256, q=2, p=8192, seed=1, iterations=0,
                             sweeps=0, production=1000, betas=(0.3, 0.6, 4096),
                             fixed_beta=ISING_BETA0),
    "potts8_L128_p4096": dict(model=POTTS, L=128, q=8, p=4096, seed=1, iterations=0,
                              sweeps=0, production=1000, betas=(1.2, 1.4, 4096),
                              fixed_beta=POTTS8_BETA0),
}

# mixed batch: many lattices of uneven size, both models, 256 chains each,
# 20 iterations x 200 sweeps
BATCHED_MIXED = dict(
    jobs=[(ISING, L, 2, 256, 1) for L in (16, 24, 32, 48, 64, 96, 128)]
    + [(POTTS, L, 8, 256, 1) for L in (16, 24, 32, 48)],
    iterations=20, sweeps=200)


def beta_grid(spec):
    """Uniform grid of inverse temperatures from a (lo, hi, n) triple."""
    lo, hi, n = spec
    return np.linspace(lo, hi, n)


def n_bins(model, L):
    return L * L + 1 if model == ISING else 2 * L * L + 1


def canonical_lnw(model, L, beta):
    """Fixed weights ln W(E) = -beta E on the bin grid (a canonical ensemble at beta)."""
    V = L * L
    b = np.arange(n_bins(model, L), dtype=np.float64)
    E = 4.0 * b - 2.0 * V if model == ISING else b - 2.0 * V
    return -beta * E


def random_lnw(model, L, seed, scale=1.0):
    """Seeded random weights for table and update tests."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, n_bins(model, L))


def random_histogram(model, L, seed, lo=1, hi=10 ** 6, zero_frac=0.0):
    rng = np.random.default_rng(seed)
    h = rng.integers(lo, hi, n_bins(model, L)).astype(np.uint64)
    if zero_frac > 0:
        h[rng.random(len(h)) < zero_frac] = 0
    return h
