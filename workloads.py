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


# Synthetic production sums for reweighting tests: exact integer per-bin sums
# (count n, sum |M|, sum M^2) and the weights they were "produced" with, shaped like a
# production run of the configurations, with neither the GPU path nor the oracle
# involved.  The energy distribution of the records is exp(V h(e) + ln W(E)) on the
# accessible bins, with a smooth concave entropy density h(e) whose canonical peak
# e*(beta) moves through the configurations' beta ranges (Ising: e* = -2 beta,
# i.e. -0.6 .. -1.2 on [0.3, 0.6]; 8-Potts: e* = -0.75 beta, -0.9 .. -1.05 on
# [1.2, 1.4]).  "flat": ln W = -V h(e), as after converged weight iterations
# (a multicanonical production run); "canonical": ln W = -beta_prod E (fixed weights,
# narrow histogram: reweighting far from beta_prod sits on its edge bins).
# |M| per record: round(V |m(e)| + noise) clipped to [0, Mmax], m(e) a smooth
# order parameter; the sums are exact.
def _entropy_density(model, e):
    if model == ISING:
        return 1.0 - 0.25 * e * e
    return 2.0 * (1.0 - e * e / 3.0)


def synthetic_samples(model, L, mode, n_records, seed, beta_prod=None):
    """(n, s1, s2, lnw): uint64 [n_bins] x 3 and FP64 [n_bins]."""
    rng = np.random.default_rng(seed)
    V = L * L
    nb = n_bins(model, L)
    b = np.arange(nb)
    E = 4.0 * b - 2.0 * V if model == ISING else b - 2.0 * V
    e = E / V
    acc = np.ones(nb, dtype=bool)
    if model == ISING:
        acc[[1, nb - 2]] = False                  # E = -2V + 4 and 2V - 4
    else:
        acc[[1, 2, 3, 5]] = False                 # 1, 2, 3 and 5 broken bonds
    h = V * _entropy_density(model, e)
    if mode == "flat":
        lnw = -h
    else:
        lnw = -beta_prod * E
    lnp = np.where(acc, h + lnw, -np.inf)
    prob = np.exp(lnp - lnp.max())
    prob /= prob.sum()
    n = rng.multinomial(n_records, prob).astype(np.uint64)
    mmax = V if model == ISING else (8 - 1) * V
    mbar = np.clip(-e * 0.6, 0.0, 1.0) if model == ISING else np.clip(-e - 0.5, 0.0, 1.0)
    s1 = np.zeros(nb, dtype=np.uint64)
    s2 = np.zeros(nb, dtype=np.uint64)
    idx = np.nonzero(n)[0]
    counts = n[idx].astype(np.int64)
    rec_bin = np.repeat(idx, counts)
    m = np.rint(mmax * mbar[rec_bin] + rng.normal(0.0, 0.02 * mmax, rec_bin.size))
    m = np.clip(m, 0, mmax).astype(np.uint64)
    np.add.at(s1, rec_bin, m)
    np.add.at(s2, rec_bin, m * m)
    lnw = np.where(acc, lnw - lnw[acc].max(), 0.0)
    return n, s1, s2, lnw


# reweighting cases of the configurations: (model, L, mode, production beta, beta grid,
# records = chains x production sweeps, at most 10^7)
REWEIGHT_CASES = {
    "ising_L64_p1024": (ISING, 64, "flat", None, (0.3, 0.6, 512), 10_000_000),
    "potts8_L32_p4096": (POTTS, 32, "canonical", POTTS8_BETA0, (1.2, 1.4, 1024), 10_000_000),
    "ising_L256_p8192": (ISING, 256, "canonical", ISING_BETA0, (0.3, 0.6, 4096), 8_192_000),
    "potts8_L128_p4096": (POTTS, 128, "canonical", POTTS8_BETA0, (1.2, 1.4, 4096), 4_096_000),
}
