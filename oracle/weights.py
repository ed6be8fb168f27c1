"""Weights side of the oracle: bins, acceptance thresholds, the recursive ln W update.

TEST INFRASTRUCTURE ONLY (plain Python loops in FP64, written to be read against the
paper, not to be fast).

Paper passages followed:
  * Sec. 2, Eq. 1: multicanonical weights W(E); a move E -> E' is accepted with
    probability min(1, W(E')/W(E)).
  * Sec. 2: simple recursion W^(n+1)(E) = W^(n)(E) / H^(n)(E); the accumulated form
    that uses "the full statistics of previous iterations" (Berg's error-weighted
    recursion, cited there as Janke 1998); logarithmic weights throughout.
  * Sec. 2, Parallel Version: H^(n)(E) = sum_i H_i^(n)(E) feeds the update.
  * Sec. 3: after each estimate a correction linearly extrapolates ln W beyond the
    sampled region "with a range of L bins"; convergence = full range covered and
    every entry within [1/2, 2] of the mean.

Readings (the paper is silent): only accessible bins take part; inaccessible bins
carry ln W = 0 and are never entered; the additive constant is fixed by
max_{accessible} ln W = 0.
"""
import math
import numpy as np

ISING, POTTS = 0, 1
ALWAYS = 0xFFFFFFFF


def n_bins(model, L):
    V = L * L
    return V + 1 if model == ISING else 2 * V + 1


def n_de(model):
    return 4 if model == ISING else 8


def bin_energies(model, L):
    """Energy of every bin: Ising E = 4b - 2V, Potts E = b - 2V."""
    V = L * L
    b = np.arange(n_bins(model, L), dtype=np.int64)
    return 4 * b - 2 * V if model == ISING else b - 2 * V


def bin_deltas(model):
    """Bin offset of each threshold-table column (ascending dE, dE != 0)."""
    return [-2, -1, 1, 2] if model == ISING else [-4, -3, -2, -1, 1, 2, 3, 4]


def accessible(model, L):
    """Accessible energy bins of the periodic L x L lattice (L >= 3, even L for Ising).

    Ising: E = -2V + 4 and E = 2V - 4 cannot occur (the smallest excitation of a
    uniform or a staggered state changes 4 bonds).  Potts: with 1, 2, 3 or 5 broken
    bonds no configuration exists (a single differing spin breaks 4, two adjacent
    ones 6 or 7).  The tests confirm the rule by full enumeration at small L.
    """
    nb = n_bins(model, L)
    acc = np.ones(nb, dtype=bool)
    if model == ISING:
        acc[1] = False
        acc[nb - 2] = False
    else:
        for k in (1, 2, 3, 5):
            if k < nb:
                acc[k] = False
    return acc


def thresholds(model, L, lnw, acc=None):
    """Integer acceptance thresholds for every (current bin, dE) pair.

    d = lnW[b'] - lnW[b] in FP64; A = 0xFFFFFFFF if d >= 0, else
    A = min(floor(2^32 * exp(d)), 0xFFFFFFFF); A = 0 where b' is outside the range or
    inaccessible.  A move is accepted iff A == 0xFFFFFFFF or u < A for a raw 32-bit
    draw u, i.e. with probability A / 2^32 ~ min(1, W(E')/W(E)) (Eq. 1).
    """
    if acc is None:
        acc = accessible(model, L)
    nb = n_bins(model, L)
    deltas = bin_deltas(model)
    out = np.zeros((nb, len(deltas)), dtype=np.uint32)
    for b in range(nb):
        if not acc[b]:
            continue
        for j, dlt in enumerate(deltas):
            bp = b + dlt
            if bp < 0 or bp >= nb or not acc[bp]:
                continue
            d = float(lnw[bp]) - float(lnw[b])
            if d >= 0.0:
                A = ALWAYS
            else:
                A = min(math.floor(math.ldexp(math.exp(d), 32)), ALWAYS)
            out[b, j] = A
    return out


def thresholds_muma(L, lnw, beta):
    """Thresholds of the multimagnetic Ising chain (weights W(M) at inverse temperature
    beta): for M bin b = (M + V)/2 and column 5 (s == +1) + n, with n unequal
    neighbours of the flipped spin s: b' = b - s, dE = 8 - 4n,
    d = (lnW[b'] - lnW[b]) - beta dE in FP64; A as in `thresholds`; 0 for b' outside
    the range."""
    nb = L * L + 1
    out = np.zeros((nb, 10), dtype=np.uint32)
    for b in range(nb):
        for col in range(10):
            s = 1 if col >= 5 else -1
            n = col - 5 if col >= 5 else col
            bp = b - s
            if bp < 0 or bp >= nb:
                continue
            d = (float(lnw[bp]) - float(lnw[b])) - beta * float(8 - 4 * n)
            if d >= 0.0:
                A = ALWAYS
            else:
                A = min(math.floor(math.ldexp(math.exp(d), 32)), ALWAYS)
            out[b, col] = A
    return out


def iteration_stats(model, L, H, acc=None):
    """Convergence statistics of one merged histogram (Sec. 3), over accessible bins.

    covered: every accessible bin has H > 0; flat: 0.5*mean <= H[b] <= 2*mean for all
    accessible b; lo/hi: lowest/highest accessible bin with H > 0 (-1 if none)."""
    if acc is None:
        acc = accessible(model, L)
    idx = [b for b in range(len(H)) if acc[b]]
    vals = [int(H[b]) for b in idx]
    total = sum(vals)
    K = len(idx)
    mean = total / K
    sampled = [b for b in idx if H[b] > 0]
    covered = len(sampled) == K
    mn, mx = min(vals), max(vals)
    flat = covered and all(0.5 * mean <= v <= 2.0 * mean for v in vals)
    return {
        "covered": covered,
        "flat": flat,
        "converged": covered and flat,
        "lo": sampled[0] if sampled else -1,
        "hi": sampled[-1] if sampled else -1,
        "n_sampled": len(sampled),
        "min_over_mean": mn / mean if mean > 0 else 0.0,
        "max_over_mean": mx / mean if mean > 0 else 0.0,
        "total": total,
    }


def update_weights(model, L, lnw, H, P, accumulated=True, correction_width=None,
                   acc=None):
    """One weight iteration: recursion, boundary correction, normalisation.

    lnw: FP64 [n_bins] current ln W^(n).  H: merged histogram of iteration n.
    P:   FP64 [n_bins] accumulator of the accumulated recursion, indexed by the lower
         bin of each adjacent accessible pair; updated in place.
    Returns (lnw_new, stats) with stats computed on H before the update.

    Accumulated recursion, for adjacent accessible bins u < v (ln form):
        if H[u] > 0 and H[v] > 0:
            g0 = H[u] H[v] / (H[u] + H[v]);  P[u] += g0;  g = g0 / P[u]
            d  = (lnW[v] - lnW[u]) - g * (ln H[v] - ln H[u])
        else:
            d  =  lnW[v] - lnW[u]
        lnW'[a_0] = 0,  lnW'[a_(j+1)] = lnW'[a_j] + d_j   (ascending j).
    Simple recursion (accumulated=False): lnW'[b] = lnW[b] - ln H[b] where H[b] > 0.
    In the first iteration P = g0, so g = 1 and both forms give the same differences.
    """
    if acc is None:
        acc = accessible(model, L)
    if correction_width is None:
        correction_width = L
    stats = iteration_stats(model, L, H, acc)
    nb = len(lnw)
    a = [b for b in range(nb) if acc[b]]
    new = [0.0] * nb
    if accumulated:
        new[a[0]] = 0.0
        for j in range(len(a) - 1):
            u, v = a[j], a[j + 1]
            d = float(lnw[v]) - float(lnw[u])
            if H[u] > 0 and H[v] > 0:
                hu, hv = float(H[u]), float(H[v])
                g0 = hu * hv / (hu + hv)
                P[u] = P[u] + g0
                g = g0 / P[u]
                d = d - g * (math.log(hv) - math.log(hu))
            new[v] = new[u] + d
    else:
        for b in a:
            new[b] = float(lnw[b])
            if H[b] > 0:
                new[b] = new[b] - math.log(float(H[b]))

    # Boundary correction (Sec. 3): extend ln W linearly beyond the sampled range,
    # with the slope taken over (up to) L bins inside each edge.
    lo, hi = stats["lo"], stats["hi"]
    if lo >= 0 and hi > lo:
        width = min(correction_width, hi - lo)
        b2 = next(b for b in a if b >= lo + width)
        slope = (new[b2] - new[lo]) / float(b2 - lo)
        for b in a:
            if b < lo:
                new[b] = new[lo] + slope * float(b - lo)
        b1 = max(b for b in a if b <= hi - width)
        slope = (new[hi] - new[b1]) / float(hi - b1)
        for b in a:
            if b > hi:
                new[b] = new[hi] + slope * float(b - hi)

    # Fix the additive constant: max over accessible bins is 0.
    top = max(new[b] for b in a)
    out = np.zeros(nb, dtype=np.float64)
    for b in a:
        out[b] = new[b] - top
    return out, stats
