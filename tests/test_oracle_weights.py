"""Thresholds and the recursive weight update of the oracle.

Pins (none of them retypes the oracle's formulas):
  * thresholds equal floor(2^32 min(1, W'/W)) evaluated with 50-digit mpmath;
  * a flat histogram leaves ln W unchanged (both recursions);
  * the first accumulated step equals the simple step (g = 1 when P starts at 0);
  * the accumulated recursion equals the error-weighted average of the per-iteration
    estimates  d lnOmega = d ln H_k - d ln W_k  with weights g0_k (closed form of Berg's
    recursion, checked over many random iterations);
  * a perfect histogram H ~ Omega W gives ln W = -ln Omega in one step;
  * the boundary correction is linear outside the sampled range, continuous at its
    edges, with the slope of the innermost L bins;
  * the convergence test follows Sec. 3 on constructed histograms.
"""
import math

import mpmath as mp
import numpy as np
import pytest

from oracle import weights

ISING, POTTS = 0, 1


@pytest.mark.parametrize("model,L", [(ISING, 8), (POTTS, 6)])
def test_thresholds_match_high_precision(model, L):
    rng = np.random.default_rng(3)
    nb = weights.n_bins(model, L)
    lnw = rng.normal(0, 3, nb)
    acc = weights.accessible(model, L)
    thr = weights.thresholds(model, L, lnw, acc)
    deltas = weights.bin_deltas(model)
    with mp.workdps(50):
        for b in range(nb):
            for j, d in enumerate(deltas):
                bp = b + d
                if not acc[b] or bp < 0 or bp >= nb or not acc[bp]:
                    assert thr[b, j] == 0
                    continue
                x = mp.mpf(float(lnw[bp])) - mp.mpf(float(lnw[b]))
                if x >= 0:
                    assert thr[b, j] == 0xFFFFFFFF
                else:
                    exact_val = mp.floor(mp.ldexp(mp.exp(x), 32))
                    # libm exp is within an ulp; the floor can differ only on a knife edge
                    assert abs(int(thr[b, j]) - int(exact_val)) <= 1
                    frac = mp.ldexp(mp.exp(x), 32) - exact_val
                    if 1e-6 < frac < 1 - 1e-6:
                        assert int(thr[b, j]) == int(exact_val)


def test_flat_histogram_is_a_fixed_point():
    L = 8
    nb = weights.n_bins(ISING, L)
    acc = weights.accessible(ISING, L)
    rng = np.random.default_rng(1)
    lnw = np.where(acc, rng.normal(0, 1, nb), 0.0)
    lnw -= lnw[acc].max()
    lnw[~acc] = 0
    H = np.where(acc, 1000, 0).astype(np.uint64)
    for accumulated in (True, False):
        P = np.zeros(nb)
        new, st = weights.update_weights(ISING, L, lnw, H, P, accumulated=accumulated)
        assert st["converged"]
        assert np.allclose(new[acc], lnw[acc], atol=1e-12)


def test_first_accumulated_step_equals_simple_step():
    L = 8
    nb = weights.n_bins(ISING, L)
    acc = weights.accessible(ISING, L)
    rng = np.random.default_rng(2)
    lnw = np.where(acc, rng.normal(0, 1, nb), 0.0)
    H = np.where(acc, rng.integers(1, 10 ** 6, nb), 0).astype(np.uint64)
    a, _ = weights.update_weights(ISING, L, lnw, H, np.zeros(nb), accumulated=True)
    s, _ = weights.update_weights(ISING, L, lnw, H, np.zeros(nb), accumulated=False)
    assert np.allclose(a[acc], s[acc], atol=1e-11)


def test_accumulated_recursion_is_weighted_average():
    """After n steps, -[lnW(v) - lnW(u)] = sum_k g0_k e_k / sum_k g0_k with
    e_k = [ln H_k(v) - ln H_k(u)] - [ln W_k(v) - ln W_k(u)]  (Berg / Janke 1998)."""
    L = 4
    nb = weights.n_bins(ISING, L)
    acc = weights.accessible(ISING, L)
    a = [b for b in range(nb) if acc[b]]
    rng = np.random.default_rng(4)
    lnw = np.zeros(nb)
    P = np.zeros(nb)
    num = np.zeros(nb)
    den = np.zeros(nb)
    for it in range(12):
        H = np.where(acc, rng.integers(1, 10 ** 5, nb), 0).astype(np.uint64)
        for u, v in zip(a[:-1], a[1:]):
            hu, hv = float(H[u]), float(H[v])
            g0 = hu * hv / (hu + hv)
            e = (math.log(hv) - math.log(hu)) - (lnw[v] - lnw[u])
            num[u] += g0 * e
            den[u] += g0
        lnw, _ = weights.update_weights(ISING, L, lnw, H, P, accumulated=True)
        for u, v in zip(a[:-1], a[1:]):
            assert -(lnw[v] - lnw[u]) == pytest.approx(num[u] / den[u], rel=1e-10, abs=1e-10)


def test_perfect_histogram_recovers_dos():
    L = 4
    nb = weights.n_bins(ISING, L)
    acc = weights.accessible(ISING, L)
    # a fake density of states and weights; H = Omega * W exactly representable
    lnomega = np.where(acc, np.log(np.arange(1, nb + 1) ** 2.0), 0.0)
    lnw = np.where(acc, -0.5 * lnomega, 0.0)
    H = np.where(acc, np.round(np.exp(lnomega + lnw)), 0).astype(np.uint64)
    new, _ = weights.update_weights(ISING, L, lnw, H, np.zeros(nb), accumulated=False)
    target = -(np.log(H[acc].astype(float)) - lnw[acc])
    assert np.allclose(new[acc] - new[acc].max(), target - target.max(), atol=1e-12)


def test_boundary_correction_linear_extension():
    L = 8
    model = POTTS
    nb = weights.n_bins(model, L)
    acc = weights.accessible(model, L)
    rng = np.random.default_rng(5)
    lo, hi = 40, 90
    H = np.zeros(nb, dtype=np.uint64)
    for b in range(lo, hi + 1):
        if acc[b]:
            H[b] = rng.integers(100, 1000)
    lnw = np.where(acc, rng.normal(0, 1, nb), 0.0)
    new, st = weights.update_weights(model, L, lnw, H, np.zeros(nb))
    assert (st["lo"], st["hi"]) == (lo, hi) and not st["covered"]
    below = [b for b in range(nb) if acc[b] and b <= lo]
    above = [b for b in range(nb) if acc[b] and b >= hi]
    sl_lo = (new[lo + L] - new[lo]) / L
    sl_hi = (new[hi] - new[hi - L]) / L
    for b in below:
        assert new[b] == pytest.approx(new[lo] + sl_lo * (b - lo), abs=1e-9)
    for b in above:
        assert new[b] == pytest.approx(new[hi] + sl_hi * (b - hi), abs=1e-9)
    assert new[acc].max() == 0.0
    assert np.all(new[~acc] == 0.0)


def test_convergence_criterion():
    L = 4
    nb = weights.n_bins(ISING, L)
    acc = weights.accessible(ISING, L)
    H = np.where(acc, 100, 0).astype(np.uint64)
    assert weights.iteration_stats(ISING, L, H)["converged"]
    H2 = H.copy()
    H2[4] = 40                         # below half the mean (~96)
    st = weights.iteration_stats(ISING, L, H2)
    assert st["covered"] and not st["flat"]
    H3 = H.copy()
    H3[4] = 0                          # a hole
    assert not weights.iteration_stats(ISING, L, H3)["covered"]
    H4 = H.copy()
    H4[1] = 0                          # inaccessible bins do not count
    assert weights.iteration_stats(ISING, L, H4)["converged"]
