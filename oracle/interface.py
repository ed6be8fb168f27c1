"""Order-disorder interface tension of the 8-state Potts model (Sec. 5), FP64 numpy.

TEST INFRASTRUCTURE ONLY.

Sec. 5 estimates sigma_od from the reweighted energy histogram at the temperature
where its two peaks (ordered, low energy; disordered, high energy) are equally high:
sigma_od(L) = ln(P_max / P_min) / (2 L), P_min being the minimum between the peaks;
the paper's value is the L -> infinity limit of this.

Readings (the paper gives no procedure):
  * P_beta(E) ~ n(E) W(E)^-1 exp(-beta E) over the sampled bins (Eq. 2 applied to the
    energy histogram itself), normalised to sum 1; ln P is used throughout.
  * The two peaks at a given beta: split the sampled bins at s, take the highest bin on
    each side (lowest index on ties), move s to the lowest bin between the two peaks
    (lowest index on ties) and repeat until s no longer changes (at most 64 rounds); the
    first split is the midpoint of the sampled range.  They count as two peaks only if
    the dip lies strictly between them and strictly below both; otherwise (one peak)
    the height difference is undefined (nan).
  * beta_eqh solves h(beta) = ln P(peak_low) - ln P(peak_high) = 0.  h grows with beta
    (a larger beta favours low energies); it is bracketed on a uniform grid of n_grid
    betas over [beta_lo, beta_hi] (the first sign change from negative to positive)
    and refined by n_bisect bisection steps.
  * ln(P_max / P_min) is evaluated at beta_eqh as the mean of the two peak heights
    minus the minimum between them.
"""
import numpy as np

from .weights import bin_energies


def energy_distribution(model, L, lnw, n, beta):
    """ln P_beta(E_b) for every bin (-inf where n = 0), normalised: Eq. 2 applied to
    the energy histogram of a production run with weights lnw and counts n."""
    E = bin_energies(model, L).astype(np.float64)
    n = np.asarray(n, dtype=np.float64)
    g = np.full(len(n), -np.inf)
    s = n > 0
    g[s] = np.log(n[s]) - np.asarray(lnw, dtype=np.float64)[s] - beta * E[s]
    m = g[s].max()
    return g - (m + np.log(np.exp(g[s] - m).sum()))


def two_peaks(g):
    """(low peak, high peak, dip) bin indices of ln P g by the iterated split."""
    idx = np.nonzero(np.isfinite(g))[0]
    lo, hi = int(idx[0]), int(idx[-1])
    s = (lo + hi) // 2
    b1 = b2 = dip = s
    for _ in range(64):
        left = g[lo:s + 1]
        right = g[s + 1:hi + 1]
        if len(right) == 0 or not np.isfinite(right).any() or not np.isfinite(left).any():
            break
        b1 = lo + int(np.argmax(left))
        b2 = s + 1 + int(np.argmax(right))
        seg = g[b1:b2 + 1]
        seg = np.where(np.isfinite(seg), seg, np.inf)
        dip = b1 + int(np.argmin(seg))
        if dip == s:
            break
        s = dip
    return b1, b2, dip


def height_difference(model, L, lnw, n, beta):
    g = energy_distribution(model, L, lnw, n, beta)
    b1, b2, dip = two_peaks(g)
    if not (b1 < dip < b2 and g[dip] < g[b1] and g[dip] < g[b2]):
        return float("nan"), g, (b1, b2, dip)
    return g[b1] - g[b2], g, (b1, b2, dip)


def equal_height(model, L, lnw, n, beta_lo, beta_hi, n_grid=64, n_bisect=60):
    """beta_eqh and ln(P_max / P_min) there.  Returns (beta_eqh, ln ratio, (b1, b2, dip))
    or (nan, nan, None) when h(beta) does not change sign on the grid."""
    betas = np.linspace(beta_lo, beta_hi, n_grid)
    hs = [height_difference(model, L, lnw, n, b)[0] for b in betas]
    k = None
    for i in range(n_grid - 1):
        if hs[i] < 0.0 <= hs[i + 1]:  # False for nan
            k = i
            break
    if k is None:
        return float("nan"), float("nan"), None
    a, b = betas[k], betas[k + 1]
    for _ in range(n_bisect):
        mid = 0.5 * (a + b)
        h = height_difference(model, L, lnw, n, mid)[0]
        if h != h:
            return float("nan"), float("nan"), None
        if h < 0.0:
            a = mid
        else:
            b = mid
    beta = 0.5 * (a + b)
    h, g, (b1, b2, dip) = height_difference(model, L, lnw, n, beta)
    if h != h:
        return float("nan"), float("nan"), None
    return float(beta), float(0.5 * (g[b1] + g[b2]) - g[dip]), (b1, b2, dip)


def sigma_od(L, ln_ratio):
    """sigma_od(L) = ln(P_max / P_min) / (2 L) (Sec. 5)."""
    return ln_ratio / (2.0 * L)
