"""Interface-tension analysis of the oracle (Sec. 5), pinned on distributions whose
equal-height temperature and peak-to-dip ratio are known in closed form."""
import math

import numpy as np
import pytest

from oracle import interface
from oracle.weights import bin_energies, n_bins

POTTS = 1


def double_gaussian(L, beta_star, a, b, s):
    """n = 1 everywhere and ln W chosen so that ln P_beta* = ln(G_a + G_b) + const:
    two equal Gaussians in the bin index at beta*."""
    nb = n_bins(POTTS, L)
    E = bin_energies(POTTS, L).astype(np.float64)
    x = np.arange(nb, dtype=np.float64)
    ln_omega = beta_star * E + np.log(np.exp(-(x - a) ** 2 / (2 * s * s)) + np.exp(-(x - b) ** 2 / (2 * s * s)))
    return -ln_omega, np.ones(nb)


@pytest.mark.parametrize("a,b,s", [(120, 360, 30.0), (200, 300, 15.0)])
def test_equal_height_of_two_gaussians(a, b, s):
    L, beta_star = 16, 1.3
    lnw, n = double_gaussian(L, beta_star, a, b, s)
    beta, ln_ratio, (b1, b2, dip) = interface.equal_height(POTTS, L, lnw, n, 1.2, 1.4, 64, 80)
    assert beta == pytest.approx(beta_star, abs=1e-10)
    assert (b1, b2, dip) == (a, b, (a + b) // 2)
    d = b - a
    # peaks: ln(1 + e^{-d^2/2s^2}); dip at the midpoint: ln(2 e^{-d^2/8s^2})
    expect = math.log1p(math.exp(-d * d / (2 * s * s))) - (math.log(2.0) - d * d / (8 * s * s))
    assert ln_ratio == pytest.approx(expect, rel=1e-9)
    assert interface.sigma_od(L, ln_ratio) == pytest.approx(expect / 32.0, rel=1e-9)


def test_invariances_and_single_peak():
    L = 16
    lnw, n = double_gaussian(L, 1.3, 150, 330, 25.0)
    r0 = interface.equal_height(POTTS, L, lnw, n, 1.2, 1.4)
    r1 = interface.equal_height(POTTS, L, lnw + 7.5, 3 * n, 1.2, 1.4)  # constants cancel
    assert r1[0] == pytest.approx(r0[0], abs=1e-12) and r1[1] == pytest.approx(r0[1], abs=1e-10)
    # a single Gaussian never changes the sign of the height difference
    nb = n_bins(POTTS, L)
    x = np.arange(nb, dtype=np.float64)
    E = bin_energies(POTTS, L).astype(np.float64)
    lnw1 = -(1.3 * E - (x - 250) ** 2 / 800.0)
    beta, ln_ratio, peaks = interface.equal_height(POTTS, L, lnw1, np.ones(nb), 1.2, 1.4)
    assert math.isnan(beta) and peaks is None


def test_energy_distribution_normalised_and_unsampled():
    L = 8
    nb = n_bins(POTTS, L)
    rng = np.random.default_rng(3)
    n = rng.integers(0, 50, nb)
    n[:10] = 0
    lnw = rng.normal(0, 2, nb)
    g = interface.energy_distribution(POTTS, L, lnw, n, 1.33)
    assert np.all(np.isneginf(g[n == 0]))
    assert np.exp(g[n > 0]).sum() == pytest.approx(1.0, abs=1e-12)
    # direct definition, bin by bin
    E = bin_energies(POTTS, L)
    k = int(np.nonzero(n > 0)[0][0])
    j = int(np.nonzero(n > 0)[0][5])
    assert g[j] - g[k] == pytest.approx(math.log(n[j] / n[k]) - (lnw[j] - lnw[k]) - 1.33 * (E[j] - E[k]),
                                        abs=1e-12)
