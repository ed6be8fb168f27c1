"""Reweighted energy distribution and interface tension (Sec. 5) on the GPU against the
oracle: the same MUCA run on both sides (iterations, then production), then the
distributions and the equal-height analysis each from its own data."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POTTS = 1


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


def run_both(muca, L, p, seed, iters, sweeps, prod):
    from oracle import MucaOracle
    o = MucaOracle(POTTS, L, 8, p, seed)
    for _ in range(iters):
        o.iterate(sweeps)
        o.update_weights()
    E_rec, M_rec = o.produce(prod)
    g = muca.Muca(POTTS, L, 8, p, seed)
    for _ in range(iters):
        g.iterate(sweeps)
        g.update_weights()
    g.produce(prod)
    return o, E_rec, M_rec, g


def test_distribution_and_interface_tension_equal_oracle(muca):
    from oracle import interface, reweight
    L, p = 8, 16
    o, E_rec, M_rec, g = run_both(muca, L, p, 41, 12, 300, 400)
    try:
        assert np.array_equal(g.get_lnw(), o.lnw)
        n, _, _ = reweight.bin_series(POTTS, L, E_rec, M_rec)
        betas = np.array([1.2, 1.3, 1.3425, 1.4])
        lnP = g.energy_distribution(betas)
        for k, beta in enumerate(betas):
            ref = interface.energy_distribution(POTTS, L, o.lnw, n, beta)
            fin = np.isfinite(ref)
            assert np.array_equal(fin, np.isfinite(lnP[k]))
            assert np.max(np.abs(lnP[k][fin] - ref[fin])) < 1e-11
        beta_o, ratio_o, peaks_o = interface.equal_height(POTTS, L, o.lnw, n, 1.2, 1.5)
        beta_g, ratio_g, peaks_g, sigma_g = g.interface_tension(1.2, 1.5)
        assert math.isfinite(beta_o) and ratio_o > 0
        assert beta_g == pytest.approx(beta_o, abs=1e-9)
        assert ratio_g == pytest.approx(ratio_o, abs=1e-8)
        assert peaks_g == tuple(peaks_o)
        assert sigma_g == pytest.approx(interface.sigma_od(L, ratio_o), abs=1e-9)
    finally:
        g.close()


def test_interface_tension_without_two_peaks(muca):
    # a short canonical run far from the transition: one peak, no equal-height beta
    with muca.Muca(POTTS, 8, 8, 8, 5) as g:
        g.produce(20)
        beta, ratio, peaks, sigma = g.interface_tension(2.0, 2.2, 16, 10)
        assert math.isnan(beta) and math.isnan(ratio) and peaks == (-1, -1, -1)


def test_energy_distribution_needs_production(muca):
    with muca.Muca(POTTS, 4, 8, 4, 1) as g:
        with pytest.raises(muca.MucaError):
            g.energy_distribution([1.3])
