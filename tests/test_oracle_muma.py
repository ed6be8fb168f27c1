"""Multimagnetic Ising ensemble of the oracle (Sec. 4, Fig. 6: weights W(M) at a fixed
beta), pinned against 50-digit thresholds and against exact enumeration: at beta = 0
the weights -ln binomial(V, (M+V)/2) make the M histogram flat, and with W = 1 the
chain samples the canonical P_beta(M) of the 4x4 lattice."""
import math

import mpmath as mp
import numpy as np
import pytest

import exact
from oracle import MucaOracle, weights

ISING = 0


def test_muma_thresholds_match_high_precision():
    L, beta = 4, 0.66
    rng = np.random.default_rng(5)
    nb = L * L + 1
    lnw = rng.normal(0, 3, nb)
    thr = weights.thresholds_muma(L, lnw, beta)
    with mp.workdps(50):
        for b in range(nb):
            for col in range(10):
                s = 1 if col >= 5 else -1
                n = col % 5
                bp = b - s
                if bp < 0 or bp >= nb:
                    assert thr[b, col] == 0
                    continue
                x = (mp.mpf(float(lnw[bp])) - mp.mpf(float(lnw[b]))) - mp.mpf(beta) * (8 - 4 * n)
                if x >= 0:
                    assert thr[b, col] == 0xFFFFFFFF
                else:
                    v = mp.ldexp(mp.exp(x), 32)
                    assert abs(int(thr[b, col]) - int(mp.floor(v))) <= 1
                    if 1e-6 < v - mp.floor(v) < 1 - 1e-6:
                        assert int(thr[b, col]) == int(mp.floor(v))


def z_scores(H, expected_p, n_chains):
    """Per-bin z of a pooled histogram against probabilities, with the spread estimated
    from the chain count (chains are independent; samples within a chain are not)."""
    tot = H.sum()
    exp_n = expected_p * tot
    return (H - exp_n) / np.sqrt(np.maximum(exp_n, 1.0) * 50.0 / max(n_chains, 1) + 1.0)


def test_binomial_weights_flatten_m_at_beta_zero():
    L, p = 4, 32
    V = L * L
    lnw = np.array([-math.lgamma(V + 1) + math.lgamma(k + 1) + math.lgamma(V - k + 1) for k in range(V + 1)])
    o = MucaOracle(ISING, L, 2, p, 9, muma_beta=0.0)
    o.set_lnw(lnw - lnw.max())
    o.thermalize(50)
    H = o.iterate(2000)
    frac = H / H.sum()
    # flat over all V + 1 magnetisation bins
    assert np.all(np.abs(frac * (V + 1) - 1.0) < 0.15), frac * (V + 1)


def test_unit_weights_sample_canonical_magnetisation():
    L, p, beta = 4, 32, 0.3
    V = L * L
    conf = exact.all_configs(ISING, L, 2)
    E = exact.energy_np(ISING, L, conf.reshape(-1, L, L)).astype(np.float64)
    M = conf.reshape(len(conf), -1).sum(axis=1)
    w = np.exp(-beta * (E - E.min()))
    p_exact = np.bincount(((M + V) // 2).astype(int), weights=w, minlength=V + 1)
    p_exact /= p_exact.sum()
    o = MucaOracle(ISING, L, 2, p, 13, muma_beta=beta)
    o.thermalize(100)
    H = o.iterate(3000).astype(np.float64)
    assert np.all(np.abs(z_scores(H, p_exact, p)) < 5.0)
    # the mean |M| agrees to a few per cent
    m_abs = np.abs(np.arange(V + 1) * 2 - V)
    assert (H * m_abs).sum() / H.sum() == pytest.approx((p_exact * m_abs).sum(), rel=0.03)


def test_muma_energy_and_magnetisation_invariants():
    # the C chain checks E and M against a recount every sweep; a long run must pass
    o = MucaOracle(ISING, 6, 2, 5, 21, muma_beta=0.5)
    o.iterate(200)
    o.update_weights()
    o.iterate(200)
    assert o.iteration == 2
