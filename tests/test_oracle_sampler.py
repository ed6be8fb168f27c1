"""The oracle's Markov chains: invariants and stationary distributions.

Pins: histogram mass = sweeps * V per chain; running E/M = recount (checked inside
the C code every sweep); with ln W = -beta E the sampled energy distribution is the
exact canonical one Omega(E) exp(-beta E) / Z (enumeration / transfer matrix); with
ln W = -ln Omega it is flat (the multicanonical goal of Eq. 1); subsets of chains
replay exactly; iteration/sweep/phase counters change the stream.
"""
import numpy as np
import pytest

import exact
from oracle import sampler, weights

ISING, POTTS = 0, 1


def _run(model, L, q, lnw, n_chains, n_sweeps, seed=7, phase=1, iteration=0):
    thr = weights.thresholds(model, L, lnw)
    spins, E, M = sampler.init_chains(model, L, q, seed, 0, n_chains)
    # burn-in
    sampler.run_sweeps(model, L, q, seed, 2, 0, 0, 200, 0, spins, E, M, thr)
    H, _, _ = sampler.run_sweeps(model, L, q, seed, phase, iteration, 0, n_sweeps, 0,
                                 spins, E, M, thr, per_chain_hist=True)
    return H


def _zscores(H, expected_p, acc):
    """Per-bin z of the pooled fraction, with the error from the spread over the
    independent chains."""
    frac = H / H.sum(axis=1, keepdims=True)
    mean = frac.mean(axis=0)
    err = frac.std(axis=0, ddof=1) / np.sqrt(H.shape[0])
    # floor: the binomial error of the pooled count (chains that never visit a rare
    # bin give no spread)
    n_tot = H.sum()
    err = np.maximum(err, np.sqrt(expected_p * (1 - expected_p) / n_tot) + 1.0 / n_tot)
    z = []
    for b in range(H.shape[1]):
        if not acc[b]:
            assert mean[b] == 0
            continue
        z.append((mean[b] - expected_p[b]) / err[b])
    return np.array(z)


def test_histogram_mass():
    L, n_chains, n_sweeps = 6, 5, 37
    thr = weights.thresholds(ISING, L, np.zeros(L * L + 1))
    spins, E, M = sampler.init_chains(ISING, L, 2, 3, 0, n_chains)
    H, _, _ = sampler.run_sweeps(ISING, L, 2, 3, 1, 0, 0, n_sweeps, 0, spins, E, M, thr,
                                 per_chain_hist=True)
    assert np.all(H.sum(axis=1) == n_sweeps * L * L)


def test_zero_weights_ising_flips_everything():
    """ln W = 0: every move is accepted (W(E')/W(E) = 1), so one Ising sweep flips
    every spin exactly once."""
    L = 4
    thr = weights.thresholds(ISING, L, np.zeros(L * L + 1))
    spins, E, M = sampler.init_chains(ISING, L, 2, 11, 0, 3)
    s0 = spins.copy()
    sampler.run_sweeps(ISING, L, 2, 11, 1, 0, 0, 1, 0, spins, E, M, thr)
    assert np.array_equal(spins, -s0)


@pytest.mark.parametrize("beta", [0.25, 0.45])
def test_canonical_ising_4x4(beta):
    L, V = 4, 16
    om = np.array(exact.enumerate_dos(ISING, L, 2), dtype=np.float64)
    Eb = weights.bin_energies(ISING, L)
    lnw = -beta * Eb.astype(np.float64)
    p = om * np.exp(-beta * Eb - (-beta * Eb).max())
    p /= p.sum()
    H = _run(ISING, L, 2, lnw, 48, 3000)
    z = _zscores(H.astype(np.float64), p, weights.accessible(ISING, L))
    assert np.all(np.abs(z) < 5), z


def test_flat_with_exact_weights_ising_8x8(ising8_dos):
    L = 8
    om = np.array([float(w) for w in ising8_dos])
    acc = weights.accessible(ISING, L)
    lnw = np.zeros(len(om))
    lnw[acc] = -np.log(om[acc])
    lnw -= lnw[acc].max()
    lnw[~acc] = 0.0
    H = _run(ISING, L, 2, lnw, 64, 3000)
    K = acc.sum()
    p = np.where(acc, 1.0 / K, 0.0)
    z = _zscores(H.astype(np.float64), p, acc)
    assert np.all(np.abs(z) < 5), z


def test_flat_with_exact_weights_potts_3x3(potts3_q8_dos):
    L = 3
    om = np.array([float(w) for w in potts3_q8_dos])
    acc = weights.accessible(POTTS, L)
    lnw = np.zeros(len(om))
    lnw[acc] = -np.log(om[acc])
    lnw -= lnw[acc].max()
    lnw[~acc] = 0.0
    H = _run(POTTS, L, 8, lnw, 48, 4000)
    p = np.where(acc, 1.0 / acc.sum(), 0.0)
    z = _zscores(H.astype(np.float64), p, acc)
    assert np.all(np.abs(z) < 5), z


def test_canonical_potts_3x3(potts3_q8_dos):
    L, beta = 3, 1.0
    om = np.array([float(w) for w in potts3_q8_dos])
    Eb = weights.bin_energies(POTTS, L).astype(np.float64)
    lnw = -beta * Eb
    a = np.log(np.where(om > 0, om, 1.0)) - beta * Eb
    p = np.where(om > 0, np.exp(a - a[om > 0].max()), 0.0)
    p /= p.sum()
    H = _run(POTTS, L, 8, lnw, 48, 4000)
    z = _zscores(H.astype(np.float64), p, weights.accessible(POTTS, L))
    assert np.all(np.abs(z) < 5), z


@pytest.mark.parametrize("model,L,q", [(ISING, 8, 2), (POTTS, 6, 8)])
def test_subset_replay_and_counters(model, L, q):
    seed = 5
    rng = np.random.default_rng(0)
    nb = weights.n_bins(model, L)
    lnw = -0.3 * weights.bin_energies(model, L).astype(np.float64) * (1 if model == ISING else 3)
    lnw += rng.normal(0, 0.1, nb)
    thr = weights.thresholds(model, L, lnw)
    spins, E, M = sampler.init_chains(model, L, q, seed, 0, 6)
    H_all, er, mr = sampler.run_sweeps(model, L, q, seed, 3, 0, 10, 20, 0, spins, E, M,
                                       thr, per_chain_hist=True, record=True)
    s4, E4, M4 = sampler.init_chains(model, L, q, seed, 4, 1)
    H4, er4, mr4 = sampler.run_sweeps(model, L, q, seed, 3, 0, 10, 20, 4, s4, E4, M4, thr,
                                      per_chain_hist=True, record=True)
    assert np.array_equal(H4[0], H_all[4])
    assert np.array_equal(er4[:, 0], er[:, 4]) and np.array_equal(mr4[:, 0], mr[:, 4])
    assert np.array_equal(s4[0], spins[4])
    # running the 20 sweeps as 10 + 10 with the sweep counter continuing is identical
    s5, E5, M5 = sampler.init_chains(model, L, q, seed, 4, 1)
    sampler.run_sweeps(model, L, q, seed, 3, 0, 10, 10, 4, s5, E5, M5, thr)
    sampler.run_sweeps(model, L, q, seed, 3, 0, 20, 10, 4, s5, E5, M5, thr)
    assert np.array_equal(s5[0], s4[0])
    # other phase / iteration / sweep offset -> a different trajectory
    for args in ((2, 0, 10), (3, 1, 10), (3, 0, 11)):
        s6, E6, M6 = sampler.init_chains(model, L, q, seed, 4, 1)
        sampler.run_sweeps(model, L, q, seed, args[0], args[1], args[2], 20, 4, s6, E6, M6,
                           thr)
        assert not np.array_equal(s6[0], s4[0])
