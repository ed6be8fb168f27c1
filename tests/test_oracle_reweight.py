"""Eq. 2 reweighting of the oracle against exact canonical results.

Pins: binned form = series form (1e-12); with n(E) = Omega(E) and ln W = 0 the
binned reweighting gives the exact canonical e and C (Kaufman, 4x4 and 8x8); with the
exact per-energy magnetisation sums it gives <|m|> and chi of full enumeration
(Ising 4x4, Potts 3x3 q = 3); MUCA records with ln W = -beta' E reweight to the same
canonical curves within statistics.
"""
import numpy as np
import pytest

import exact
from oracle import reweight, sampler, weights

ISING, POTTS = 0, 1


def test_binned_equals_series():
    L, q = 6, 8
    lnw = -1.2 * weights.bin_energies(POTTS, L).astype(np.float64)
    thr = weights.thresholds(POTTS, L, lnw)
    spins, E, M = sampler.init_chains(POTTS, L, q, 9, 0, 8)
    _, er, mr = sampler.run_sweeps(POTTS, L, q, 9, 3, 0, 0, 400, 0, spins, E, M, thr,
                                   record=True)
    betas = np.linspace(1.0, 1.5, 7)
    a = reweight.reweight_series(POTTS, L, q, lnw, er, mr, betas)
    n, s1, s2 = reweight.bin_series(POTTS, L, er, mr)
    assert int(n.sum()) == er.size
    b = reweight.reweight_binned(POTTS, L, q, lnw, n, s1, s2, betas)
    for k in a:
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-14), k


@pytest.mark.parametrize("L", [4, 8])
def test_canonical_from_exact_dos_matches_kaufman(L, ising8_dos):
    om = exact.enumerate_dos(ISING, 4, 2) if L == 4 else ising8_dos
    betas = np.array([0.3, 0.4, 0.4406867935097715, 0.5, 0.6])
    e, C = reweight.canonical_from_dos(ISING, L, [float(w) for w in om], betas)
    for j, beta in enumerate(betas):
        ee, cc = exact.kaufman_e_c(L, beta)
        assert e[j] == pytest.approx(ee, rel=1e-10)
        assert C[j] == pytest.approx(cc, rel=1e-10)


@pytest.mark.parametrize("model,L,q", [(ISING, 4, 2), (POTTS, 3, 3)])
def test_magnetisation_observables_match_enumeration(model, L, q):
    conf = exact.all_configs(model, L, q)
    E = exact.energy_np(model, L, conf.reshape(-1, L, L))
    M = exact.magnetization_np(model, q, conf)
    n, s1, s2 = reweight.bin_series(model, L, E, M)
    nb = weights.n_bins(model, L)
    for beta in (0.2, 0.44, 0.9):
        r = reweight.reweight_binned(model, L, q, np.zeros(nb), n, s1, s2, [beta])
        ee, cc, am, chi = exact.enumerate_joint(model, L, q, beta)
        assert r["e"][0] == pytest.approx(ee, rel=1e-12)
        assert r["C"][0] == pytest.approx(cc, rel=1e-10)
        assert r["absm"][0] == pytest.approx(am, rel=1e-12)
        assert r["chi"][0] == pytest.approx(chi, rel=1e-9)


def test_muca_like_records_reweight_to_canonical(ising8_dos):
    """Records sampled with weights W = exp(-0.42 E) reweight (Eq. 2) to the exact
    canonical e(beta) of the 8x8 lattice at nearby beta."""
    L = 8
    lnw = -0.42 * weights.bin_energies(ISING, L).astype(np.float64)
    thr = weights.thresholds(ISING, L, lnw)
    spins, E, M = sampler.init_chains(ISING, L, 2, 21, 0, 32)
    sampler.run_sweeps(ISING, L, 2, 21, 2, 0, 0, 200, 0, spins, E, M, thr)
    _, er, mr = sampler.run_sweeps(ISING, L, 2, 21, 3, 0, 0, 3000, 0, spins, E, M, thr,
                                   record=True)
    betas = np.array([0.40, 0.42, 0.44])
    r = reweight.reweight_series(ISING, L, 2, lnw, er, mr, betas)
    e_ex, _ = reweight.canonical_from_dos(ISING, L, [float(w) for w in ising8_dos], betas)
    # per-chain spread as error bar
    per = np.array([reweight.reweight_series(ISING, L, 2, lnw, er[:, c], mr[:, c], betas)["e"]
                    for c in range(er.shape[1])])
    err = per.std(axis=0, ddof=1) / np.sqrt(er.shape[1])
    assert np.all(np.abs(r["e"] - e_ex) < 5 * err + 1e-4), (r["e"], e_ex, err)
