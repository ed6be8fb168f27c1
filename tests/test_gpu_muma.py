"""Multimagnetic Ising ensemble on the GPU (Sec. 4, Fig. 6) against the oracle:
sweeps bit for bit with the same tables, thresholds built on each side, production
records, and convergence-driven iteration (N_iter and the weights)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ISING = 0
BETA = 1.5 * math.log(1.0 + math.sqrt(2.0)) / 2.0   # (3/2) beta_0 of Sec. 4


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


def random_m_weights(L, seed):
    rng = np.random.default_rng(seed)
    V = L * L
    k = np.arange(V + 1)
    base = np.array([-math.lgamma(V + 1) + math.lgamma(j + 1) + math.lgamma(V - j + 1) for j in k])
    return base + rng.normal(0, 0.5, V + 1)


@pytest.mark.parametrize("L,p,sweeps", [(4, 5, 40), (6, 37, 20), (8, 33, 20), (12, 40, 6), (34, 9, 2)])
def test_muma_sweeps_bit_exact_with_injected_table(muca, L, p, sweeps):
    from oracle import MucaOracle, weights
    lnw = random_m_weights(L, L + p)
    thr = weights.thresholds_muma(L, lnw, BETA)
    with muca.Muca(ISING, L, 2, p, 77, muma_beta=BETA) as g:
        assert g.n_de == 10 and g.n_bins == L * L + 1
        g.set_thresholds(thr)
        H1 = g.iterate(sweeps)
        g.thermalize(3)
        E_rec, M_rec = g.produce(4)
        spins = g.get_spins()
        E, M = g.get_energies()
    o = MucaOracle(ISING, L, 2, p, 77, muma_beta=BETA)
    h1 = o.iterate(sweeps, thr=thr)
    o.thermalize(3, thr=thr)
    e_rec, m_rec = o.produce(4, thr=thr)
    assert int(H1.sum()) == p * sweeps * L * L
    assert np.array_equal(H1, h1)
    assert np.array_equal(E_rec, e_rec) and np.array_equal(M_rec, m_rec)
    assert np.array_equal(spins, o.spins)
    assert np.array_equal(E, o.E) and np.array_equal(M, o.M)


def test_muma_thresholds_match_oracle(muca):
    from oracle import weights
    L = 8
    lnw = random_m_weights(L, 3)
    with muca.Muca(ISING, L, 2, 4, 1, muma_beta=BETA) as g:
        g.set_lnw(lnw)
        thr = g.get_thresholds()
    ref = weights.thresholds_muma(L, lnw, BETA)
    diff = np.abs(thr.astype(np.int64) - ref.astype(np.int64))
    assert diff.max() <= 1 and int((diff > 0).sum()) <= 2   # CUDA vs libm exp: knife edges only


@pytest.mark.parametrize("L,p,sweeps", [(4, 8, 60), (6, 16, 80)])
def test_muma_converge_equals_oracle(muca, L, p, sweeps):
    from oracle import MucaOracle
    o = MucaOracle(ISING, L, 2, p, 5, muma_beta=BETA)
    n_o, _ = o.converge(sweeps, 300)
    with muca.Muca(ISING, L, 2, p, 5, muma_beta=BETA) as g:
        n_g, st = g.converge(sweeps, 300)
        assert n_g == n_o
        assert n_g > 0 and st["flat"]
        assert np.array_equal(g.get_lnw(), o.lnw)
        E, M = g.get_energies()
        assert np.array_equal(E, o.E) and np.array_equal(M, o.M)


def test_muma_refuses_energy_analyses(muca):
    with muca.Muca(ISING, 4, 2, 4, 1, muma_beta=BETA) as g:
        g.produce(3)
        with pytest.raises(muca.MucaError):
            g.reweight(np.array([0.4]))
        with pytest.raises(muca.MucaError):
            g.energy_distribution([0.4])
    with pytest.raises(muca.MucaError):
        muca.Muca(1, 4, 8, 4, 1, muma_beta=BETA)   # Potts: energy ensemble only
