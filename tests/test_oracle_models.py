"""Oracle Hamiltonians, bins, accessible energies and the infinite-temperature start."""
import numpy as np
import pytest

import exact
from oracle import sampler, weights

ISING, POTTS = 0, 1


@pytest.mark.parametrize("model,L,q", [(ISING, 4, 2), (ISING, 6, 2), (ISING, 8, 2),
                                       (POTTS, 3, 8), (POTTS, 5, 8), (POTTS, 8, 8)])
def test_energy_and_magnetization_match_numpy(model, L, q):
    rng = np.random.default_rng(L * 10 + model)
    V = L * L
    for _ in range(20):
        if model == ISING:
            s = rng.choice(np.array([-1, 1], dtype=np.int8), size=V)
        else:
            s = rng.integers(0, q, size=V).astype(np.int8)
        assert sampler.energy(model, L, s) == int(exact.energy_np(model, L, s.reshape(L, L)))
        assert sampler.magnetization(model, L, q, s) == int(exact.magnetization_np(model, q, s))


def test_ground_states():
    L = 6
    V = L * L
    up = np.ones(V, dtype=np.int8)
    assert sampler.energy(ISING, L, up) == -2 * V
    stag = np.array([1 if (x + y) % 2 == 0 else -1 for y in range(L) for x in range(L)],
                    dtype=np.int8)
    assert sampler.energy(ISING, L, stag) == 2 * V
    assert sampler.magnetization(ISING, L, 2, stag) == 0
    assert sampler.energy(POTTS, L, np.zeros(V, dtype=np.int8)) == -2 * V
    assert sampler.magnetization(POTTS, L, 8, np.full(V, 3, dtype=np.int8)) == 7 * V


def test_bins_cover_energy_range():
    for model, L in ((ISING, 4), (ISING, 64), (POTTS, 32)):
        E = weights.bin_energies(model, L)
        V = L * L
        assert E[0] == -2 * V
        assert E[-1] == (2 * V if model == ISING else 0)
        assert len(E) == weights.n_bins(model, L)


def test_accessible_ising_by_enumeration(ising8_dos):
    for L, om in ((4, exact.enumerate_dos(ISING, 4, 2)), (8, ising8_dos),
                  (6, exact.transfer_dos(ISING, 6, 2))):
        acc = weights.accessible(ISING, L)
        assert list(acc) == [w > 0 for w in om]


def test_accessible_potts_q8_by_transfer_matrix(potts3_q8_dos):
    acc = weights.accessible(POTTS, 3)
    assert list(acc) == [w > 0 for w in potts3_q8_dos]


def test_accessible_potts_low_end_q3_L4():
    """The low-energy pattern (1, 2, 3 and 5 broken bonds impossible) is independent of
    q; checked on the 4x4 lattice with q = 3 by transfer matrix."""
    om = exact.transfer_dos(POTTS, 4, 3)
    acc = weights.accessible(POTTS, 4)
    for b in range(0, 12):
        assert acc[b] == (om[b] > 0), b


@pytest.mark.parametrize("model,L,q", [(ISING, 16, 2), (POTTS, 16, 8)])
def test_init_is_uniform_and_consistent(model, L, q):
    spins, E, M = sampler.init_chains(model, L, q, 1, 0, 64)
    for c in range(64):
        assert E[c] == int(exact.energy_np(model, L, spins[c].reshape(L, L)))
        assert M[c] == int(exact.magnetization_np(model, q, spins[c]))
    vals = spins.ravel()
    if model == ISING:
        frac = (vals == 1).mean()
        assert abs(frac - 0.5) < 5 * np.sqrt(0.25 / vals.size)
    else:
        cnt = np.bincount(vals.astype(np.int64), minlength=q) / vals.size
        assert np.all(np.abs(cnt - 1 / q) < 5 * np.sqrt((1 / q) / vals.size))
    # different chains and different seeds give different lattices
    assert not np.array_equal(spins[0], spins[1])
    s2, _, _ = sampler.init_chains(model, L, q, 2, 0, 1)
    assert not np.array_equal(spins[0], s2[0])
    # a chain's start depends only on (seed, chain id)
    s3, _, _ = sampler.init_chains(model, L, q, 1, 5, 1)
    assert np.array_equal(s3[0], spins[5])
