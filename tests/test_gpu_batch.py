"""Batched form against standalone contexts (and graph replay against eager launches).

Each lattice of a batch must follow exactly the trajectory it follows alone: the
persistent kernel only changes where and when a work unit runs.  Histograms, spins,
energies and ln W are compared bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ISING, POTTS = 0, 1
JOBS = [(ISING, 8, 2, 40, 3), (ISING, 16, 2, 33, 4), (POTTS, 8, 8, 50, 5), (ISING, 32, 2, 64, 6),
        (POTTS, 12, 8, 32, 7)]


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


def standalone(m, job, iters, sweeps):
    model, L, q, p, seed = job
    g = m.Muca(model, L, q, p, seed)
    H = None
    for _ in range(iters):
        H = g.iterate(sweeps)
        g.update_weights()
    return g, H


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_standalone(muca, graph):
    iters, sweeps = 3, 12
    b = muca.MucaBatch(JOBS)
    b.iterate(iters, sweeps, graph=graph)
    for j, job in enumerate(JOBS):
        g, H = standalone(muca, job, iters, sweeps)
        v = b.job(j)
        assert np.array_equal(v.get_histogram(), H), job
        assert np.array_equal(v.get_spins(), g.get_spins()), job
        Eb, Mb = v.get_energies()
        Es, Ms = g.get_energies()
        assert np.array_equal(Eb, Es) and np.array_equal(Mb, Ms), job
        assert np.array_equal(v.get_lnw(), g.get_lnw()), job
        assert v.iteration == g.iteration == iters
        g.close()
    b.close()


def test_graph_replay_equals_eager_and_continues(muca):
    a = muca.MucaBatch(JOBS)
    c = muca.MucaBatch(JOBS)
    a.iterate(2, 8, graph=True)
    a.iterate(2, 8, graph=True)      # replay of the cached graph continues the chains
    c.iterate(4, 8, graph=False)
    for j in range(len(JOBS)):
        assert np.array_equal(a.job(j).get_spins(), c.job(j).get_spins())
        assert np.array_equal(a.job(j).get_lnw(), c.job(j).get_lnw())
    # a standalone call on a batched context continues the same streams
    g, _ = standalone(muca, JOBS[1], 5, 8)
    v = a.job(1)
    v.iterate(8)
    v.update_weights()
    assert np.array_equal(v.get_spins(), g.get_spins())
    a.close()
    c.close()


def test_autotune_cache_and_equivalence(muca, tmp_path):
    path = str(tmp_path / "tune.json")
    b = muca.MucaBatch(JOBS)
    choice = b.autotune(6, path)
    assert choice[0] >= 1 and choice[1] in (0, 2) and choice[2] in (1, 2)
    text = open(path).read()
    assert str(list(choice)).replace(" ", "") in text.replace(" ", "")
    b2 = muca.MucaBatch(JOBS)
    assert b2.autotune(6, path) == choice        # served from the cache
    # whatever the tuned launch shape, the trajectories are unchanged
    b.iterate(2, 10)
    for j, job in enumerate(JOBS):
        g, H = standalone(muca, job, 2, 10)
        assert np.array_equal(b.job(j).get_histogram(), H)
        g.close()
    b.close()
    b2.close()
