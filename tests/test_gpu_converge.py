"""Convergence-driven iteration on the GPU (Sec. 3 stopping rule, N_iter of Sec. 4).

muca_converge against the oracle's converge loop: the same N_iter and bit-identical
weights, spins and energies.  muca_batch_converge against muca_converge on separate
contexts: every lattice freezes in the iteration it converges, so each one's N_iter
and state equal its standalone run; afterwards every lattice iterates again."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ISING, POTTS = 0, 1


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("model,L,q,p,sweeps", [(ISING, 4, 2, 4, 60), (ISING, 8, 2, 8, 150),
                                                (POTTS, 4, 8, 5, 100), (ISING, 12, 2, 37, 60)])
def test_converge_equals_oracle(muca, model, L, q, p, sweeps):
    from oracle import MucaOracle
    o = MucaOracle(model, L, q, p, 21)
    n_o, st_o = o.converge(sweeps, 300)
    with muca.Muca(model, L, q, p, 21) as g:
        n_g, st_g = g.converge(sweeps, 300)
        assert n_g == n_o > 0
        assert st_g["flat"] and st_g["total"] == st_o["total"]
        assert np.array_equal(g.get_lnw(), o.lnw)
        E, M = g.get_energies()
        assert np.array_equal(E, o.E) and np.array_equal(M, o.M)
        assert g.iteration == n_o


@pytest.mark.parametrize("model,L,q,p,sweeps,therm", [(POTTS, 4, 8, 5, 100, 7), (ISING, 8, 2, 8, 150, 13)])
def test_converge_with_thermalization_equals_oracle(muca, model, L, q, p, sweeps, therm):
    from oracle import MucaOracle
    o = MucaOracle(model, L, q, p, 23)
    n_o, _ = o.converge(sweeps, 300, therm)
    with muca.Muca(model, L, q, p, 23) as g:
        n_g, st = g.converge(sweeps, 300, therm)
        assert n_g == n_o
        assert n_g > 0 and st["flat"]
        assert np.array_equal(g.get_lnw(), o.lnw)
        E, M = g.get_energies()
        assert np.array_equal(E, o.E) and np.array_equal(M, o.M)


def test_converge_reports_no_convergence(muca):
    with muca.Muca(ISING, 4, 2, 1, 3) as g:
        n, st = g.converge(1, 2)
        assert n == -1 and not st["flat"]
        assert g.iteration == 2


JOBS = [(ISING, 8, 2, 7, 31), (ISING, 16, 2, 40, 32), (POTTS, 8, 8, 33, 33), (ISING, 8, 2, 64, 34),
        (POTTS, 4, 8, 3, 35), (ISING, 4, 2, 1, 36)]


@pytest.mark.parametrize("therm", [0, 9])
def test_batch_converge_equals_standalone(muca, therm):
    sweeps, max_it = 120, 60
    b = muca.MucaBatch(JOBS)
    n_b = b.converge(sweeps, max_it, therm)
    for j, (model, L, q, p, seed) in enumerate(JOBS):
        with muca.Muca(model, L, q, p, seed) as g:
            n_s, _ = g.converge(sweeps, max_it, therm)
            assert n_b[j] == n_s, (JOBS[j], n_b[j], n_s)
            v = b.job(j)
            assert np.array_equal(v.get_lnw(), g.get_lnw()), JOBS[j]
            assert np.array_equal(v.get_spins(), g.get_spins()), JOBS[j]
            assert np.array_equal(v.get_energies()[0], g.get_energies()[0]), JOBS[j]
            assert v.iteration == g.iteration, JOBS[j]
    assert (n_b > 0).sum() >= len(JOBS) // 2
    # afterwards every lattice iterates again, as its standalone context does
    b.iterate(1, 10, graph=False)
    for j, (model, L, q, p, seed) in enumerate(JOBS):
        with muca.Muca(model, L, q, p, seed) as g:
            g.converge(sweeps, max_it, therm)
            H = g.iterate(10)
            g.update_weights()
            v = b.job(j)
            assert np.array_equal(v.get_histogram(), H), JOBS[j]
            assert np.array_equal(v.get_lnw(), g.get_lnw()), JOBS[j]
    b.close()


def test_study_scan_small(muca):
    import math
    from paper_1212_3975_gb300 import study
    scan = study.m_scan(ISING, 4, [1, 4], [1.0, 2.0, 4.0], 3, 300)
    for p in (1, 4):
        Ms, n, tot = scan[p]
        assert len(Ms) == 3 and all(v == math.inf or v >= 1 for v in n)
        assert all(t == math.inf or t == v * M * p for t, v, M in zip(tot, n, Ms))
    m_opt, per_chain, S = study.speedup_from_scan(scan)
    assert S[1] == 1.0 and math.isfinite(m_opt[4])
