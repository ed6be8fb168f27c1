"""Convergence-driven weight iteration of the oracle (Sec. 3's stopping rule, counted
as N_iter in Sec. 4): the loop stops at the first iteration whose histogram, before
its update, covers every accessible bin and lies within [1/2, 2] of its mean.

The flatness test here is written out on the histograms themselves, independently of
the oracle's statistics, with the accessible bins taken from exact enumeration."""
import numpy as np
import pytest

import exact
from oracle import MucaOracle

ISING, POTTS = 0, 1


def flat_by_definition(H, accessible):
    h = H[accessible].astype(np.float64)
    if (h == 0).any():
        return False
    mean = h.sum() / len(h)
    return bool(((h >= 0.5 * mean) & (h <= 2.0 * mean)).all())


def accessible_by_enumeration(model, L, q):
    dos = exact.enumerate_dos(model, L, q) if model == ISING else exact.transfer_dos(model, L, q)
    return np.array([int(v) > 0 for v in dos])


@pytest.mark.parametrize("model,L,q,p,sweeps", [(ISING, 4, 2, 4, 60), (POTTS, 3, 8, 3, 80)])
def test_converge_stops_at_first_flat_histogram(model, L, q, p, sweeps):
    acc = accessible_by_enumeration(model, L, q)
    o = MucaOracle(model, L, q, p, 11)
    n_iter, stats = o.converge(sweeps, 200)
    assert n_iter > 0 and stats["flat"]
    # replay step by step: every earlier histogram fails the definition, the last passes
    r = MucaOracle(model, L, q, p, 11)
    for it in range(1, n_iter + 1):
        H = r.iterate(sweeps)
        assert flat_by_definition(H, acc) == (it == n_iter), it
        r.update_weights()
    assert np.array_equal(r.lnw, o.lnw)


def test_converge_reports_no_convergence():
    o = MucaOracle(ISING, 4, 2, 1, 3)
    n_iter, stats = o.converge(1, 2)   # one sweep per iteration cannot cover 15 bins
    assert n_iter == -1 and not stats["flat"]
    assert o.iteration == 2


def test_intermediate_thermalization_runs_between_iterations():
    # the thermalisation sweeps advance the thermalisation counter only after
    # unconverged updates that are not the last allowed iteration
    o = MucaOracle(ISING, 4, 2, 2, 5)
    n_iter, _ = o.converge(1, 3, therm_sweeps=4)
    assert n_iter == -1
    from oracle.muca import PHASE_THERMALIZE
    assert o.sweep_counter[PHASE_THERMALIZE] == 8
    r = MucaOracle(ISING, 4, 2, 2, 5)
    n_iter2, st = r.converge(60, 100, therm_sweeps=5)
    assert n_iter2 > 0 and st["flat"]
    assert r.sweep_counter[PHASE_THERMALIZE] == 5 * (n_iter2 - 1)
