"""Exact results the oracle is checked against, checked among themselves first.

Brute-force enumeration, the transfer matrix and Kaufman's partition function are
three independent routes; they must agree exactly (integers) or to 1e-40 (mpmath).
The 4x4 Ising counts also match the literature values stored in tests/golden.
"""
import os

import mpmath as mp
import numpy as np
import pytest

import exact

HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden_dos():
    rows = [line.split() for line in open(os.path.join(HERE, "golden/ising_4x4_dos.txt"))
            if line.strip() and not line.startswith("#")]
    return {int(e): int(w) for e, w in rows}


def test_ising4_enumeration_matches_literature():
    gold = load_golden_dos()
    om = exact.enumerate_dos(0, 4, 2)
    for b, w in enumerate(om):
        assert gold[4 * b - 32] == w
    assert sum(om) == 2 ** 16


def test_transfer_matrix_matches_enumeration():
    assert list(exact.transfer_dos(0, 4, 2)) == list(exact.enumerate_dos(0, 4, 2))
    assert list(exact.transfer_dos(1, 3, 3)) == list(exact.enumerate_dos(1, 3, 3))
    assert list(exact.transfer_dos(1, 3, 4)) == list(exact.enumerate_dos(1, 3, 4))


def test_potts_q8_closed_counts(potts3_q8_dos):
    om = potts3_q8_dos
    assert sum(om) == 8 ** 9
    assert om[0] == 8                # the q uniform ground states
    assert om[4] == 9 * 7 * 8        # one spin differs: 9 sites x 7 states x 8 grounds


@pytest.mark.parametrize("beta", [0.2, 0.4406867935097715, 0.7])
def test_kaufman_matches_dos(beta, ising8_dos):
    with mp.workdps(60):
        assert abs(exact.kaufman_lnz(4, beta) -
                   exact.lnz_from_dos(0, 4, exact.enumerate_dos(0, 4, 2), beta)) < 1e-40
        assert abs(exact.kaufman_lnz(8, beta) -
                   exact.lnz_from_dos(0, 8, ising8_dos, beta)) < 1e-40


def test_ising8_dos_total(ising8_dos):
    assert sum(ising8_dos) == 2 ** 64
    assert ising8_dos[0] == 2 and ising8_dos[1] == 0 and ising8_dos[2] == 2 * 64


def test_kaufman_specific_heat_peaks_near_beta0():
    """Sec. 3 states beta_0 = ln(1+sqrt 2)/2; the exact finite-L C(beta) of L = 32
    peaks within a finite-size shift of it."""
    beta0 = float(mp.log(1 + mp.sqrt(2)) / 2)
    grid = np.linspace(0.40, 0.46, 25)
    cs = [exact.kaufman_e_c(32, b, dps=40)[1] for b in grid]
    peak = grid[int(np.argmax(cs))]
    assert abs(peak - beta0) < 0.01
