"""Host-side fits of the performance study (Sec. 4, Eq. 7): pinned on synthetic data
with known answers."""
import math

import numpy as np
import pytest

from paper_1212_3975_gb300 import study


def test_m_opt_from_scan_parabola_minimum():
    # total(M) = (log M - log 300)^2 + 5 sampled on a geometric grid: minimum at 300
    M = [50, 100, 200, 400, 800]
    t = [(math.log(m) - math.log(300.0)) ** 2 + 5.0 for m in M]
    m_opt, t_min = study.m_opt_from_scan(M, t)
    assert m_opt == pytest.approx(300.0, rel=1e-9)
    assert t_min == pytest.approx(5.0, abs=1e-9)


def test_m_opt_from_scan_edge_and_unconverged():
    assert study.m_opt_from_scan([10, 20, 40], [3.0, 2.0, 1.0])[0] == 40
    # an unconverged point (inf) never wins
    assert study.m_opt_from_scan([10, 20, 40], [math.inf, 2.0, 4.0])[0] == 20
    assert math.isnan(study.m_opt_from_scan([10, 20], [math.inf, math.inf])[0])


def test_fit_m1_recovers_inverse_p_law():
    p = np.array([1, 2, 4, 8, 16, 32])
    m1 = 1234.5
    assert study.fit_m1(p, m1 / p) == pytest.approx(m1, rel=1e-12)
    # multiplicative noise that is symmetric in log averages out
    noisy = m1 / p * np.exp(np.array([0.1, -0.1, 0.2, -0.2, 0.05, -0.05]))
    assert study.fit_m1(p, noisy) == pytest.approx(m1, rel=1e-12)


def test_fit_power_recovers_eq7():
    L = np.array([8, 16, 24, 32, 48, 64, 96])
    a, b = 5.7, 0.51
    a_fit, b_fit = study.fit_power(L, a * L ** (2 + b))
    assert a_fit == pytest.approx(a, rel=1e-10) and b_fit == pytest.approx(b, abs=1e-12)


def test_eq7_and_speedup():
    assert study.eq7_m_opt(study.ISING, 8, 1) == pytest.approx(5.7 * 8 ** 2.51)
    assert study.eq7_m_opt(study.POTTS, 16, 4) == pytest.approx(24.0 * 16 ** 2.67 / 4)
    s = study.statistical_speedup({1: 1000.0, 2: 500.0, 4: 300.0})
    assert s == {1: 1.0, 2: 2.0, 4: pytest.approx(1000.0 / 300.0)}


def test_mean_n_iter():
    assert study.mean_n_iter([3, 5, 7]) == 5.0
    assert study.mean_n_iter([3, -1]) == math.inf


def test_speedup_from_scan():
    # totals N_iter M p with minima 1000 (p = 1), 1000 (p = 2), 2000 (p = 4)
    scan = {1: ([100, 200, 400], [20.0, 5.0, 4.0], [2000.0, 1000.0, 1600.0]),
            2: ([50, 100, 200], [20.0, 5.0, 4.0], [2000.0, 1000.0, 1600.0]),
            4: ([25, 50, 100], [40.0, 10.0, 8.0], [4000.0, 2000.0, 3200.0])}
    m, per_chain, S = study.speedup_from_scan(scan)
    assert S[1] == 1.0
    assert S[2] == pytest.approx(2.0, rel=1e-9)
    assert S[4] == pytest.approx(2.0, rel=1e-9)
    assert per_chain[4] == pytest.approx(study.m_opt_from_scan(*scan[4][::2])[1] / 4)


def test_fit_inverse_l():
    L = np.array([16, 24, 32, 48])
    v_inf, c = study.fit_inverse_l(L, 0.045 + 0.3 / L)
    assert v_inf == pytest.approx(0.045, abs=1e-12) and c == pytest.approx(0.3, abs=1e-10)
