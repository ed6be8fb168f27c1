"""End-to-end physics of the oracle on the 8x8 Ising workload (statistical pins).

The workload: periodic 8x8 Ising, p = 8 chains, ln W = 0 start, 30 accumulated weight
iterations x 2000 sweeps (Sec. 2 recursion, Sec. 3 correction).  Over independent
seeds, the converged ln W must equal -ln Omega (exact, transfer matrix) and the
reweighted specific heat (Eq. 2, C_V of Sec. 5) must equal the exact C(beta) of
Kaufman's solution, within the seed-to-seed spread (the paper also averages over
independent runs, Sec. 5).
"""
import numpy as np

import exact
from oracle import MucaOracle, reweight

SEEDS = range(1, 9)


def run_c1(seed):
    o = MucaOracle(0, 8, 2, 8, seed)
    stats = []
    for _ in range(30):
        o.iterate(2000)
        stats.append(o.update_weights())
    return o, stats


def test_c1_weights_and_specific_heat(ising8_dos):
    om = np.array([float(w) for w in ising8_dos])
    betas = np.linspace(0.3, 0.6, 31)
    e_ex = np.array([exact.kaufman_e_c(8, b, dps=30) for b in betas])
    devs, cs, converged = [], [], 0
    for seed in SEEDS:
        o, stats = run_c1(seed)
        converged += stats[-1]["converged"]
        acc = o.acc
        target = -np.log(om[acc])
        d = o.lnw[acc] - target
        devs.append(d - d.mean())
        er, mr = o.produce(1000)
        r = o.reweight(er, mr, betas)
        cs.append(r["C"])
    assert converged >= len(SEEDS) - 1
    devs = np.array(devs)
    mean = devs.mean(axis=0)
    err = devs.std(axis=0, ddof=1) / np.sqrt(len(SEEDS))
    assert np.all(np.abs(mean) < 5 * err + 0.02), (mean, err)
    cs = np.array(cs)
    cm = cs.mean(axis=0)
    cerr = cs.std(axis=0, ddof=1) / np.sqrt(len(SEEDS))
    assert np.all(np.abs(cm - e_ex[:, 1]) < 5 * cerr + 1e-3), (cm, e_ex[:, 1], cerr)
    # the paper's quality measure <dC_V> (Eq. 9) for the pooled estimate
    dcv = np.mean(np.abs(cm - e_ex[:, 1]) / e_ex[:, 1])
    assert dcv < 0.02


def test_binned_and_series_agree_on_muca_records():
    o, _ = run_c1(11)
    er, mr = o.produce(200)
    betas = np.linspace(0.3, 0.6, 9)
    a = reweight.reweight_series(0, 8, 2, o.lnw, er, mr, betas)
    b = o.reweight(er, mr, betas)
    for k in a:
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-14)
