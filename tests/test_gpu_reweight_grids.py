"""Reweighting (Eq. 2; C_V of Sec. 5) at the configurations' full beta grids against
the oracle's FP64 binned form.

Inputs are seeded synthetic production sums (workloads.synthetic_samples): exact integer
per-bin sums shaped like the configurations' production runs, fed to both sides, so
that no input of the oracle comes from the GPU.  The grids are the configurations':
Ising 64x64 with 512 betas on [0.3, 0.6] (flat multicanonical sums over all bins),
8-Potts 32x32 with 1024 betas on [1.2, 1.4], Ising 256x256 and 8-Potts 128x128 with
4096 betas (canonical sums at beta_0, so that most of the grid reweights to the edge
bins of a narrow histogram, where C and chi come from bins of relative weight down to
~1e-12).  Bounds: FP64 1e-10, FP32 1e-6 relative per observable; BF16 (tensor cores,
three-term split operands) is measured and bounded by 1e-5.
"""
import numpy as np
import pytest

import workloads
from oracle import reweight

pytestmark = pytest.mark.gpu

BOUNDS = {"fp64": 1e-10, "fp32": 1e-6, "bf16": 1e-5}


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("name", sorted(workloads.REWEIGHT_CASES))
def test_reweight_full_grid(muca, name):
    model, L, mode, beta_prod, grid, records = workloads.REWEIGHT_CASES[name]
    q = 2 if model == workloads.ISING else 8
    n, s1, s2, lnw = workloads.synthetic_samples(model, L, mode, records, 29, beta_prod)
    betas = workloads.beta_grid(grid)
    ref = reweight.reweight_binned(model, L, q, lnw, n, s1, s2, betas)
    worst = {}
    with muca.Muca(model, L, q, 32, 1) as g:
        g.set_lnw(lnw)
        g.set_samples(n, s1, s2)
        for prec in ("fp64", "fp32", "bf16"):
            r = g.reweight(betas, prec)
            for k in ("e", "C", "absm", "chi"):
                assert np.all(np.isfinite(r[k])), (prec, k)
                rel = np.abs(r[k] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-300)
                worst[(prec, k)] = float(rel.max())
    print(name, {"%s/%s" % pk: "%.2e" % v for pk, v in worst.items()})
    for (prec, k), v in worst.items():
        assert v <= BOUNDS[prec], (name, prec, k, v)


@pytest.mark.parametrize("model,L", [(workloads.ISING, 4), (workloads.ISING, 8), (workloads.ISING, 12),
                                     (workloads.POTTS, 4), (workloads.POTTS, 6)])
def test_reweight_windows_at_the_top_bin(muca, model, L):
    """Flat sums over every bin up to the top of the energy range on small lattices: a
    tile's window then ends at the last bin, and its chunks (whole multiples of 32 bins)
    reach past it.  Every precision against the oracle, all values finite."""
    q = 2 if model == workloads.ISING else 8
    n, s1, s2, lnw = workloads.synthetic_samples(model, L, "flat", 200000, 31)
    assert n[-1] > 0                       # the top bin is sampled
    betas = np.linspace(0.3, 0.6, 40) if model == workloads.ISING else np.linspace(1.2, 1.4, 40)
    ref = reweight.reweight_binned(model, L, q, lnw, n, s1, s2, betas)
    with muca.Muca(model, L, q, 8, 1) as g:
        g.set_lnw(lnw)
        g.set_samples(n, s1, s2)
        for prec in ("fp64", "fp32", "bf16"):
            r = g.reweight(betas, prec)
            for k in ("e", "C", "absm", "chi"):
                assert np.all(np.isfinite(r[k])), (prec, k)
                rel = np.abs(r[k] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-300)
                assert rel.max() <= BOUNDS[prec], (prec, k, float(rel.max()))


def test_set_samples_equals_production(muca):
    """Production sums injected through muca_set_samples reweight exactly as the same
    sums accumulated by muca_produce."""
    m = muca
    with m.Muca(m.MUCA_ISING, 16, 2, 64, 3) as g:
        lnw = workloads.canonical_lnw(m.MUCA_ISING, 16, 0.42)
        g.set_lnw(lnw - lnw.max())
        g.thermalize(10)
        g.produce(200, None, None)
        n, s1, s2 = g.get_samples()
        betas = np.linspace(0.3, 0.6, 40)
        a = g.reweight(betas, "fp64")
        with m.Muca(m.MUCA_ISING, 16, 2, 8, 5) as h:
            h.set_lnw(g.get_lnw())
            h.set_samples(n, s1, s2)
            b = h.reweight(betas, "fp64")
    for k in a:
        assert np.array_equal(a[k], b[k]), k
