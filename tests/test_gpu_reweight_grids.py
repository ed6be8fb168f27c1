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
import ctypes

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


def _sparse_samples(model, L, bins, seed):
    """Exact integer sums on a few bins only (counts, sum |M|, sum M^2 consistent)."""
    rng = np.random.default_rng(seed)
    nb = workloads.n_bins(model, L)
    V = L * L
    mmax = V if model == workloads.ISING else 7 * V
    n = np.zeros(nb, dtype=np.uint64)
    s1 = np.zeros(nb, dtype=np.uint64)
    s2 = np.zeros(nb, dtype=np.uint64)
    for b in bins:
        k = int(rng.integers(1, 50))
        m = rng.integers(0, mmax + 1, k).astype(np.uint64)
        n[b], s1[b], s2[b] = k, m.sum(), (m * m).sum()
    lnw = rng.normal(0.0, 3.0, nb)
    return n, s1, s2, lnw


@pytest.mark.parametrize("model,L,bins", [
    (workloads.ISING, 6, [18]),                       # one sampled bin: a one-bin window
    (workloads.ISING, 6, [0, 17, 36]),                # both ends of the range
    (workloads.ISING, 10, [3, 4, 50, 51, 100]),
    (workloads.POTTS, 6, [0, 4, 70, 72])])
def test_reweight_sparse_bins_ragged_and_far_betas(muca, model, L, bins):
    """A few sampled bins (down to one), beta counts that do not fill a tile of 8 (1,
    7, 13), and betas far outside any sampled range (negative, zero, ten times beta_c),
    so that the betas of one tile have their weights peak at opposite ends of the
    energy range: FP64, FP32 and the allocation-free call against the oracle (every beta
    is centred on its own reference bin), all finite.  BF16 centres a tile of 16 betas on
    one bin (its columns are the shared operand of the tensor-core product), so it is
    bounded here on the single beta only; on the configurations' dense grids it is
    bounded above."""
    torch = pytest.importorskip("torch")
    m = muca
    q = 2 if model == workloads.ISING else 8
    n, s1, s2, lnw = _sparse_samples(model, L, bins, 7 + L)
    grids = [np.array([0.44]), np.array([-0.5, 0.0, 0.1, 0.44, 1.0, 2.5, 4.4]),
             np.linspace(-0.3, 3.0, 13)]
    with m.Muca(model, L, q, 8, 1) as g:
        g.set_lnw(lnw)
        g.set_samples(n, s1, s2)
        for betas in grids:
            ref = reweight.reweight_binned(model, L, q, lnw, n, s1, s2, betas)
            for prec in ("fp64", "fp32", "bf16") if len(betas) == 1 else ("fp64", "fp32"):
                r = g.reweight(betas, prec)
                for k in ("e", "C", "absm", "chi"):
                    assert np.all(np.isfinite(r[k])), (prec, k, betas)
                    scale = np.maximum(np.abs(ref[k]), 1e-300)
                    if k in ("C", "chi"):
                        # where one bin dominates, C and chi come from bins of relative
                        # weight below e^-100 (skipped in FP64): bounded absolutely
                        scale = np.maximum(scale, 1e-12)
                    rel = np.abs(r[k] - ref[k]) / scale
                    assert rel.max() <= BOUNDS[prec], (prec, k, betas, float(rel.max()))
            for prec in ("fp64", "fp32"):
                samples = torch.tensor(np.stack([n, s1, s2]).view(np.int64), device="cuda")
                lnw_d = torch.tensor(lnw, device="cuda")
                betas_d = torch.tensor(betas, device="cuda")
                out = torch.full((4, len(betas)), float("nan"), dtype=torch.float64, device="cuda")
                m.check(m.lib().muca_reweight_noalloc(model, L, q, ctypes.c_void_p(samples.data_ptr()),
                                                      ctypes.c_void_p(lnw_d.data_ptr()),
                                                      ctypes.c_void_p(betas_d.data_ptr()), len(betas),
                                                      m.PRECISIONS[prec], ctypes.c_void_p(out.data_ptr()), None))
                torch.cuda.synchronize()
                a = g.reweight(betas, prec)
                got = out.cpu().numpy()
                for row, k in enumerate(("e", "C", "absm", "chi")):
                    assert np.array_equal(got[row], a[k]), (prec, k)


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
