"""muca_reweight_noalloc: reweighting for callers that cannot allocate device memory.

Such callers (a framework allocator already owns the free device memory, or a
latency-critical loop must not stall on cudaMalloc/cudaFree) pass their own device
buffers; the scratch is a fixed array inside the library.  This test calls the
entry point through the C ABI and checks its output against the context-based
muca_reweight, on two calls in a row with different lattices (the second call must
not see anything the first one left in the shared scratch).  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _produce(m, model, L, q, beta, seed):
    g = m.Muca(model, L, q, 64, seed)
    lnw = workloads.canonical_lnw(model, L, beta)
    g.set_lnw(lnw - lnw.max())
    g.thermalize(20)
    g.produce(300, None, None)
    return g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-12)])
def test_noalloc_matches_context_reweight(precision, tol):
    torch = pytest.importorskip("torch")
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    lib = m.lib()
    prec = m.PRECISIONS[precision]
    # two calls in a row, the larger lattice (289 bins) first, so that the second call
    # (257 bins) would read anything stale the first one left in the shared scratch
    cases = [(m.MUCA_POTTS, 12, 8, 1.33, 1.20, 1.40, 37), (m.MUCA_ISING, 16, 2, 0.42, 0.30, 0.55, 61)]
    for model, L, q, beta, lo, hi, n_beta in cases:
        g = _produce(m, model, L, q, beta, seed=11)
        betas = np.linspace(lo, hi, n_beta)
        ref = g.reweight(betas, precision)
        n, s1, s2 = g.get_samples()
        samples = torch.tensor(np.stack([n, s1, s2]).view(np.int64), device="cuda")
        lnw = torch.tensor(g.get_lnw(), device="cuda")
        betas_d = torch.tensor(betas, device="cuda")
        out = torch.full((4, n_beta), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.muca_reweight_noalloc(model, L, q, _ptr(samples), _ptr(lnw), _ptr(betas_d), n_beta, prec,
                                       _ptr(out), None)
        m.check(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for row, key in enumerate(("e", "C", "absm", "chi")):
            rel = np.abs(got[row] - ref[key]) / np.maximum(np.abs(ref[key]), 1e-300)
            assert rel.max() <= tol, (model, key, rel.max())
        # a repeated call takes no device memory (the scratch is already loaded) and
        # gives the same result
        out2 = torch.full((4, n_beta), float("nan"), dtype=torch.float64, device="cuda")
        free1 = torch.cuda.mem_get_info()[0]
        m.check(lib.muca_reweight_noalloc(model, L, q, _ptr(samples), _ptr(lnw), _ptr(betas_d), n_beta, prec,
                                          _ptr(out2), None))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1, "the allocation-free call changed free device memory"
        assert torch.equal(out2, out)
        g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_several_passes(precision):
    """More betas than one pass of the fixed scratch holds (512): 1100 betas in three
    passes give exactly what muca_reweight gives in one call."""
    torch = pytest.importorskip("torch")
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    lib = m.lib()
    g = _produce(m, m.MUCA_ISING, 16, 2, 0.42, seed=5)
    betas = np.linspace(0.25, 0.6, 1100)
    ref = g.reweight(betas, precision)
    n, s1, s2 = g.get_samples()
    samples = torch.tensor(np.stack([n, s1, s2]).view(np.int64), device="cuda")
    lnw = torch.tensor(g.get_lnw(), device="cuda")
    betas_d = torch.tensor(betas, device="cuda")
    out = torch.full((4, len(betas)), float("nan"), dtype=torch.float64, device="cuda")
    m.check(lib.muca_reweight_noalloc(m.MUCA_ISING, 16, 2, _ptr(samples), _ptr(lnw), _ptr(betas_d), len(betas),
                                      m.PRECISIONS[precision], _ptr(out), None))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for row, key in enumerate(("e", "C", "absm", "chi")):
        assert np.all(np.isfinite(got[row])), key
        rel = np.abs(got[row] - ref[key]) / np.maximum(np.abs(ref[key]), 1e-300)
        assert rel.max() <= 1e-12, (key, rel.max())
    g.close()


def test_noalloc_rejects_oversized_and_host_buffers():
    torch = pytest.importorskip("torch")
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    lib = m.lib()
    dev = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 130 x 130 Ising has 16901 bins, above the fixed scratch
    rc = lib.muca_reweight_noalloc(m.MUCA_ISING, 130, 2, _ptr(dev), _ptr(dev), _ptr(dev), 1, m.MUCA_FP64,
                                   _ptr(dev), None)
    assert rc == -1 and b"16385" in lib.muca_last_error()
    host = np.zeros(16)
    rc = lib.muca_reweight_noalloc(m.MUCA_ISING, 8, 2, ctypes.c_void_p(host.ctypes.data), _ptr(dev),
                                   _ptr(dev), 1, m.MUCA_FP64, _ptr(dev), None)
    assert rc == -1
