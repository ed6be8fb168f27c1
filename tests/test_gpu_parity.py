"""GPU path (through the C ABI) against the CPU oracle, element by element.

Trajectories, histograms and records are compared bit for bit when both sides use the
same threshold table (the GPU's table is injected into the oracle, or the oracle's
into the GPU).  ln W after the recursion must agree within 1e-12 (relative, absolute
below 1); tables built from the same ln W may differ by at most 1 in rare entries
(CUDA's and libm's exp may differ in the last bit), which is counted and bounded.
"""
import numpy as np
import pytest

import workloads
from oracle import MucaOracle, reweight, sampler, weights

pytestmark = pytest.mark.gpu

ISING, POTTS = 0, 1


@pytest.fixture(scope="module")
def muca():
    import paper_1212_3975_gb300 as m
    from paper_1212_3975_gb300 import build
    build.build()
    return m


def lnw_close(a, b, tol=1e-12):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.maximum(1.0, np.maximum(np.abs(a), np.abs(b)))
    return np.all(np.abs(a - b) <= tol * scale), np.max(np.abs(a - b) / scale)


def oracle_state(model, L, q, seed, chains):
    spins, E, M = [], [], []
    for c in chains:
        s, e, m = sampler.init_chains(model, L, q, seed, c, 1)
        spins.append(s[0]); E.append(e[0]); M.append(m[0])
    return np.array(spins), np.array(E), np.array(M)


def random_weights(model, L, seed, beta):
    """Seeded weights that make the chains move through many bins."""
    lnw = workloads.canonical_lnw(model, L, beta) + workloads.random_lnw(model, L, seed, 0.3)
    acc = weights.accessible(model, L)
    lnw = np.where(acc, lnw - lnw[acc].max(), 0.0)
    return lnw


INIT_CASES = [(ISING, 4, 2, 5), (ISING, 6, 2, 33), (ISING, 8, 2, 8), (ISING, 24, 2, 70),
              (ISING, 64, 2, 40), (ISING, 96, 2, 3), (POTTS, 3, 8, 7), (POTTS, 5, 8, 65),
              (POTTS, 32, 8, 40), (POTTS, 30, 8, 3)]


@pytest.mark.parametrize("model,L,q,p", INIT_CASES)
def test_init_matches_oracle(muca, model, L, q, p):
    seed = 0x0000000300000011
    with muca.Muca(model, L, q, p, seed) as g:
        spins = g.get_spins()
        E, M = g.get_energies()
        assert np.all(g.get_lnw() == 0)
    s_o, E_o, M_o = sampler.init_chains(model, L, q, seed, 0, p)
    assert np.array_equal(spins, s_o)
    assert np.array_equal(E, E_o)
    assert np.array_equal(M, M_o)


@pytest.mark.parametrize("model,L", [(ISING, 8), (ISING, 64), (POTTS, 6), (POTTS, 32)])
def test_thresholds_from_same_lnw(muca, model, L):
    q = 2 if model == ISING else 8
    lnw = random_weights(model, L, 3, 0.4 if model == ISING else 1.3)
    with muca.Muca(model, L, q, 32, 1) as g:
        g.set_lnw(lnw)
        assert np.array_equal(g.get_lnw(), lnw)
        thr_g = g.get_thresholds()
    thr_o = weights.thresholds(model, L, lnw)
    diff = np.abs(thr_g.astype(np.int64) - thr_o.astype(np.int64))
    assert diff.max() <= 1
    assert (diff > 0).sum() <= max(2, thr_o.size // 10000)


SWEEP_CASES = [
    # model, L, p, sweeps, chains_per_block, staging
    (ISING, 4, 5, 40, 0, 0), (ISING, 6, 37, 20, 0, 0), (ISING, 8, 8, 30, 0, 0),
    (ISING, 24, 70, 6, 64, 0), (ISING, 48, 33, 3, 32, 2), (ISING, 64, 96, 3, 0, 1),
    (ISING, 64, 40, 3, 128, 2), (ISING, 96, 9, 2, 0, 0),
    (POTTS, 3, 7, 40, 0, 0), (POTTS, 4, 9, 40, 0, 0), (POTTS, 8, 33, 20, 0, 2),
    (POTTS, 5, 65, 20, 0, 0), (POTTS, 6, 40, 20, 64, 2),
    (POTTS, 32, 40, 3, 0, 0), (POTTS, 30, 33, 3, 32, 2), (POTTS, 32, 130, 2, 128, 1),
    (POTTS, 64, 35, 2, 0, 0), (POTTS, 128, 20, 1, 0, 0), (POTTS, 160, 8, 1, 0, 0)]


@pytest.mark.parametrize("model,L,p,sweeps,cpb,staging", SWEEP_CASES)
def test_iterate_bit_exact_with_injected_table(muca, model, L, p, sweeps, cpb, staging):
    q = 2 if model == ISING else 8
    seed = 1234
    lnw = random_weights(model, L, L + p, 0.35 if model == ISING else 1.25)
    thr = weights.thresholds(model, L, lnw)
    with muca.Muca(model, L, q, p, seed, chains_per_block=cpb, staging=staging) as g:
        g.set_thresholds(thr)
        H1 = g.iterate(sweeps)
        H2 = g.iterate(max(1, sweeps // 2))
        spins = g.get_spins()
        E, M = g.get_energies()
    o = MucaOracle(model, L, q, p, seed)
    h1 = o.iterate(sweeps, thr=thr)
    h2 = o.iterate(max(1, sweeps // 2), thr=thr)
    assert int(H1.sum()) == p * sweeps * L * L
    assert np.array_equal(H1, h1)
    assert np.array_equal(H2, h2)
    assert np.array_equal(spins, o.spins)
    assert np.array_equal(E, o.E)
    assert np.array_equal(M, o.M)


@pytest.mark.parametrize("model,L,p", [(POTTS, 4, 9), (POTTS, 8, 33), (POTTS, 12, 40), (POTTS, 64, 35),
                                       (ISING, 4, 5), (ISING, 32, 40), (ISING, 64, 33)])
def test_thermalize_bit_exact_with_injected_table(muca, model, L, p):
    """Thermalisation launches (no histogram, no records) against the oracle with the
    same tables, including lattices of one word per row."""
    q = 2 if model == ISING else 8
    seed = 91
    lnw = random_weights(model, L, 8, 0.42 if model == ISING else 1.3)
    thr = weights.thresholds(model, L, lnw)
    with muca.Muca(model, L, q, p, seed) as g:
        g.set_lnw(lnw)
        g.set_thresholds(thr)
        g.thermalize(7)
        g.thermalize(5)
        spins = g.get_spins()
        E, M = g.get_energies()
    o = MucaOracle(model, L, q, p, seed)
    o.thermalize(7, thr=thr)
    o.thermalize(5, thr=thr)
    assert np.array_equal(spins, o.spins)
    assert np.array_equal(E, o.E) and np.array_equal(M, o.M)


@pytest.mark.parametrize("model,L,p", [(ISING, 8, 37), (ISING, 64, 33), (POTTS, 6, 40),
                                       (POTTS, 32, 35), (POTTS, 64, 33), (POTTS, 160, 8)])
def test_produce_records_and_samples(muca, model, L, p):
    q = 2 if model == ISING else 8
    seed = 77
    lnw = random_weights(model, L, 5, 0.42 if model == ISING else 1.3)
    thr = weights.thresholds(model, L, lnw)
    with muca.Muca(model, L, q, p, seed) as g:
        g.set_lnw(lnw)
        g.set_thresholds(thr)
        g.thermalize(3)
        E1, M1 = g.produce(7)
        E2, M2 = g.produce(5)
        n, s1, s2 = g.get_samples()
    o = MucaOracle(model, L, q, p, seed)
    o.thermalize(3, thr=thr)
    e1, m1 = o.produce(7, thr=thr)
    e2, m2 = o.produce(5, thr=thr)
    assert np.array_equal(E1, e1) and np.array_equal(M1, m1)
    assert np.array_equal(E2, e2) and np.array_equal(M2, m2)
    on, os1, os2 = reweight.bin_series(model, L, np.concatenate([e1, e2]),
                                       np.concatenate([m1, m2]))
    assert np.array_equal(n, on) and np.array_equal(s1, os1) and np.array_equal(s2, os2)


@pytest.mark.parametrize("L,per_sm", [(48, 1), (64, 1), (64, 2)])
def test_compact_staging_bit_exact(muca, L, per_sm):
    """More groups of 32 chains than SMs: the compact staging (two blocks per SM, the
    table and a histogram of single attempts in shared memory, the lattices in global
    memory, three draw-ring slots), with a ragged last group; more than two groups per
    SM at L = 64: three blocks per SM with the table of 16-bit threshold halves, whose
    ties (about 2^-16 of the attempts, a few thousand here) replay their word from the
    32-bit table.  Every chain runs on both sides with the same tables: iteration
    histograms, spins, E, M, thermalisation, production records and sums bit for bit."""
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    p = 32 * (per_sm * n_sm + 2) + 5
    seed = 4321
    lnw = random_weights(ISING, L, L + 3, 0.38)
    thr = weights.thresholds(ISING, L, lnw)
    with muca.Muca(ISING, L, 2, p, seed) as g:
        plan = g.plan()
        assert plan & muca.MUCA_PLAN_COMPACT and plan & muca.MUCA_PLAN_TABLE_SMEM, plan
        assert not plan & muca.MUCA_PLAN_LATTICE_SMEM and not plan & muca.MUCA_PLAN_PAIR_HIST, plan
        assert bool(plan & muca.MUCA_PLAN_TABLE16) == (per_sm == 2), plan
        g.set_thresholds(thr)
        H1 = g.iterate(2)
        H2 = g.iterate(1)
        spins = g.get_spins()
        E, M = g.get_energies()
        g.set_lnw(lnw)
        g.set_thresholds(thr)
        g.thermalize(1)
        Er, Mr = g.produce(2)
        n, s1, s2 = g.get_samples()
    o = MucaOracle(ISING, L, 2, p, seed)
    h1 = o.iterate(2, thr=thr)
    h2 = o.iterate(1, thr=thr)
    assert int(H1.sum()) == 2 * p * L * L
    assert np.array_equal(H1, h1) and np.array_equal(H2, h2)
    assert np.array_equal(spins, o.spins)
    assert np.array_equal(E, o.E) and np.array_equal(M, o.M)
    o.thermalize(1, thr=thr)
    er, mr = o.produce(2, thr=thr)
    assert np.array_equal(Er, er) and np.array_equal(Mr, mr)
    on, os1, os2 = reweight.bin_series(ISING, L, er, mr)
    assert np.array_equal(n, on) and np.array_equal(s1, os1) and np.array_equal(s2, os2)


@pytest.mark.parametrize("L,p", [(240, 9), (256, 40)])
def test_hist16_bit_exact(muca, L, p):
    """Ising histograms too large for 32-bit counts in shared memory, with lattices too
    large to stage (L = 240: rows of partial words, the per-word decider; L = 256: the
    stream decider): 16-bit counts, two bins per word, flushed into the merged histogram
    every floor(65535 / (32 L)) rows (7 rows at L = 256: a 2-sweep iteration flushes 73
    times).  Iteration histograms,
    spins, E, M, thermalisation, production records and sums bit for bit against the
    oracle."""
    seed = 2718
    lnw = random_weights(ISING, L, L + 9, 0.40)
    thr = weights.thresholds(ISING, L, lnw)
    with muca.Muca(ISING, L, 2, p, seed) as g:
        plan = g.plan()
        assert plan & muca.MUCA_PLAN_HIST16 and plan & muca.MUCA_PLAN_HIST_SMEM, plan
        assert not plan & muca.MUCA_PLAN_TABLE_SMEM and not plan & muca.MUCA_PLAN_LATTICE_SMEM, plan
        g.set_thresholds(thr)
        H1 = g.iterate(2)
        H2 = g.iterate(1)
        spins = g.get_spins()
        E, M = g.get_energies()
        g.set_lnw(lnw)
        g.set_thresholds(thr)
        g.thermalize(1)
        Er, Mr = g.produce(2)
        n, s1, s2 = g.get_samples()
    o = MucaOracle(ISING, L, 2, p, seed)
    h1 = o.iterate(2, thr=thr)
    h2 = o.iterate(1, thr=thr)
    assert int(H1.sum()) == 2 * p * L * L
    assert np.array_equal(H1, h1) and np.array_equal(H2, h2)
    assert np.array_equal(spins, o.spins)
    assert np.array_equal(E, o.E) and np.array_equal(M, o.M)
    o.thermalize(1, thr=thr)
    er, mr = o.produce(2, thr=thr)
    assert np.array_equal(Er, er) and np.array_equal(Mr, mr)
    on, os1, os2 = reweight.bin_series(ISING, L, er, mr)
    assert np.array_equal(n, on) and np.array_equal(s1, os1) and np.array_equal(s2, os2)


@pytest.mark.parametrize("model,L,p,accumulated", [(ISING, 8, 16, True), (ISING, 8, 16, False),
                                                   (POTTS, 6, 24, True), (ISING, 32, 40, True)])
def test_update_matches_oracle_given_histogram(muca, model, L, p, accumulated):
    q = 2 if model == ISING else 8
    rec = muca.MUCA_RECURSION_ACCUMULATED if accumulated else muca.MUCA_RECURSION_SIMPLE
    nb = weights.n_bins(model, L)
    P = np.zeros(nb)
    lnw_o = np.zeros(nb)
    worst = 0.0
    with muca.Muca(model, L, q, p, 9, recursion=rec) as g:
        for it in range(6):
            H = g.iterate(20)
            lnw_before = g.get_lnw()
            ok, err = lnw_close(lnw_before, lnw_o, 1e-12)
            assert ok, (it, err)
            st = g.update_weights()
            lnw_o, st_o = weights.update_weights(model, L, lnw_before, H, P,
                                                 accumulated=accumulated)
            for k in ("covered", "flat", "lo", "hi", "n_sampled", "total"):
                assert int(st[k]) == int(st_o[k]), k
            assert st["min_over_mean"] == pytest.approx(st_o["min_over_mean"], rel=1e-15)
            ok, err = lnw_close(g.get_lnw(), lnw_o, 1e-12)
            worst = max(worst, err)
            assert ok, (it, err)
            lnw_o = g.get_lnw()       # continue from the GPU's weights


def test_workload_ising_L8_p8_full_loop(muca):
    """The 8x8 Ising workload end to end: 30 x 2000 sweeps, both sides computing their
    own tables; histograms bit-exact, ln W within 1e-12, table mismatches counted."""
    w = workloads.WORKLOADS["ising_L8_p8"]
    g = muca.Muca(w["model"], w["L"], w["q"], w["p"], w["seed"])
    o = MucaOracle(w["model"], w["L"], w["q"], w["p"], w["seed"])
    mismatched_entries = 0
    for it in range(w["iterations"]):
        thr_g = g.get_thresholds()
        mismatched_entries += int((thr_g != o.thr).sum())
        H = g.iterate(w["sweeps"])
        h = o.iterate(w["sweeps"], thr=thr_g)
        assert np.array_equal(H, h), it
        st = g.update_weights()
        st_o = o.update_weights(H)
        assert bool(st["flat"]) == st_o["flat"] and bool(st["covered"]) == st_o["covered"]
        ok, err = lnw_close(g.get_lnw(), o.lnw)
        assert ok, (it, err)
    assert mismatched_entries <= 3
    assert st_o["converged"]
    g.close()


@pytest.mark.parametrize("name,iters,sweeps,sample", [
    ("ising_L64_p1024", 2, 40, [0, 1, 511, 1023]),
    ("potts8_L32_p4096", 2, 20, [0, 2047, 4095]),
])
def test_full_size_sampled_chains(muca, name, iters, sweeps, sample):
    """Full-size workloads in the bench's launch configuration: every chain runs on the
    GPU; sampled chains are replayed by the oracle with the GPU's tables; histogram
    mass and the update are checked in full."""
    w = workloads.WORKLOADS[name]
    model, L, q, p = w["model"], w["L"], w["q"], w["p"]
    g = muca.Muca(model, L, q, p, w["seed"])
    o = MucaOracle(model, L, q, p, w["seed"], chains=sample)
    nb = weights.n_bins(model, L)
    P = np.zeros(nb)
    for it in range(iters):
        thr = g.get_thresholds()
        lnw = g.get_lnw()
        H = g.iterate(sweeps)
        assert int(H.sum()) == p * sweeps * L * L
        o.iterate(sweeps, thr=thr)
        st = g.update_weights()
        lnw_o, st_o = weights.update_weights(model, L, lnw, H, P)
        assert st["lo"] == st_o["lo"] and st["hi"] == st_o["hi"]
        ok, err = lnw_close(g.get_lnw(), lnw_o)
        assert ok, err
    spins = g.get_spins()
    E, M = g.get_energies()
    for k, c in enumerate(sample):
        assert np.array_equal(spins[c], o.spins[k]), c
        assert E[c] == o.E[k] and M[c] == o.M[k]
    g.close()


@pytest.mark.parametrize("name,sweeps,sample", [
    ("ising_L256_p8192", 2, [0, 4097, 8191]),
    ("potts8_L128_p4096", 2, [0, 4095]),
])
def test_large_lattices_fixed_weights(muca, name, sweeps, sample):
    w = workloads.WORKLOADS[name]
    model, L, q, p = w["model"], w["L"], w["q"], w["p"]
    lnw = workloads.canonical_lnw(model, L, w["fixed_beta"])
    acc = weights.accessible(model, L)
    lnw = np.where(acc, lnw - lnw[acc].max(), 0.0)
    g = muca.Muca(model, L, q, p, w["seed"])
    g.set_lnw(lnw)
    thr = g.get_thresholds()
    E_rec, M_rec = g.produce(sweeps)
    n, _, _ = g.get_samples()
    assert int(n.sum()) == p * sweeps
    o = MucaOracle(model, L, q, p, w["seed"], chains=sample)
    e_o, m_o = o.produce(sweeps, thr=thr)
    for k, c in enumerate(sample):
        assert np.array_equal(E_rec[:, c], e_o[:, k]), c
        assert np.array_equal(M_rec[:, c], m_o[:, k]), c
    g.close()


@pytest.mark.parametrize("model,L,p,prec,tol", [
    (ISING, 16, 64, "fp64", 1e-10), (POTTS, 12, 64, "fp64", 1e-10),
    (ISING, 16, 64, "fp32", 1e-6), (POTTS, 12, 64, "fp32", 1e-6)])
def test_reweight_matches_oracle(muca, model, L, p, prec, tol):
    q = 2 if model == ISING else 8
    beta = 0.42 if model == ISING else 1.33
    lnw = random_weights(model, L, 11, beta)
    betas = np.linspace(beta - 0.08, beta + 0.08, 67)
    with muca.Muca(model, L, q, p, 5) as g:
        g.set_lnw(lnw)
        g.thermalize(20)
        E_rec, M_rec = g.produce(200)
        r = g.reweight(betas, prec)
        lnw_g = g.get_lnw()
    ref = reweight.reweight_binned(model, L, q, lnw_g,
                                   *reweight.bin_series(model, L, E_rec, M_rec), betas)
    for k in ("e", "C", "absm", "chi"):
        rel = np.abs(r[k] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-300)
        assert rel.max() <= tol, (k, rel.max())


def test_checkpoint_resume_is_bit_identical(muca, tmp_path):
    path = str(tmp_path / "ck.bin")
    a = muca.Muca(ISING, 16, 2, 40, 3)
    for _ in range(2):
        a.iterate(10)
        a.update_weights()
    a.save(path)
    a.iterate(10)
    a.update_weights()
    Ea, Ma = a.produce(5)
    b = muca.Muca.load(path)
    b.iterate(10)
    b.update_weights()
    Eb, Mb = b.produce(5)
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    assert np.array_equal(a.get_lnw(), b.get_lnw())
    a.close()
    b.close()


@pytest.mark.parametrize("model,L,q,p", [(POTTS, 32, 8, 40), (ISING, 64, 2, 33)])
def test_checkpoint_mid_production_resumes_bit_identically(muca, tmp_path, model, L, q, p):
    """A checkpoint taken between production runs (8-Potts: state counts of the slot
    form's bookkeeper; Ising: the stream decider) resumes with the same records, the
    same production sums and the same reweighted observables; the resumed context was
    validated by the loader's recount."""
    path = str(tmp_path / "prod.ckpt")
    lnw = random_weights(model, L, 11, 0.42 if model == ISING else 1.3)
    a = muca.Muca(model, L, q, p, 21)
    a.set_lnw(lnw)
    a.thermalize(5)
    a.produce(7)
    a.save(path)
    Ea, Ma = a.produce(9)
    na, s1a, s2a = a.get_samples()
    b = muca.Muca.load(path)
    Eb, Mb = b.produce(9)
    nb, s1b, s2b = b.get_samples()
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    assert np.array_equal(na, nb) and np.array_equal(s1a, s1b) and np.array_equal(s2a, s2b)
    betas = np.linspace(0.35, 0.5, 9) if model == ISING else np.linspace(1.25, 1.4, 9)
    ra, rb = a.reweight(betas, "fp64"), b.reweight(betas, "fp64")
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
    a.close()
    b.close()


def test_errors_and_state(muca):
    g = muca.Muca(ISING, 8, 2, 8, 1)
    with pytest.raises(muca.MucaError) as ei:
        g.update_weights()
    assert ei.value.code == muca._muca.MUCA_ERR_STATE
    with pytest.raises(muca.MucaError):
        g.reweight([0.4])
    with pytest.raises(muca.MucaError):
        g.iterate(0)
    g.produce(2)
    g.set_lnw(np.zeros(g.n_bins))
    with pytest.raises(muca.MucaError) as ei:
        g.produce(2)               # weights changed under running production sums
    assert ei.value.code == muca._muca.MUCA_ERR_STATE
    g.reset_samples()
    g.produce(2)
    with pytest.raises(muca.MucaError) as ei:
        muca.Muca.load("/nonexistent/ck.bin")
    assert ei.value.code == muca._muca.MUCA_ERR_IO
    g.close()


@pytest.mark.parametrize("model,L,p,sweeps", [(ISING, 16, 64, 200), (POTTS, 12, 64, 200),
                                              (ISING, 96, 256, 40)])
def test_reweight_precisions_against_oracle(muca, model, L, p, sweeps):
    """FP64 / FP32 / BF16 tensor-core reweighting against the oracle's FP64 binned form:
    FP64 within 1e-10; FP32 and BF16 (three-term split operands, FP32 accumulation
    flushed to FP64) within 1e-6, the bar of the reweighting metric."""
    q = 2 if model == ISING else 8
    beta = 0.42 if model == ISING else 1.33
    lnw = random_weights(model, L, 13, beta)
    betas = np.linspace(beta - 0.06, beta + 0.06, 203)
    with muca.Muca(model, L, q, p, 17) as g:
        g.set_lnw(lnw)
        g.thermalize(20)
        E_rec, M_rec = g.produce(sweeps)
        res = {prec: g.reweight(betas, prec) for prec in ("fp64", "fp32", "bf16")}
        lnw_g = g.get_lnw()
    ref = reweight.reweight_binned(model, L, q, lnw_g,
                                   *reweight.bin_series(model, L, E_rec, M_rec), betas)
    bounds = {"fp64": 1e-10, "fp32": 1e-6, "bf16": 1e-6}
    for prec, r in res.items():
        for k in ("e", "C", "absm", "chi"):
            rel = np.abs(r[k] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-300)
            assert rel.max() <= bounds[prec], (prec, k, rel.max())
