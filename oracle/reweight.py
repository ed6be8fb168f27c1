"""Time-series reweighting of the oracle (Eq. 2 and the C_V of Sec. 5), FP64 numpy.

TEST INFRASTRUCTURE ONLY.

Eq. 2: <O>_beta = < O_i exp(-beta E_i) W^-1(E_i) >_MUCA / < exp(-beta E_i) W^-1(E_i) >_MUCA
over all records i (the parallel production run of Sec. 5 pools every chain).
Sec. 5: C_V = beta^2 (<E^2> - <E>^2) / V.

Outputs per beta (readings where the paper defines nothing):
  e    = <E> / V
  C    = beta^2 (<E^2> - <E>^2) / V     (computed as a centred second pass)
  absm = <|M|> / Mnorm                  Mnorm = V (Ising), (q - 1) V (Potts)
  chi  = beta V (<m^2> - <|m|>^2)       m = M / Mnorm, the variance of |m| computed as
                                        a centred second pass, as C

Two forms are given.  ``reweight_series`` is Eq. 2 written out over the records.
``reweight_binned`` regroups the same sums by energy bin, using the exact integer sums
n(E), sum |M|, sum M^2 of ``bin_series``; with lnOmega(E) = ln n(E) - ln W(E) it is the
same expression, so the two agree to rounding.
"""
import numpy as np

from .weights import ISING, bin_energies, n_bins


def m_norm(model, L, q):
    V = L * L
    return float(V) if model == ISING else float((q - 1) * V)


def reweight_series(model, L, q, lnw, E_rec, M_rec, betas):
    """Eq. 2 over the pooled records (E_rec, M_rec: any shape, same size)."""
    V = L * L
    E = np.asarray(E_rec, dtype=np.float64).ravel()
    Mabs = np.abs(np.asarray(M_rec, dtype=np.float64).ravel())
    Eint = np.asarray(E_rec, dtype=np.int64).ravel()
    b = (Eint + 2 * V) // 4 if model == ISING else Eint + 2 * V
    lw = np.asarray(lnw, dtype=np.float64)[b]
    mn = m_norm(model, L, q)
    out = {k: np.zeros(len(betas)) for k in ("e", "C", "absm", "chi")}
    for j, beta in enumerate(betas):
        arg = -beta * E - lw
        w = np.exp(arg - arg.max())
        Z = w.sum()
        meanE = (w * E).sum() / Z
        var = (w * (E - meanE) ** 2).sum() / Z
        meanM = (w * Mabs).sum() / Z
        varM = (w * (Mabs - meanM) ** 2).sum() / Z
        out["e"][j] = meanE / V
        out["C"][j] = beta * beta * var / V
        out["absm"][j] = meanM / mn
        out["chi"][j] = beta * V * varM / (mn * mn)
    return out


def bin_series(model, L, E_rec, M_rec):
    """Exact integer per-bin sums of the records: n, sum |M|, sum M^2 (uint64)."""
    V = L * L
    nb = n_bins(model, L)
    E = np.asarray(E_rec, dtype=np.int64).ravel()
    M = np.abs(np.asarray(M_rec, dtype=np.int64).ravel())
    b = (E + 2 * V) // 4 if model == ISING else E + 2 * V
    n = np.zeros(nb, dtype=np.uint64)
    s1 = np.zeros(nb, dtype=np.uint64)
    s2 = np.zeros(nb, dtype=np.uint64)
    np.add.at(n, b, np.uint64(1))
    np.add.at(s1, b, M.astype(np.uint64))
    np.add.at(s2, b, (M * M).astype(np.uint64))
    return n, s1, s2


def reweight_binned(model, L, q, lnw, n, s1, s2, betas):
    """Eq. 2 regrouped by energy bin; FP64 throughout."""
    V = L * L
    Eb = bin_energies(model, L).astype(np.float64)
    n = np.asarray(n)
    keep = n > 0
    nk = n[keep].astype(np.float64)
    lnomega = np.log(nk) - np.asarray(lnw, dtype=np.float64)[keep]
    Ek = Eb[keep]
    mabs_mean = np.asarray(s1)[keep].astype(np.float64) / nk
    # within-bin variance of |M|, (n s2 - s1^2) / n^2, from exact integers
    vin = np.array([float((int(a) * int(c) - int(b) * int(b))) / float(int(a) * int(a))
                    for a, b, c in zip(np.asarray(n)[keep], np.asarray(s1)[keep], np.asarray(s2)[keep])])
    mn = m_norm(model, L, q)
    out = {k: np.zeros(len(betas)) for k in ("e", "C", "absm", "chi")}
    for j, beta in enumerate(betas):
        arg = lnomega - beta * Ek
        w = np.exp(arg - arg.max())
        Z = w.sum()
        meanE = (w * Ek).sum() / Z
        var = (w * (Ek - meanE) ** 2).sum() / Z
        meanM = (w * mabs_mean).sum() / Z
        # <|M|^2> - <|M|>^2 = sum_b w_b (within-bin variance + (bin mean - <|M|>)^2) / Z
        varM = (w * (vin + (mabs_mean - meanM) ** 2)).sum() / Z
        out["e"][j] = meanE / V
        out["C"][j] = beta * beta * var / V
        out["absm"][j] = meanM / mn
        out["chi"][j] = beta * V * varM / (mn * mn)
    return out


def canonical_from_dos(model, L, omega, betas):
    """Canonical <E>/V and C from a density of states Omega(E) given per bin.

    This is reweight_binned with ln W = 0 and n(E) = Omega(E): the special case the
    tests compare with exact results."""
    nb = n_bins(model, L)
    zeros = np.zeros(nb, dtype=np.uint64)
    r = reweight_binned(model, L, 2, np.zeros(nb), np.asarray(omega, dtype=np.float64),
                        zeros, zeros, betas)
    return r["e"], r["C"]
