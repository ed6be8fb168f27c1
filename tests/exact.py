"""Exact results used to pin the oracle; independent of ``oracle/`` (no shared code).

* ``energy_np`` / ``magnetization_np``: the Hamiltonians of Sec. 3 (Eqs. 3-4) written
  with numpy rolls on [.., L, L] arrays (site i = y*L + x, x fastest).
* ``enumerate_dos``: brute force over all q^V configurations (tiny lattices only).
* ``transfer_dos``: exact density of states by a site-by-site transfer matrix with the
  first row held fixed (periodic in both directions); integers, no rounding.
* ``kaufman_lnz``: Kaufman's exact partition function of the periodic L x L Ising
  model (B. Kaufman, Phys. Rev. 76, 1232 (1949); in the form of A. E. Ferdinand and
  M. E. Fisher, Phys. Rev. 185, 832 (1969)), evaluated with mpmath.
"""
import itertools
import numpy as np


def energy_np(model, L, s):
    s = np.asarray(s).reshape(s.shape[:-1] + (L, L)) if s.shape[-1] == L * L else s
    r = np.roll(s, -1, axis=-1)
    d = np.roll(s, -1, axis=-2)
    if model == 0:
        return -(s.astype(np.int64) * r + s.astype(np.int64) * d).sum(axis=(-1, -2))
    return -((s == r).astype(np.int64) + (s == d)).sum(axis=(-1, -2))


def magnetization_np(model, q, s):
    s = np.asarray(s)
    if model == 0:
        return s.astype(np.int64).sum(axis=-1)
    V = s.shape[-1]
    counts = np.stack([(s == k).sum(axis=-1) for k in range(q)], axis=-1)
    return q * counts.max(axis=-1) - V


def all_configs(model, L, q):
    V = L * L
    vals = [-1, 1] if model == 0 else list(range(q))
    idx = np.indices((len(vals),) * V).reshape(V, -1).T
    return np.asarray(vals, dtype=np.int8)[idx]


def enumerate_dos(model, L, q):
    """Omega per bin by brute force (bins: Ising (E+2V)/4, Potts E+2V)."""
    V = L * L
    conf = all_configs(model, L, q)
    E = energy_np(model, L, conf.reshape(-1, L, L))
    nb = V + 1 if model == 0 else 2 * V + 1
    b = (E + 2 * V) // 4 if model == 0 else E + 2 * V
    return np.bincount(b, minlength=nb).astype(object)


def enumerate_joint(model, L, q, beta):
    """Canonical <E>/V, C, <|m|>, chi by brute force (tiny lattices)."""
    V = L * L
    conf = all_configs(model, L, q)
    E = energy_np(model, L, conf.reshape(-1, L, L)).astype(np.float64)
    M = np.abs(magnetization_np(model, q, conf)).astype(np.float64)
    mn = float(V) if model == 0 else float((q - 1) * V)
    a = -beta * E
    w = np.exp(a - a.max())
    Z = w.sum()
    e = (w * E).sum() / Z
    var = (w * (E - e) ** 2).sum() / Z
    am = (w * M).sum() / Z / mn
    m2 = (w * M * M).sum() / Z / (mn * mn)
    return e / V, beta * beta * var / V, am, beta * V * (m2 - am * am)


def transfer_dos(model, L, q):
    """Exact Omega per bin via a site-by-site transfer matrix (exact integers).

    The first row r0 is fixed; the frontier holds the newest spin of every column.
    Placing site (x, y) adds its bond to the spin above (frontier[x], row y-1), to its
    left neighbour (frontier[x-1], already row y), for x = L-1 the wrap bond to row y's
    site 0, and for y = L-1 the wrap bond to r0[x].  Counted: satisfied bonds.
    """
    V = L * L
    nstates = q ** L
    nsat = 2 * V + 1
    digits = np.array([[(st // q ** k) % q for k in range(L)] for st in range(nstates)])
    total = [0] * nsat
    for r0 in range(nstates):
        row0 = digits[r0]
        sat0 = sum(int(row0[x] == row0[(x + 1) % L]) for x in range(L))
        D = np.zeros((nstates, nsat), dtype=np.int64)
        D[r0, sat0] = 1
        for y in range(1, L):
            for x in range(L):
                newD = np.zeros_like(D)
                for t in range(q):
                    inc = (digits[:, x] == t).astype(np.int64)            # up
                    if x >= 1:
                        inc += digits[:, x - 1] == t                       # left
                    if x == L - 1:
                        inc += digits[:, 0] == t                           # wrap right
                    if y == L - 1:
                        inc += int(row0[x] == t)                           # wrap down
                    dest = np.arange(nstates) + (t - digits[:, x]) * q ** x
                    for k in range(5):
                        sel = np.nonzero(inc == k)[0]
                        if len(sel) == 0:
                            continue
                        shifted = np.zeros((len(sel), nsat), dtype=np.int64)
                        shifted[:, k:] = D[sel, :nsat - k]
                        np.add.at(newD, dest[sel], shifted)
                D = newD
        col = D.sum(axis=0)
        for k in range(nsat):
            total[k] += int(col[k])
    nb = V + 1 if model == 0 else 2 * V + 1
    omega = [0] * nb
    for sat, cnt in enumerate(total):
        if cnt == 0:
            continue
        E = 2 * V - 2 * sat if model == 0 else -sat
        b = (E + 2 * V) // 4 if model == 0 else E + 2 * V
        omega[b] += cnt
    return np.array(omega, dtype=object)


def kaufman_lnz(L, beta, dps=60):
    """ln Z of the periodic L x L Ising model (J = 1) at coupling K = beta."""
    import mpmath as mp
    with mp.workdps(max(dps, mp.mp.dps)):
        K = mp.mpf(beta)
        n = m = L
        c = mp.cosh(2 * K) * mp.coth(2 * K)

        def gamma(l):
            if l == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(c - mp.cos(mp.pi * l / n))

        z1 = z2 = z3 = z4 = mp.mpf(1)
        for r in range(n):
            go, ge = gamma(2 * r + 1), gamma(2 * r)
            z1 *= 2 * mp.cosh(m * go / 2)
            z2 *= 2 * mp.sinh(m * go / 2)
            z3 *= 2 * mp.cosh(m * ge / 2)
            z4 *= 2 * mp.sinh(m * ge / 2)
        return (mp.log(mp.mpf(1) / 2) + mp.mpf(m * n) / 2 * mp.log(2 * mp.sinh(2 * K))
                + mp.log(z1 + z2 + z3 + z4))


def kaufman_e_c(L, beta, dps=60):
    """Exact e = <E>/V and C = beta^2 d^2 lnZ/dbeta^2 / V of the periodic Ising model."""
    import mpmath as mp
    with mp.workdps(dps):
        f = lambda b: kaufman_lnz(L, b, 0)  # noqa: E731
        b = mp.mpf(beta)
        d1 = mp.diff(f, b, 1)
        d2 = mp.diff(f, b, 2)
        V = L * L
        return float(-d1 / V), float(b * b * d2 / V)


def lnz_from_dos(model, L, omega, beta, dps=60):
    import mpmath as mp
    V = L * L
    with mp.workdps(dps):
        z = mp.mpf(0)
        for b, w in enumerate(omega):
            if w:
                E = 4 * b - 2 * V if model == 0 else b - 2 * V
                z += mp.mpf(int(w)) * mp.exp(-mp.mpf(beta) * E)
        return mp.log(z)


__all__ = ["energy_np", "magnetization_np", "enumerate_dos", "enumerate_joint",
           "transfer_dos", "kaufman_lnz", "kaufman_e_c", "lnz_from_dos", "itertools"]
