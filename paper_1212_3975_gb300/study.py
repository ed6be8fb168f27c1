"""The performance study of Sec. 4, with chains in the role of cores.

For each lattice size L and number of chains p, parallel MUCA runs start from
ln W = 0 and iterate until the merged histogram is covered and flat (Sec. 3); the
mean number of iterations over independent seeds is N_iter(M, p).  Following Sec. 4:

* the total number of sweeps to convergence is N_iter M p, and its minimum over the
  sweeps per iteration and chain M is M_opt(L, p) (Fig. 2, left);
* M_opt(L, p) = M_1(L) / p is fitted for each L (Fig. 2, right) and
  M_1(L) = a L^(2+b) over L (Fig. 3; Eq. 7 gives a = 5.7(5), b = 0.51(4) for Ising and
  a = 24(4), b = 0.67(6) for 8-Potts);
* the statistical speedup S*_p = [N_iter M_opt(L,1)]_1 / [N_iter M_opt(L,p)]_p compares
  the sweeps per chain to convergence with p chains and with one.

The runs go through the batched C entry point muca_batch_converge (every lattice of a
batch freezes in the iteration it converges); this module only arranges jobs and does
the least-squares fits on the host.
"""
import math

import numpy as np

from . import MucaBatch

ISING, POTTS = 0, 1
# Eq. 7: M_opt(L, p) = a L^(2+b) / p
EQ7 = {ISING: (5.7, 0.51), POTTS: (24.0, 0.67)}


def eq7_m_opt(model, L, p):
    """M_opt(L, p) of Eq. 7 (the paper's fit on its own implementation)."""
    a, b = EQ7[model]
    return a * L ** (2.0 + b) / p


def n_iter_runs(model, L, p_list, M, seeds, max_iterations, seed0=1, therm_sweeps=0, muma_beta=None):
    """N_iter of every (p, seed) at M sweeps per iteration and chain, from one batch
    (therm_sweeps: intermediate thermalisation after every unconverged update).  With
    muma_beta the runs are multimagnetic Ising runs (weights in M at that beta), one
    context after another (batches hold the energy ensemble only).

    Returns {p: array of N_iter over the seeds} (-1 where a run did not converge
    within max_iterations)."""
    q = 2 if model == ISING else 8
    jobs = [(model, L, q, int(p), seed0 + 1000 * i + s) for i, p in enumerate(p_list) for s in range(seeds)]
    if muma_beta is not None:
        from . import Muca
        n = np.full(len(jobs), -1, dtype=np.int32)
        for k, (m, LL, qq, pp, sd) in enumerate(jobs):
            with Muca(m, LL, qq, pp, sd, muma_beta=muma_beta) as g:
                n[k] = g.converge(int(M), max_iterations, therm_sweeps)[0]
        return {int(p): n[i * seeds:(i + 1) * seeds].copy() for i, p in enumerate(p_list)}
    b = MucaBatch(jobs)
    try:
        n = b.converge(int(M), max_iterations, therm_sweeps)
    finally:
        b.close()
    return {int(p): n[i * seeds:(i + 1) * seeds].copy() for i, p in enumerate(p_list)}


def mean_n_iter(runs):
    """Mean N_iter over seeds; infinite when any run failed to converge."""
    runs = np.asarray(runs)
    return math.inf if (runs < 0).any() else float(runs.mean())


def m_opt_from_scan(M_list, totals):
    """M_opt as the minimum of the total sweeps N_iter M p over the scanned M (Sec. 4,
    Fig. 2 left), refined by a parabola in log M through the smallest point and its two
    neighbours when the minimum is interior.  Returns (M_opt, total at the minimum)."""
    M = np.asarray(M_list, dtype=np.float64)
    t = np.asarray(totals, dtype=np.float64)
    order = np.argsort(M)
    M, t = M[order], t[order]
    finite = np.isfinite(t)
    if not finite.any():
        return math.nan, math.inf
    i = int(np.argmin(np.where(finite, t, np.inf)))
    if 0 < i < len(M) - 1 and finite[i - 1] and finite[i + 1]:
        x = np.log(M[i - 1:i + 2])
        y = t[i - 1:i + 2]
        c2, c1, c0 = np.polyfit(x, y, 2)
        if c2 > 0:
            xm = -c1 / (2 * c2)
            if x[0] <= xm <= x[2]:
                return float(math.exp(xm)), float(c0 + c1 * xm + c2 * xm * xm)
    return float(M[i]), float(t[i])


def fit_m1(p_list, m_opt):
    """M_1 of M_opt(p) = M_1 / p: least squares in log space with the exponent fixed
    at -1 (Sec. 4), i.e. the geometric mean of M_opt(p) p."""
    p = np.asarray(p_list, dtype=np.float64)
    m = np.asarray(m_opt, dtype=np.float64)
    ok = np.isfinite(m) & (m > 0)
    return float(np.exp(np.mean(np.log(m[ok] * p[ok]))))


def fit_power(L_list, m1):
    """(a, b) of M_1(L) = a L^(2+b): linear least squares of log(M_1 / L^2) on log L."""
    L = np.asarray(L_list, dtype=np.float64)
    m = np.asarray(m1, dtype=np.float64)
    b, loga = np.polyfit(np.log(L), np.log(m / L ** 2), 1)
    return float(math.exp(loga)), float(b)


def statistical_speedup(sweeps_per_chain):
    """S*_p = [N_iter M]_1 / [N_iter M]_p from {p: mean sweeps per chain to convergence}."""
    base = sweeps_per_chain[1]
    return {p: base / v for p, v in sweeps_per_chain.items()}


def m_scan(model, L, p_list, M_factors, seeds, max_iterations, M_center=None, seed0=1, therm_sweeps=0,
           muma_beta=None):
    """N_iter over a grid of M for every p.  The grid is geometric around M_center(p)
    (default: Eq. 7's M_opt(L, p)); runs sharing an M share one batch.

    Returns {p: (M list, mean N_iter list, total sweeps N_iter M p list)}."""
    if M_center is None:
        M_center = lambda p: eq7_m_opt(model, L, p)  # noqa: E731
    grid = {int(p): sorted({max(1, int(round(M_center(p) * f))) for f in M_factors}) for p in p_list}
    by_M = {}
    for p, Ms in grid.items():
        for M in Ms:
            by_M.setdefault(M, []).append(p)
    res = {p: {} for p in grid}
    for M, ps in sorted(by_M.items()):
        runs = n_iter_runs(model, L, ps, M, seeds, max_iterations, seed0, therm_sweeps, muma_beta)
        for p in ps:
            res[p][M] = mean_n_iter(runs[p])
    out = {}
    for p in grid:
        Ms = sorted(res[p])
        n = [res[p][M] for M in Ms]
        out[p] = (Ms, n, [v * M * p for v, M in zip(n, Ms)])
    return out


def speedup_from_scan(scan):
    """S*_p from the minima of an M scan: the sweeps per chain to convergence at the
    optimal M of each p are min_M(N_iter M p) / p, so
    S*_p = min_total(1) / (min_total(p) / p)."""
    best = {p: m_opt_from_scan(Ms, tot) for p, (Ms, n, tot) in scan.items()}
    per_chain = {p: t / p for p, (m, t) in best.items()}
    return {p: m for p, (m, t) in best.items()}, per_chain, (statistical_speedup(per_chain) if 1 in per_chain
                                                            else {})


def speedup_runs(model, L, p_list, m1, seeds, max_iterations, seed0=7):
    """Mean sweeps per chain to convergence N_iter M_opt(L, p) at M_opt = M_1 / p for
    every p (one batch per p), and S*_p."""
    per_chain = {}
    n_iter = {}
    for p in p_list:
        M = max(1, int(round(m1 / p)))
        runs = n_iter_runs(model, L, [p], M, seeds, max_iterations, seed0)[int(p)]
        n_iter[int(p)] = mean_n_iter(runs)
        per_chain[int(p)] = n_iter[int(p)] * M
    return n_iter, per_chain, statistical_speedup(per_chain) if 1 in per_chain else {}


def fit_inverse_l(L_list, values):
    """(v_inf, c) of v(L) = v_inf + c / L by linear least squares in 1/L."""
    x = 1.0 / np.asarray(L_list, dtype=np.float64)
    c, v_inf = np.polyfit(x, np.asarray(values, dtype=np.float64), 1)
    return float(v_inf), float(c)


def sigma_od_scan(L_list, p=16, runs=4, max_iterations=300, therm_sweeps=200, production=4000,
                  beta_range=(1.25, 1.45), seed0=3, m_factor=1.0, all_runs=False):
    """Order-disorder interface tension of the 8-state Potts model (Sec. 5) for every L:
    `runs` independent MUCA runs of p chains each, iterated to convergence together
    (muca_batch_converge at M = m_factor x Eq. 7's M_opt(L, p)); every converged run is thermalised,
    runs a production that keeps only the per-bin sums, and gives sigma_od(L) from the
    equal-height analysis of muca_interface_tension.  sigma_od(L) is the mean over the
    converged runs; finally sigma_od(L) = sigma_inf + c/L is fitted.  With all_runs, the
    runs that did not pass the flatness test within max_iterations also produce with
    their last weights (the equal-height analysis needs weights that sample both phases,
    not a flat histogram in one iteration); their values are reported apart
    (sigma_od_all over every run whose production shows two peaks).

    Returns ({L: dict(M, converged, N_iter, beta_eqh, sigma_od, sigma_err)},
    (sigma_inf, c))."""
    from . import check, lib
    out = {}
    for L in L_list:
        M = max(10, int(round(m_factor * eq7_m_opt(POTTS, L, p))))
        jobs = [(POTTS, L, 8, p, seed0 + 100 * L + r) for r in range(runs)]
        b = MucaBatch(jobs)
        try:
            n_iter = b.converge(M, max_iterations)
            sig, bet, sig_all = [], [], []
            for j in range(runs):
                if n_iter[j] < 0 and not all_runs:
                    continue
                g = b.job(j)
                g.thermalize(therm_sweeps)
                check(lib().muca_produce(g.handle, production, None, None))
                beta, ratio, peaks, sigma = g.interface_tension(*beta_range)
                if math.isfinite(sigma):
                    sig_all.append(sigma)
                    if n_iter[j] >= 0:
                        sig.append(sigma)
                        bet.append(beta)
        finally:
            b.close()
        conv = [int(x) for x in n_iter if x > 0]
        out[int(L)] = {"M": M, "converged": "%d/%d" % (len(conv), runs),
                       "N_iter": float(np.mean(conv)) if conv else math.nan,
                       "beta_eqh": float(np.mean(bet)) if bet else math.nan,
                       "sigma_od": float(np.mean(sig)) if sig else math.nan,
                       "sigma_err": float(np.std(sig, ddof=1) / math.sqrt(len(sig))) if len(sig) > 1 else math.nan}
        if all_runs:
            out[int(L)].update({"runs_with_two_peaks": len(sig_all),
                                "sigma_od_all": float(np.mean(sig_all)) if sig_all else math.nan,
                                "sigma_err_all": float(np.std(sig_all, ddof=1) / math.sqrt(len(sig_all)))
                                if len(sig_all) > 1 else math.nan})
    # the 1/L fit needs at least three sizes
    Ls = [L for L in out if math.isfinite(out[L]["sigma_od"])]
    fit = fit_inverse_l(Ls, [out[L]["sigma_od"] for L in Ls]) if len(Ls) >= 3 else (math.nan, math.nan)
    return out, fit


def eq7_scan(model, L_list, p_list, M_factors, seeds, max_iterations):
    """Sec. 4 / Eq. 7 from scratch: an M scan at every L, M_opt(L, p) from its minima,
    M_1(L) from M_opt(L, p) = M_1 / p, and (a, b) of M_1(L) = a L^(2+b)."""
    per_L = {}
    for L in L_list:
        scan = m_scan(model, L, p_list, M_factors, seeds, max_iterations)
        m_opt, per_chain, S = speedup_from_scan(scan)
        per_L[int(L)] = {"M_opt": {int(p): m_opt[p] for p in p_list}, "M1": fit_m1(p_list, [m_opt[p] for p in p_list]),
                         "S_star": {int(p): S.get(p, math.nan) for p in p_list}}
    Ls = [L for L in per_L if math.isfinite(per_L[L]["M1"])]
    ab = fit_power(Ls, [per_L[L]["M1"] for L in Ls]) if len(Ls) >= 2 else (math.nan, math.nan)
    return per_L, ab


def main(argv=None):
    """Command line of the longer study runs (their results are quoted in the design
    notes):  python -m paper_1212_3975_gb300.study sigma|eq7 [options]; prints JSON."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["sigma", "eq7"])
    ap.add_argument("--L", type=int, nargs="+", required=True)
    ap.add_argument("--p", type=int, nargs="+", default=[16])
    ap.add_argument("--runs", type=int, default=4, help="sigma: independent runs per L")
    ap.add_argument("--seeds", type=int, default=10, help="eq7: seeds per (p, M)")
    ap.add_argument("--m-factor", type=float, default=1.0, help="sigma: M = factor x Eq. 7 M_opt(L, p)")
    ap.add_argument("--factors", type=float, nargs="+", default=[0.5, 0.7, 1.0, 1.4, 2.0, 2.8, 4.0])
    ap.add_argument("--max-iterations", type=int, default=300)
    ap.add_argument("--production", type=int, default=4000)
    ap.add_argument("--all-runs", action="store_true",
                    help="sigma: also analyse the runs that did not converge (reported apart)")
    ap.add_argument("--model", choices=["ising", "potts"], default="ising")
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    if a.what == "sigma":
        res, (s_inf, c) = sigma_od_scan(a.L, p=a.p[0], runs=a.runs, max_iterations=a.max_iterations,
                                        production=a.production, m_factor=a.m_factor, all_runs=a.all_runs)
        out = {"per_L": res, "sigma_inf": s_inf, "c": c}
        if a.all_runs:
            Ls = [L for L in res if math.isfinite(res[L]["sigma_od_all"])]
            out["sigma_inf_all"], out["c_all"] = (fit_inverse_l(Ls, [res[L]["sigma_od_all"] for L in Ls])
                                                  if len(Ls) >= 3 else (math.nan, math.nan))
    else:
        model = ISING if a.model == "ising" else POTTS
        per_L, (aa, bb) = eq7_scan(model, a.L, a.p, a.factors, a.seeds, a.max_iterations)
        out = {"per_L": per_L, "a": aa, "b": bb, "eq7": EQ7[model]}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    print(json.dumps(out, default=lambda x: None if isinstance(x, float) and not math.isfinite(x) else x))


if __name__ == "__main__":
    main()
