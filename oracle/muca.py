"""The whole parallel MUCA procedure on the CPU, step by step (test infrastructure).

Mirrors the order of the paper: p chains with identical weights and different random
streams (Sec. 2, Parallel Version); each iteration runs M sweeps per chain, merges
H = sum_i H_i, estimates the next weights (Sec. 2 recursion, Sec. 3 correction and
convergence test); afterwards the chains are thermalised and a production run records
(E, M) per sweep (Secs. 3 and 5), which Eq. 2 reweights.

``chains`` may be a subset of 0 .. p-1: every chain's random stream depends only on
(seed, chain id, phase, iteration, sweep, site), so a subset replays exactly the same
trajectories as the full run when it is given the same thresholds.
"""
import numpy as np

from . import sampler, weights, reweight

PHASE_INIT, PHASE_ITERATE, PHASE_THERMALIZE, PHASE_PRODUCE = 0, 1, 2, 3


class MucaOracle:
    def __init__(self, model, L, q, p, seed, chains=None, accumulated=True,
                 correction_width=None, muma_beta=None):
        """muma_beta: the multimagnetic Ising ensemble (weights in M at this beta,
        Sec. 4 / Fig. 6) instead of weights in E."""
        if model == weights.ISING:
            q = 2
        self.model, self.L, self.q, self.p, self.seed = model, L, q, p, seed
        self.muma_beta = muma_beta
        self.V = L * L
        self.n_bins = weights.n_bins(model, L)
        self.acc = weights.accessible(model, L)
        if muma_beta is not None:
            assert model == weights.ISING
            self.acc = np.ones(self.n_bins, dtype=bool)  # every M = -V..V step 2
        self.accumulated = accumulated
        self.correction_width = L if correction_width is None else correction_width
        if chains is None:
            chains = range(p)
        chains = list(chains)
        self.chain_ids = chains
        # chains are initialised one contiguous run at a time
        blocks = []
        for c in chains:
            s, E, M = sampler.init_chains(model, L, q, seed, c, 1)
            blocks.append((s, E, M))
        self.spins = np.ascontiguousarray(np.concatenate([b[0] for b in blocks]))
        self.E = np.concatenate([b[1] for b in blocks])
        self.M = np.concatenate([b[2] for b in blocks])
        self.lnw = np.zeros(self.n_bins)
        self.P = np.zeros(self.n_bins)
        self.iteration = 0
        self.sweep_counter = {PHASE_THERMALIZE: 0, PHASE_PRODUCE: 0}
        self.thr = self._thresholds(self.lnw)

    def _thresholds(self, lnw):
        if self.muma_beta is not None:
            return weights.thresholds_muma(self.L, lnw, self.muma_beta)
        return weights.thresholds(self.model, self.L, lnw, self.acc)

    def _contiguous(self):
        ids = self.chain_ids
        return ids == list(range(ids[0], ids[0] + len(ids)))

    def _run(self, phase, iteration, sweep0, n_sweeps, thr, hist, record):
        if self.muma_beta is not None:
            assert self._contiguous()
            H, er, mr = sampler.run_muma_sweeps(self.L, self.seed, phase, iteration, sweep0, n_sweeps,
                                                self.chain_ids[0], self.spins, self.E, self.M, thr, record)
            return (H if hist else None), [], er, mr
        if self._contiguous():
            # one call over all chains (run in parallel on the host cores)
            h, er, mr = sampler.run_sweeps(self.model, self.L, self.q, self.seed, phase,
                                           iteration, sweep0, n_sweeps, self.chain_ids[0],
                                           self.spins, self.E, self.M, thr,
                                           per_chain_hist=True, record=record)
            H = None
            if hist:
                H = np.zeros(self.n_bins, dtype=np.uint64)
                for c in range(h.shape[0]):           # merge in chain order
                    H += h[c]
            return H, (list(h) if hist else []), er, mr
        # one chain at a time, so that arbitrary (non-contiguous) subsets replay
        H = np.zeros(self.n_bins, dtype=np.uint64) if hist else None
        per_chain_H = []
        recs_E, recs_M = [], []
        for k, c in enumerate(self.chain_ids):
            s = self.spins[k:k + 1].copy()
            E = self.E[k:k + 1].copy()
            M = self.M[k:k + 1].copy()
            h, er, mr = sampler.run_sweeps(self.model, self.L, self.q, self.seed, phase,
                                           iteration, sweep0, n_sweeps, c, s, E, M, thr,
                                           per_chain_hist=True, record=record)
            self.spins[k] = s[0]
            self.E[k] = E[0]
            self.M[k] = M[0]
            if hist:
                H += h[0]
                per_chain_H.append(h[0])
            if record:
                recs_E.append(er[:, 0])
                recs_M.append(mr[:, 0])
        out_E = np.stack(recs_E, axis=1) if record else None
        out_M = np.stack(recs_M, axis=1) if record else None
        return H, per_chain_H, out_E, out_M

    def iterate(self, n_sweeps, thr=None, per_chain=False):
        """One weight iteration's sweeps; returns the merged histogram (uint64)."""
        thr = self.thr if thr is None else np.asarray(thr, dtype=np.uint32)
        H, per, _, _ = self._run(PHASE_ITERATE, self.iteration, 0, n_sweeps, thr, True,
                                 False)
        self.iteration += 1
        self.last_H = H
        return (H, per) if per_chain else H

    def update_weights(self, H=None):
        """Recursion + correction + normalisation from the last (or a given) histogram."""
        H = self.last_H if H is None else H
        self.lnw, stats = weights.update_weights(self.model, self.L, self.lnw, H, self.P,
                                                 accumulated=self.accumulated,
                                                 correction_width=self.correction_width,
                                                 acc=self.acc)
        self.thr = self._thresholds(self.lnw)
        return stats

    def converge(self, n_sweeps, max_iterations, therm_sweeps=0):
        """Weight iterations until convergence (Sec. 3): sweeps of one iteration, then the
        update; stop after the first iteration whose histogram (before its update) is
        covered and flat.  With therm_sweeps > 0 the chains are thermalised with the new
        weights after every update that did not converge, unless it was the last allowed
        iteration (the intermediate thermalisation of Sec. 4).  Returns (N_iter, its
        statistics); N_iter = -1 if no iteration up to max_iterations converged."""
        stats = None
        for it in range(1, max_iterations + 1):
            self.iterate(n_sweeps)
            stats = self.update_weights()
            if stats["flat"]:
                return it, stats
            if therm_sweeps > 0 and it < max_iterations:
                self.thermalize(therm_sweeps)
        return -1, stats

    def set_lnw(self, lnw):
        self.lnw = np.asarray(lnw, dtype=np.float64).copy()
        self.thr = self._thresholds(self.lnw)

    def thermalize(self, n_sweeps, thr=None):
        thr = self.thr if thr is None else thr
        c0 = self.sweep_counter[PHASE_THERMALIZE]
        self._run(PHASE_THERMALIZE, 0, c0, n_sweeps, thr, False, False)
        self.sweep_counter[PHASE_THERMALIZE] = c0 + n_sweeps

    def produce(self, n_sweeps, thr=None, hist=False):
        """Production sweeps; returns (E_rec, M_rec) [n_sweeps, n_chains] int32."""
        thr = self.thr if thr is None else thr
        c0 = self.sweep_counter[PHASE_PRODUCE]
        H, _, E_rec, M_rec = self._run(PHASE_PRODUCE, 0, c0, n_sweeps, thr, hist, True)
        self.sweep_counter[PHASE_PRODUCE] = c0 + n_sweeps
        if hist:
            self.last_H = H
        return E_rec, M_rec

    def reweight(self, E_rec, M_rec, betas, lnw=None):
        lnw = self.lnw if lnw is None else lnw
        n, s1, s2 = reweight.bin_series(self.model, self.L, E_rec, M_rec)
        return reweight.reweight_binned(self.model, self.L, self.q, lnw, n, s1, s2, betas)
