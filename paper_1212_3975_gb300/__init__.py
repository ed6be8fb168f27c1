"""GB300 (sm_103a) parallel multicanonical (MUCA) library: Python binding.

Method: Zierenberg, Marenz, Janke, arXiv:1212.3975.  The computation is in
``libmuca.so`` (include/muca.h); this package only marshals arguments.  Buffers may be
numpy arrays (host) or CUDA torch tensors (device; then the call is asynchronous on
the context's stream).
"""
import ctypes

import numpy as np

from ._muca import (  # noqa: F401
    MUCA_BF16, MUCA_PLAN_COMPACT, MUCA_PLAN_HIST_SMEM, MUCA_PLAN_LATTICE_SMEM, MUCA_PLAN_PAIR_HIST,
    MUCA_PLAN_HIST16, MUCA_PLAN_TABLE16, MUCA_PLAN_TABLE_SMEM, MUCA_PLAN_WARP_SPECIALIZED,
    MUCA_ENSEMBLE_ENERGY, MUCA_ENSEMBLE_MAGNETIZATION, MUCA_FP32, MUCA_FP64, MUCA_ISING, MUCA_POTTS, MUCA_RECURSION_ACCUMULATED, MUCA_RECURSION_SIMPLE, MUCA_STAGING_AUTO, MUCA_STAGING_GLOBAL,
    MUCA_STAGING_SHARED,
    MucaConfig, MucaError, MucaIterStats, MucaJob, check, declared_symbols, lib)

PRECISIONS = {"fp64": MUCA_FP64, "fp32": MUCA_FP32, "bf16": MUCA_BF16}


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError("unsupported buffer type %r" % type(x))


def kernel_launches():
    return int(lib().muca_kernel_launches())


class Muca:
    """One set of p chains sharing ln W(E) (a muca_ctx)."""

    def __init__(self, model, L, q, p, seed, recursion=MUCA_RECURSION_ACCUMULATED,
                 correction_width=0, chains_per_block=0, staging=MUCA_STAGING_AUTO,
                 stream=None, _handle=None, muma_beta=None):
        """muma_beta: multimagnetic Ising ensemble (weights in M at this inverse
        temperature) instead of the multicanonical one."""
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
        else:
            ens = MUCA_ENSEMBLE_ENERGY if muma_beta is None else MUCA_ENSEMBLE_MAGNETIZATION
            cfg = MucaConfig(recursion, correction_width, chains_per_block, staging, ens,
                             0.0 if muma_beta is None else float(muma_beta))
            check(lib().muca_init(ctypes.byref(self._h), model, L, q, p, seed,
                                  ctypes.byref(cfg), _ptr(stream)))
        self.model, self.L, self.q, self.p = model, L, q, p
        self.n_bins = lib().muca_n_bins(self._h)
        self.n_de = lib().muca_n_de(self._h)
        self.V = L * L

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if self._h and getattr(self, "_owned", True):
            lib().muca_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def reset(self, seed):
        """Restart every chain at infinite temperature with a new seed (no allocation)."""
        check(lib().muca_reset(self._h, seed))

    # -- method steps ------------------------------------------------------------
    def iterate(self, n_sweeps, H_out="host"):
        """Sweeps of one weight iteration; returns the merged histogram (uint64)."""
        if isinstance(H_out, str):
            H = np.zeros(self.n_bins, dtype=np.uint64)
            check(lib().muca_iterate(self._h, n_sweeps, _ptr(H)))
            return H
        check(lib().muca_iterate(self._h, n_sweeps, _ptr(H_out)))
        return H_out

    def update_weights(self):
        st = MucaIterStats()
        check(lib().muca_update_weights(self._h, ctypes.byref(st)))
        return st.as_dict()

    def converge(self, n_sweeps, max_iterations, therm_sweeps=0):
        """Weight iterations until the histogram is covered and flat (with therm_sweeps
        of intermediate thermalisation after every update that did not converge);
        returns (N_iter or -1, statistics of the last iteration)."""
        n = ctypes.c_int(-1)
        st = MucaIterStats()
        check(lib().muca_converge(self._h, n_sweeps, therm_sweeps, max_iterations, ctypes.byref(n),
                                  ctypes.byref(st)))
        return n.value, st.as_dict()

    def thermalize(self, n_sweeps):
        check(lib().muca_thermalize(self._h, n_sweeps))

    def energy_distribution(self, betas):
        """ln P_beta(E) of the production sums for every beta: [n_beta, n_bins] FP64."""
        b = np.ascontiguousarray(betas, dtype=np.float64)
        out = np.zeros((len(b), self.n_bins))
        check(lib().muca_energy_distribution(self._h, _ptr(b), len(b), _ptr(out)))
        return out

    def interface_tension(self, beta_lo, beta_hi, n_grid=64, n_bisect=60):
        """(beta_eqh, ln(P_max/P_min), (low peak, high peak, dip) bins, sigma_od(L)) of Sec. 5."""
        be, lr = ctypes.c_double(), ctypes.c_double()
        peaks = np.full(3, -1, dtype=np.int32)
        check(lib().muca_interface_tension(self._h, beta_lo, beta_hi, n_grid, n_bisect, ctypes.byref(be),
                                           ctypes.byref(lr), _ptr(peaks)))
        return be.value, lr.value, tuple(int(x) for x in peaks), lr.value / (2.0 * self.L)

    def produce(self, n_sweeps, E_out="host", M_out="host"):
        """Production sweeps; returns (E, M) records [n_sweeps, p] (int32)."""
        if isinstance(E_out, str):
            E_out = np.zeros((n_sweeps, self.p), dtype=np.int32)
        if isinstance(M_out, str):
            M_out = np.zeros((n_sweeps, self.p), dtype=np.int32)
        check(lib().muca_produce(self._h, n_sweeps, _ptr(E_out), _ptr(M_out)))
        return E_out, M_out

    def reset_samples(self):
        check(lib().muca_reset_samples(self._h))

    def set_samples(self, n, sum_abs_m, sum_m2):
        """Production sums [n_bins] uint64 x 3, taken with the current ln W."""
        arrs = [np.ascontiguousarray(x, dtype=np.uint64) for x in (n, sum_abs_m, sum_m2)]
        for x in arrs:
            assert x.shape == (self.n_bins,)
        check(lib().muca_set_samples(self._h, *[_ptr(x) for x in arrs]))

    def reweight(self, betas, precision="fp64", out=None):
        """Eq. 2 to every beta; returns dict e, C, absm, chi (numpy FP64)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        if out is None:
            b = np.ascontiguousarray(betas, dtype=np.float64)
            res = {k: np.zeros(len(b)) for k in ("e", "C", "absm", "chi")}
            check(lib().muca_reweight(self._h, _ptr(b), len(b), prec, _ptr(res["e"]),
                                      _ptr(res["C"]), _ptr(res["absm"]), _ptr(res["chi"])))
            return res
        check(lib().muca_reweight(self._h, _ptr(betas), int(betas.numel()), prec,
                                  _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(out[3])))
        return out

    # -- state -------------------------------------------------------------------
    def get_lnw(self):
        x = np.zeros(self.n_bins)
        check(lib().muca_get_lnw(self._h, _ptr(x)))
        return x

    def set_lnw(self, lnw):
        x = np.ascontiguousarray(lnw, dtype=np.float64)
        assert x.shape == (self.n_bins,)
        check(lib().muca_set_lnw(self._h, _ptr(x)))

    def get_thresholds(self):
        x = np.zeros((self.n_bins, self.n_de), dtype=np.uint32)
        check(lib().muca_get_thresholds(self._h, _ptr(x)))
        return x

    def set_thresholds(self, thr):
        x = np.ascontiguousarray(thr, dtype=np.uint32)
        assert x.shape == (self.n_bins, self.n_de)
        check(lib().muca_set_thresholds(self._h, _ptr(x)))

    def get_spins(self):
        x = np.zeros((self.p, self.V), dtype=np.int8)
        check(lib().muca_get_spins(self._h, _ptr(x)))
        return x

    def get_energies(self):
        E = np.zeros(self.p, dtype=np.int64)
        M = np.zeros(self.p, dtype=np.int64)
        check(lib().muca_get_energies(self._h, _ptr(E), _ptr(M)))
        return E, M

    def get_histogram(self):
        x = np.zeros(self.n_bins, dtype=np.uint64)
        check(lib().muca_get_histogram(self._h, _ptr(x)))
        return x

    def get_samples(self):
        n = np.zeros(self.n_bins, dtype=np.uint64)
        s1 = np.zeros(self.n_bins, dtype=np.uint64)
        s2 = np.zeros(self.n_bins, dtype=np.uint64)
        check(lib().muca_get_samples(self._h, _ptr(n), _ptr(s1), _ptr(s2)))
        return n, s1, s2

    def plan(self):
        """Staging of the sweep kernels for this context (MUCA_PLAN_* bit mask)."""
        return check(lib().muca_sweep_plan(self._h))

    @property
    def iteration(self):
        return lib().muca_get_iteration(self._h)

    def save(self, path):
        check(lib().muca_save(self._h, path.encode()))

    @classmethod
    def load(cls, path, stream=None):
        h = ctypes.c_void_p()
        check(lib().muca_load(ctypes.byref(h), path.encode(), _ptr(stream)))
        obj = cls.__new__(cls)
        obj._h = h
        obj.n_bins = lib().muca_n_bins(h)
        obj.n_de = lib().muca_n_de(h)
        obj.p = lib().muca_num_chains(h)
        obj.model = 0 if obj.n_de == 4 else 1
        nb = obj.n_bins
        V = nb - 1 if obj.model == 0 else (nb - 1) // 2
        obj.V = V
        obj.L = int(round(V ** 0.5))
        obj.q = 2 if obj.model == 0 else 8
        return obj


class MucaBatch:
    """Many lattices advanced together: one persistent sweep kernel per iteration, a
    batched weight update, optional CUDA-graph replay (a muca_batch)."""

    def __init__(self, jobs, recursion=MUCA_RECURSION_ACCUMULATED, correction_width=0,
                 staging=MUCA_STAGING_AUTO, stream=None):
        arr = (MucaJob * len(jobs))(*[MucaJob(m, L, q, p, seed) for (m, L, q, p, seed) in jobs])
        cfg = MucaConfig(recursion, correction_width, 0, staging, MUCA_ENSEMBLE_ENERGY, 0.0)
        self._h = ctypes.c_void_p()
        check(lib().muca_batch_create(ctypes.byref(self._h), arr, len(jobs), ctypes.byref(cfg),
                                      _ptr(stream)))
        self.jobs = list(jobs)
        self._views = []
        for j, (m, L, q, p, _) in enumerate(jobs):
            v = Muca.__new__(Muca)
            v._h = ctypes.c_void_p(lib().muca_batch_job(self._h, j))
            v._owned = False
            v.model, v.L, v.q, v.p = m, L, q, p
            v.n_bins = lib().muca_n_bins(v._h)
            v.n_de = lib().muca_n_de(v._h)
            v.V = L * L
            self._views.append(v)

    def job(self, j):
        return self._views[j]

    def __len__(self):
        return len(self.jobs)

    def iterate(self, n_iterations, n_sweeps, graph=True):
        check(lib().muca_batch_iterate(self._h, n_iterations, n_sweeps, 1 if graph else 0))

    def converge(self, n_sweeps, max_iterations, therm_sweeps=0):
        """Iterate every lattice until it converges (frozen from then on); returns
        N_iter per lattice (int32, -1 where max_iterations was reached)."""
        out = np.full(len(self.jobs), -1, dtype=np.int32)
        check(lib().muca_batch_converge(self._h, n_sweeps, therm_sweeps, max_iterations, _ptr(out)))
        return out

    def plan(self, j):
        """Staging of job j in the persistent kernel (MUCA_PLAN_* bit mask)."""
        return check(lib().muca_batch_plan(self._h, j))

    def autotune(self, n_sweeps, cache_path=None):
        chosen = (ctypes.c_int * 3)()
        check(lib().muca_batch_autotune(self._h, n_sweeps,
                                        cache_path.encode() if cache_path else None, chosen))
        return tuple(chosen)

    def close(self):
        if self._h:
            for v in self._views:
                v._h = ctypes.c_void_p()
            lib().muca_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
