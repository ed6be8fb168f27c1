"""ctypes binding of the C sampler of the oracle (test infrastructure only).

Functions here marshal numpy arrays into ``muca_oracle.c``; all arithmetic of the
Markov chains (Philox draws, energy changes, acceptance, histograms) is in that file.
"""
import ctypes
import numpy as np

from .build import build_oracle

ISING, POTTS = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_energy.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.orc_energy.restype = ctypes.c_int64
        L.orc_magnetization.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p]
        L.orc_magnetization.restype = ctypes.c_int64
        L.orc_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                               ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]
        L.orc_init.restype = ctypes.c_int
        L.orc_sweeps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                 ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
        L.orc_sweeps.restype = ctypes.c_int
        L.orc_muma_sweeps.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_muma_sweeps.restype = ctypes.c_int
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter, key):
    """Philox4x32-10 block for a 4-word counter and a 2-word key (SC'11)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(o[i]) for i in range(4)]


def energy(model, L, spins):
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().orc_energy(model, L, _ptr(s)))


def magnetization(model, L, q, spins):
    s = np.ascontiguousarray(spins, dtype=np.int8)
    return int(lib().orc_magnetization(model, L, q, _ptr(s)))


def init_chains(model, L, q, seed, chain0, n_chains):
    """Infinite-temperature start (Sec. 3) of chains chain0 .. chain0+n_chains-1.

    Returns (spins[n_chains, V] int8, E[n_chains] int64, M[n_chains] int64)."""
    V = L * L
    spins = np.zeros((n_chains, V), dtype=np.int8)
    E = np.zeros(n_chains, dtype=np.int64)
    M = np.zeros(n_chains, dtype=np.int64)
    rc = lib().orc_init(model, L, q, seed, chain0, n_chains, _ptr(spins), _ptr(E), _ptr(M))
    if rc != 0:
        raise RuntimeError("orc_init failed")
    return spins, E, M


def run_sweeps(model, L, q, seed, phase, iteration, sweep0, n_sweeps, chain0,
               spins, E, M, thr, per_chain_hist=False, record=False):
    """Advance every chain in ``spins`` (modified in place) by ``n_sweeps`` sweeps.

    thr: uint32 [n_bins, n_de] acceptance thresholds.
    Returns (H, E_rec, M_rec): H is [n_chains, n_bins] uint64 when per_chain_hist, else
    the merged histogram H = sum_i H_i (Sec. 2, Parallel Version) as [n_bins] uint64;
    E_rec/M_rec are [n_sweeps, n_chains] int32 records, or None.
    """
    n_chains = spins.shape[0]
    n_bins = (L * L + 1) if model == ISING else (2 * L * L + 1)
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    assert thr.shape[0] == n_bins
    H = np.zeros((n_chains, n_bins), dtype=np.uint64)
    E_rec = np.zeros((n_sweeps, n_chains), dtype=np.int32) if record else None
    M_rec = np.zeros((n_sweeps, n_chains), dtype=np.int32) if record else None
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    assert E.dtype == np.int64 and M.dtype == np.int64
    rc = lib().orc_sweeps(model, L, q, seed, phase, iteration, sweep0, n_sweeps, chain0,
                          n_chains, _ptr(spins), _ptr(E), _ptr(M), _ptr(thr), _ptr(H),
                          _ptr(E_rec), _ptr(M_rec))
    if rc != 0:
        raise RuntimeError("oracle invariant failed: running E/M != recomputed")
    if not per_chain_hist:
        merged = np.zeros(n_bins, dtype=np.uint64)
        for c in range(n_chains):          # merge in chain order
            merged += H[c]
        H = merged
    return H, E_rec, M_rec


def max_threads():
    return int(lib().orc_max_threads())


def set_threads(n):
    """Threads of the loops over chains from now on."""
    lib().orc_set_threads(int(n))


def run_muma_sweeps(L, seed, phase, iteration, sweep0, n_sweeps, chain0, spins, E, M, thr,
                    record=False):
    """Multimagnetic Ising sweeps (weights in M at a fixed beta, folded into thr
    [V + 1, 10]); returns (merged M histogram [V + 1] uint64, E_rec, M_rec)."""
    n_chains = spins.shape[0]
    nb = L * L + 1
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    assert thr.shape == (nb, 10)
    H = np.zeros((n_chains, nb), dtype=np.uint64)
    E_rec = np.zeros((n_sweeps, n_chains), dtype=np.int32) if record else None
    M_rec = np.zeros((n_sweeps, n_chains), dtype=np.int32) if record else None
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    rc = lib().orc_muma_sweeps(L, seed, phase, iteration, sweep0, n_sweeps, chain0, n_chains, _ptr(spins),
                               _ptr(E), _ptr(M), _ptr(thr), _ptr(H), _ptr(E_rec), _ptr(M_rec))
    if rc != 0:
        raise RuntimeError("oracle invariant failed: running E/M != recomputed")
    merged = np.zeros(nb, dtype=np.uint64)
    for c in range(n_chains):
        merged += H[c]
    return merged, E_rec, M_rec
