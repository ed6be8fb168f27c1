"""ctypes binding of libmuca.so: same entry-point names as include/muca.h.

Argument marshalling only.  Every step of the method runs in the CUDA library; there
is no Python or CPU fallback: if libmuca.so is missing or CUDA is unavailable, the
calls raise.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmuca.so")

MUCA_ISING, MUCA_POTTS = 0, 1
MUCA_OK = 0
MUCA_ERR_ARG, MUCA_ERR_CUDA, MUCA_ERR_OOM = -1, -2, -3
MUCA_ERR_TIMEOUT, MUCA_ERR_STATE, MUCA_ERR_IO = -4, -5, -6
MUCA_FP64, MUCA_FP32, MUCA_BF16 = 0, 1, 2
MUCA_RECURSION_ACCUMULATED, MUCA_RECURSION_SIMPLE = 0, 1
MUCA_STAGING_AUTO, MUCA_STAGING_SHARED, MUCA_STAGING_GLOBAL = 0, 1, 2
MUCA_ENSEMBLE_ENERGY, MUCA_ENSEMBLE_MAGNETIZATION = 0, 1
MUCA_PLAN_LATTICE_SMEM, MUCA_PLAN_HIST_SMEM, MUCA_PLAN_TABLE_SMEM, MUCA_PLAN_PAIR_HIST = 1, 2, 4, 8
MUCA_PLAN_COMPACT, MUCA_PLAN_WARP_SPECIALIZED, MUCA_PLAN_TABLE16, MUCA_PLAN_HIST16 = 16, 32, 64, 128

ERROR_NAMES = {-1: "MUCA_ERR_ARG", -2: "MUCA_ERR_CUDA", -3: "MUCA_ERR_OOM",
               -4: "MUCA_ERR_TIMEOUT", -5: "MUCA_ERR_STATE", -6: "MUCA_ERR_IO"}


class MucaConfig(ctypes.Structure):
    _fields_ = [("recursion", ctypes.c_int), ("correction_width", ctypes.c_int),
                ("chains_per_block", ctypes.c_int), ("staging", ctypes.c_int),
                ("ensemble", ctypes.c_int), ("beta", ctypes.c_double)]


class MucaIterStats(ctypes.Structure):
    _fields_ = [("covered", ctypes.c_int32), ("flat", ctypes.c_int32),
                ("lo", ctypes.c_int32), ("hi", ctypes.c_int32),
                ("n_sampled", ctypes.c_int64), ("min_over_mean", ctypes.c_double),
                ("max_over_mean", ctypes.c_double), ("total", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MucaJob(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("L", ctypes.c_int), ("q", ctypes.c_int), ("p", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


class MucaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "error"), code, msg))
        self.code = code


# name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "muca_last_error": (ctypes.c_char_p, []),
    "muca_kernel_launches": (ctypes.c_uint64, []),
    "muca_init": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(MucaConfig), _P]),
    "muca_destroy": (ctypes.c_int, [_P]),
    "muca_reset": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "muca_n_bins": (ctypes.c_int, [_P]),
    "muca_n_de": (ctypes.c_int, [_P]),
    "muca_num_chains": (ctypes.c_int, [_P]),
    "muca_get_iteration": (ctypes.c_int, [_P]),
    "muca_sweep_plan": (ctypes.c_int, [_P]),
    "muca_iterate": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "muca_update_weights": (ctypes.c_int, [_P, ctypes.POINTER(MucaIterStats)]),
    "muca_thermalize": (ctypes.c_int, [_P, ctypes.c_int]),
    "muca_energy_distribution": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "muca_interface_tension": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_void_p]),
    "muca_converge": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(MucaIterStats)]),
    "muca_produce": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "muca_reset_samples": (ctypes.c_int, [_P]),
    "muca_set_samples": (ctypes.c_int, [_P, _P, _P, _P]),
    "muca_reweight": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "muca_reweight_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                             ctypes.c_int, ctypes.c_int, _P, _P]),
    "muca_get_lnw": (ctypes.c_int, [_P, _P]),
    "muca_set_lnw": (ctypes.c_int, [_P, _P]),
    "muca_get_thresholds": (ctypes.c_int, [_P, _P]),
    "muca_set_thresholds": (ctypes.c_int, [_P, _P]),
    "muca_get_spins": (ctypes.c_int, [_P, _P]),
    "muca_get_energies": (ctypes.c_int, [_P, _P, _P]),
    "muca_get_histogram": (ctypes.c_int, [_P, _P]),
    "muca_get_samples": (ctypes.c_int, [_P, _P, _P, _P]),
    "muca_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(MucaJob), ctypes.c_int,
                                         ctypes.POINTER(MucaConfig), _P]),
    "muca_batch_destroy": (ctypes.c_int, [_P]),
    "muca_batch_iterate": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "muca_batch_converge": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "muca_batch_job": (_P, [_P, ctypes.c_int]),
    "muca_batch_plan": (ctypes.c_int, [_P, ctypes.c_int]),
    "muca_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    "muca_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "muca_load": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_char_p, _P]),
}

_lib = None


def lib():
    """Load libmuca.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmuca.so not built; run __graft_entry__.build() "
                              "or python paper_1212_3975_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code < 0:
        msg = lib().muca_last_error()
        raise MucaError(code, msg.decode() if msg else "")
    return code


def declared_symbols():
    return list(_SIGS.keys())
