"""ctypes declarations of include/lmmew.h (argument marshalling only).

Loading fails loudly when liblmmew.so has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblmmew.so")

LMMEW_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "OUT_OF_RANGE", -3: "CUDA", -4: "OOM", -5: "TIMEOUT",
    -6: "NOT_IMPLEMENTED",
}


class LmmewError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("pixel_cm", ctypes.c_float),
                ("n_angles", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("bin_cm", ctypes.c_float), ("r_det_cm", ctypes.c_float),
                ("coll_fwhm0_cm", ctypes.c_float), ("coll_fwhm_slope", ctypes.c_float),
                ("scan_time", ctypes.c_float)]


class Attenuation(ctypes.Structure):
    _fields_ = [("rho", ctypes.POINTER(ctypes.c_float)), ("n_knots", ctypes.c_int32),
                ("knot_keV", ctypes.POINTER(ctypes.c_float)),
                ("mu_water_cm", ctypes.POINTER(ctypes.c_float)),
                ("scatter_n", ctypes.c_int32)]


class Lines(ctypes.Structure):
    _fields_ = [("n_lines", ctypes.c_int32), ("energy_keV", ctypes.POINTER(ctypes.c_float)),
                ("yield_", ctypes.POINTER(ctypes.c_float))]


class EnergyModel(ctypes.Structure):
    _fields_ = [("fwhm_frac_ref", ctypes.c_float), ("e_ref_keV", ctypes.c_float),
                ("exponent", ctypes.c_float), ("n_windows", ctypes.c_int32),
                ("win_lo_keV", ctypes.POINTER(ctypes.c_float)),
                ("win_hi_keV", ctypes.POINTER(ctypes.c_float))]


class Events(ctypes.Structure):
    _fields_ = [("angle", ctypes.c_void_p), ("bin", ctypes.c_void_p),
                ("energy_keV", ctypes.c_void_p), ("n", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None

SYMBOLS = {
    "lm_create": (ctypes.c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(Attenuation),
                                 ctypes.POINTER(Lines), ctypes.POINTER(EnergyModel),
                                 ctypes.c_void_p, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_void_p)]),
    "lm_sensitivity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "lm_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Events), ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "lm_forward_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Events),
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lm_backproject": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Events), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "lm_osem": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Events), ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]),
    "lm_set_scatter_precision": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lm_osem_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Events),
                                     ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "lm_batch_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "lm_set_tile_events": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lm_set_energy_pruning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lm_set_table_streaming": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lm_table_streaming": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "lm_set_table_budget": (ctypes.c_int, [ctypes.c_int64]),
    "lm_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lm_set_coarse_stride": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lm_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lm_last_error": (ctypes.c_char_p, []),
    "lm_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lm_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "lm_model_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "lm_surrogate_param_count": (ctypes.c_int, []),
    "lm_surrogate_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]),
    "lm_surrogate_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lm_surrogate_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lm_surrogate_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lm_surrogate_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "lm_surrogate_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "lm_surrogate_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "lm_surrogate_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Events),
                                           ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "lm_set_scatter_model": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "lm_probe_ex2_rate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "lm_selftest_wait_timeout": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
}

SCATTER_EXACT, SCATTER_SURROGATE, SCATTER_NONE, SCATTER_SURROGATE_COARSE = 0, 1, 2, 3


def load(path: str = LIB_PATH):
    """Load liblmmew.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SYMBOLS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def check(rc: int) -> None:
    if rc != LMMEW_OK:
        raise LmmewError(rc, load().lm_last_error().decode(errors="replace"))
