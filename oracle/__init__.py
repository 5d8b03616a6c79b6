"""FP64 CPU oracle of the LM-MEW path model and LM-OSEM (test infrastructure).

This package is test infrastructure.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the CUDA library and its
Python binding never do.  It wraps ``lmmew_oracle.c`` (plain double-precision
loops that follow the paper's equations and Algorithm 1) with ctypes.

Parity status of each function and what pins it (tests/test_oracle_*.py):
  mu_water, sigma_e, energy_density, window_mass  - closed forms, quadrature
  bin_prob, detector_mass                         - telescoping sums, limits
  line_integral, detector_integral                - analytic chords, brute force
  kn_shape, kn_plane_norm                         - analytic KN cross sections
  row / forward / sensitivity                     - point source in a uniform
                                                    attenuator, brute-force
                                                    bin/energy integration
  osem                                            - EM invariants, MLEM ascent
  angle_paths, sampler.sample_events              - chi-square of sampled event
                                                    histograms against the rows'
                                                    expectation
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmmew_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblmmew_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("h", ctypes.c_double), ("n_angles", ctypes.c_int),
        ("n_bins", ctypes.c_int), ("bin_w", ctypes.c_double), ("r_det", ctypes.c_double),
        ("fwhm0", ctypes.c_double), ("fwhm_slope", ctypes.c_double),
        ("scan_time", ctypes.c_double),
        ("rho", ctypes.POINTER(ctypes.c_float)), ("n_knots", ctypes.c_int),
        ("knot_e", ctypes.c_double * 16), ("knot_mu", ctypes.c_double * 16),
        ("scatter_n", ctypes.c_int),
        ("n_lines", ctypes.c_int), ("line_e", ctypes.c_double * 16),
        ("line_yield", ctypes.c_double * 16),
        ("fwhm_frac", ctypes.c_double), ("e_ref", ctypes.c_double),
        ("fwhm_expo", ctypes.c_double),
        ("n_windows", ctypes.c_int), ("win_lo", ctypes.c_double * 16),
        ("win_hi", ctypes.c_double * 16),
        ("support", ctypes.POINTER(ctypes.c_uint8)),
    ]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PF = ctypes.POINTER(ctypes.c_float)
_PU16 = ctypes.POINTER(ctypes.c_uint16)
_PU8 = ctypes.POINTER(ctypes.c_uint8)
_PI32 = ctypes.POINTER(ctypes.c_int32)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        sig = {
            "orc_create": (_P, [ctypes.POINTER(_Params)]),
            "orc_destroy": (None, [_P]),
            "orc_num_voxels": (_I, [_P]),
            "orc_num_scatter_points": (_I, [_P]),
            "orc_voxel_pixels": (None, [_P, _PI32]),
            "orc_mu_water": (_D, [_P, _D]),
            "orc_sigma_e": (_D, [_P, _D]),
            "orc_energy_density": (_D, [_P, _D, _D]),
            "orc_window_mass": (_D, [_P, _D]),
            "orc_kn_shape": (_D, [_D, _D]),
            "orc_kn_plane_norm": (_D, [_D]),
            "orc_compton_energy": (_D, [_D, _D]),
            "orc_sigma_coll": (_D, [_P, _D]),
            "orc_bin_prob": (_D, [_P, _I, _D, _D]),
            "orc_detector_mass": (_D, [_P, _D, _D]),
            "orc_line_integral": (_D, [_P, _D, _D, _D, _D]),
            "orc_detector_integral": (_D, [_P, _D, _D, _I]),
            "orc_row": (None, [_P, _I, _I, _D, _PD]),
            "orc_scatter_line_row": (None, [_P, _I, _I, _D, _I, _PD]),
            "orc_angle_paths": (None, [_P, _I, _PD, _PD, _PD, _PD, _PD, _PD, _PD]),
            "orc_forward": (None, [_P, _I64, _PU16, _PU16, _PF, _PD, _PD]),
            "orc_backproject": (None, [_P, _I64, _PU16, _PU16, _PF, _PD, _PD]),
            "orc_sensitivity": (None, [_P, _I, _I, _PD]),
            "orc_osem": (None, [_P, _I64, _PU16, _PU16, _PF, _I, _I, _I, _I, _PD, _PD]),
            "orc_max_threads": (_I, []),
            "orc_set_threads": (None, [_I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(n: int) -> None:
    """OpenMP threads for the oracle's later calls from this thread."""
    _load().orc_set_threads(int(n))


def kn_shape(e_kev: float, cos_t: float) -> float:
    return float(_load().orc_kn_shape(e_kev, cos_t))


def kn_plane_norm(e_kev: float) -> float:
    return float(_load().orc_kn_plane_norm(e_kev))


def compton_energy(e_kev: float, cos_t: float) -> float:
    return float(_load().orc_compton_energy(e_kev, cos_t))


class Model:
    """The path model on one grid/scanner/spectrum (FP64)."""

    def __init__(self, *, n, pixel_cm, n_angles, n_bins, bin_cm, r_det_cm, coll_fwhm0_cm,
                 coll_fwhm_slope, scan_time, rho, knot_keV, mu_water_cm, scatter_n,
                 line_keV, yields, fwhm_frac, e_ref_keV, fwhm_exponent, windows,
                 support=None):
        lib = _load()
        self.n = int(n)
        self._rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float32).reshape(-1))
        if support is None:
            support = self._rho > 0
        self._support = np.ascontiguousarray(np.asarray(support).reshape(-1).astype(np.uint8))
        p = _Params()
        p.n, p.h, p.n_angles, p.n_bins = self.n, pixel_cm, n_angles, n_bins
        p.bin_w = bin_cm if bin_cm > 0 else self.n * pixel_cm / n_bins
        p.r_det = r_det_cm if r_det_cm > 0 else self.n * pixel_cm / 2.0
        p.fwhm0, p.fwhm_slope, p.scan_time = coll_fwhm0_cm, coll_fwhm_slope, scan_time
        p.rho = _ptr(self._rho, ctypes.c_float)
        p.n_knots = len(knot_keV)
        for i, (e, mu) in enumerate(zip(knot_keV, mu_water_cm)):
            p.knot_e[i], p.knot_mu[i] = e, mu
        p.scatter_n = scatter_n
        p.n_lines = len(line_keV)
        for i, (e, y) in enumerate(zip(line_keV, yields)):
            p.line_e[i], p.line_yield[i] = e, y
        p.fwhm_frac, p.e_ref, p.fwhm_expo = fwhm_frac, e_ref_keV, fwhm_exponent
        p.n_windows = len(windows)
        for i, (lo, hi) in enumerate(windows):
            p.win_lo[i], p.win_hi[i] = lo, hi
        p.support = _ptr(self._support, ctypes.c_uint8)
        self.params = p
        self.n_angles = int(n_angles)
        self._h = lib.orc_create(ctypes.byref(p))
        self.nq = int(lib.orc_num_voxels(self._h))
        self.np_scatter = int(lib.orc_num_scatter_points(self._h))
        self.voxel_pixels = np.zeros(self.nq, dtype=np.int32)
        lib.orc_voxel_pixels(self._h, _ptr(self.voxel_pixels, ctypes.c_int32))

    @classmethod
    def from_scenario(cls, sc, rho=None, support=None, f32_inputs=True) -> "Model":
        """Model of a synthetic workload.  With ``f32_inputs`` every real
        parameter is first rounded to float32, the precision in which the
        CUDA library's C ABI receives them, so both sides model the same
        scanner; the oracle's arithmetic stays FP64."""
        if rho is None:
            rho = sc.make_phantom().rho
        f = (lambda x: float(np.float32(x))) if f32_inputs else float
        ft = lambda xs: tuple(f(x) for x in xs)  # noqa: E731
        return cls(n=sc.n, pixel_cm=f(sc.pixel_cm), n_angles=sc.n_angles, n_bins=sc.n_bins,
                   bin_cm=f(sc.bin_cm), r_det_cm=f(sc.r_det_cm),
                   coll_fwhm0_cm=f(sc.coll_fwhm0_cm), coll_fwhm_slope=f(sc.coll_fwhm_slope),
                   scan_time=f(sc.scan_time), rho=rho, knot_keV=ft(sc.knot_keV),
                   mu_water_cm=ft(sc.mu_water_cm), scatter_n=sc.scatter_n,
                   line_keV=ft(sc.line_keV), yields=ft(sc.yields), fwhm_frac=f(sc.fwhm_frac),
                   e_ref_keV=f(sc.e_ref_keV), fwhm_exponent=f(sc.fwhm_exponent),
                   windows=tuple(ft(w) for w in sc.windows), support=support)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    # ---- scalar physics ----
    def mu_water(self, e):
        return float(_load().orc_mu_water(self._h, e))

    def sigma_e(self, e):
        return float(_load().orc_sigma_e(self._h, e))

    def energy_density(self, e_hat, e):
        return float(_load().orc_energy_density(self._h, e_hat, e))

    def window_mass(self, e):
        return float(_load().orc_window_mass(self._h, e))

    def sigma_coll(self, depth):
        return float(_load().orc_sigma_coll(self._h, depth))

    def bin_prob(self, b, u, sigma):
        return float(_load().orc_bin_prob(self._h, int(b), u, sigma))

    def detector_mass(self, u, sigma):
        return float(_load().orc_detector_mass(self._h, u, sigma))

    def line_integral(self, x0, y0, x1, y1):
        return float(_load().orc_line_integral(self._h, x0, y0, x1, y1))

    def detector_integral(self, x, y, a):
        return float(_load().orc_detector_integral(self._h, x, y, int(a)))

    # ---- event-level operations ----
    @staticmethod
    def _ev(events):
        a = np.ascontiguousarray(np.asarray(events.angle, dtype=np.uint16))
        b = np.ascontiguousarray(np.asarray(events.bin, dtype=np.uint16))
        e = np.ascontiguousarray(np.asarray(events.energy, dtype=np.float32))
        return a, b, e

    def row(self, a, b, e_hat) -> np.ndarray:
        """System-matrix row over the voxel set (raster order of voxel_pixels)."""
        out = np.zeros(self.nq, dtype=np.float64)
        _load().orc_row(self._h, int(a), int(b), float(e_hat), _ptr(out, ctypes.c_double))
        return out

    def scatter_line_row(self, a, b, e_hat, w) -> np.ndarray:
        """Single-scatter part of line w's row: alpha_w times the n = 1 paths
        of Eq. (s_p) summed over the scatter points, times the detector
        response (voxel order of voxel_pixels)."""
        out = np.zeros(self.nq, dtype=np.float64)
        _load().orc_scatter_line_row(self._h, int(a), int(b), float(e_hat), int(w),
                                     _ptr(out, ctypes.c_double))
        return out

    def angle_paths(self, a) -> dict:
        """Path sensitivities of angle a (Eq. s_p, n = 0 and n = 1): s_prim
        [W, nq], s_scat and e_scat [W, nq, np], and the detector coordinate
        and collimator blur of every voxel (u_q, sig_q) and scatter point
        (u_p, sig_p)."""
        W, nq, npt = self.params.n_lines, self.nq, self.np_scatter
        out = {"s_prim": np.zeros((W, nq)), "s_scat": np.zeros((W, nq, max(npt, 1))),
               "e_scat": np.zeros((W, nq, max(npt, 1))), "u_q": np.zeros(nq),
               "sig_q": np.zeros(nq), "u_p": np.zeros(max(npt, 1)), "sig_p": np.zeros(max(npt, 1))}
        _load().orc_angle_paths(self._h, int(a), *[_ptr(out[k], ctypes.c_double) for k in
                                                    ("s_prim", "s_scat", "e_scat", "u_q", "sig_q",
                                                     "u_p", "sig_p")])
        if npt == 0:
            for k in ("s_scat", "e_scat"):
                out[k] = out[k][:, :, :0]
            for k in ("u_p", "sig_p"):
                out[k] = out[k][:0]
        return out

    def row_image(self, a, b, e_hat) -> np.ndarray:
        img = np.zeros(self.n * self.n)
        img[self.voxel_pixels] = self.row(a, b, e_hat)
        return img

    def forward(self, events, image) -> np.ndarray:
        a, b, e = self._ev(events)
        lam = np.ascontiguousarray(np.asarray(image, dtype=np.float64).reshape(-1))
        y = np.zeros(a.shape[0], dtype=np.float64)
        _load().orc_forward(self._h, a.shape[0], _ptr(a, ctypes.c_uint16),
                            _ptr(b, ctypes.c_uint16), _ptr(e, ctypes.c_float),
                            _ptr(lam, ctypes.c_double), _ptr(y, ctypes.c_double))
        return y

    def backproject(self, events, weight) -> np.ndarray:
        a, b, e = self._ev(events)
        w = np.ascontiguousarray(np.asarray(weight, dtype=np.float64).reshape(-1))
        out = np.zeros(self.n * self.n, dtype=np.float64)
        _load().orc_backproject(self._h, a.shape[0], _ptr(a, ctypes.c_uint16),
                                _ptr(b, ctypes.c_uint16), _ptr(e, ctypes.c_float),
                                _ptr(w, ctypes.c_double), _ptr(out, ctypes.c_double))
        return out

    def sensitivity(self, subset=-1, n_subsets=1) -> np.ndarray:
        out = np.zeros(self.n * self.n, dtype=np.float64)
        _load().orc_sensitivity(self._h, int(subset), int(n_subsets), _ptr(out, ctypes.c_double))
        return out

    def osem(self, events, image, n_subsets, n_iters, start_iter=0, start_subset=0,
             want_loglik=False):
        a, b, e = self._ev(events)
        lam = np.array(np.asarray(image, dtype=np.float64).reshape(-1), copy=True)
        ll = np.zeros(max(n_iters * n_subsets, 1), dtype=np.float64) if want_loglik else None
        _load().orc_osem(self._h, a.shape[0], _ptr(a, ctypes.c_uint16),
                         _ptr(b, ctypes.c_uint16), _ptr(e, ctypes.c_float),
                         int(n_subsets), int(n_iters), int(start_iter), int(start_subset),
                         _ptr(lam, ctypes.c_double),
                         _ptr(ll, ctypes.c_double) if ll is not None else None)
        return (lam, ll) if want_loglik else lam
