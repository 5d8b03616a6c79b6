"""GB300-native LM-MEW OSEM (list-mode multi-energy-window SPECT reconstruction).

A thin Python binding over the C ABI in include/lmmew.h: it marshals host
arrays and torch device tensors into the library's structs and pointers and
passes torch's current CUDA stream.  Every step of the computation runs in the
CUDA kernels of liblmmew.so; PyTorch only provides device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import LmmewError

__all__ = ["Model", "DeviceEvents", "Surrogate", "LmmewError", "library_path", "probe_ex2_rate"]


def library_path() -> str:
    return _native.LIB_PATH


def probe_ex2_rate(stream=None) -> dict:
    """Exponential results per clock per SM of the current GPU (FP32 ex2 and
    the packed f16x2 / bf16x2 forms) and the SM clock (MHz) they refer to."""
    out = (ctypes.c_double * 4)()
    _native.check(_native.load().lm_probe_ex2_rate(_stream(stream), out))
    return {"f32": out[0], "f16x2": out[1], "bf16x2": out[2], "sm_mhz": out[3]}


def set_table_budget(nbytes: int) -> None:
    """Process-wide limit on the path-table bytes Model creation keeps
    resident; larger tables are created streamed (0: no limit beyond the
    device's free memory)."""
    _native.check(_native.load().lm_set_table_budget(int(nbytes)))


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(t, name, dtype, numel=None, min_numel=None):
    """Refuse a tensor the library would read or write through a raw device
    pointer unless it is a contiguous CUDA tensor of the right type and size
    (the C ABI cannot tell a host pointer or a short buffer from a good one)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, not {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, not {t.numel()}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} must have at least {min_numel} elements, not {t.numel()}")
    return t


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class DeviceEvents:
    """List-mode events resident on the GPU (angle/bin as 16-bit, energy f32)."""

    def __init__(self, angle, bin_, energy_keV, device="cuda"):
        torch = _torch()

        def as_u16(x):
            if isinstance(x, torch.Tensor):
                return x.to(device=device, dtype=torch.int16).contiguous()
            arr = np.ascontiguousarray(np.asarray(x, dtype=np.uint16)).view(np.int16)
            return torch.from_numpy(arr.copy()).to(device)

        self.angle = as_u16(angle)
        self.bin = as_u16(bin_)
        if isinstance(energy_keV, torch.Tensor):
            self.energy = energy_keV.to(device=device, dtype=torch.float32).contiguous()
        else:
            self.energy = torch.from_numpy(
                np.ascontiguousarray(np.asarray(energy_keV, dtype=np.float32))).to(device)
        if not (self.angle.numel() == self.bin.numel() == self.energy.numel()):
            raise ValueError("angle, bin and energy must have the same length")

    @classmethod
    def from_list(cls, ev, device="cuda") -> "DeviceEvents":
        return cls(ev.angle, ev.bin, ev.energy, device=device)

    def __len__(self):
        return int(self.energy.numel())

    def struct(self) -> _native.Events:
        return _native.Events(self.angle.data_ptr(), self.bin.data_ptr(), self.energy.data_ptr(),
                              len(self))


class Model:
    """One scanner + object model on the GPU (an ``lm_handle``)."""

    def __init__(self, *, n, pixel_cm, n_angles, n_bins, rho, knot_keV, mu_water_cm, scatter_n,
                 line_keV, yields, windows, fwhm_frac=0.10, e_ref_keV=140.0,
                 fwhm_exponent=-0.5, bin_cm=0.0, r_det_cm=0.0, coll_fwhm0_cm=0.3,
                 coll_fwhm_slope=0.02, scan_time=1.0, support=None, n_subsets=1):
        lib = _native.load()
        self.n = int(n)
        geo = _native.Geometry(self.n, pixel_cm, n_angles, n_bins, bin_cm, r_det_cm,
                               coll_fwhm0_cm, coll_fwhm_slope, scan_time)
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float32).reshape(-1))
        kn = np.ascontiguousarray(np.asarray(knot_keV, dtype=np.float32))
        mu = np.ascontiguousarray(np.asarray(mu_water_cm, dtype=np.float32))
        att = _native.Attenuation(_fptr(rho), kn.size, _fptr(kn), _fptr(mu), int(scatter_n))
        le = np.ascontiguousarray(np.asarray(line_keV, dtype=np.float32))
        ly = np.ascontiguousarray(np.asarray(yields, dtype=np.float32))
        lines = _native.Lines(le.size, _fptr(le), _fptr(ly))
        wlo = np.ascontiguousarray(np.asarray([w[0] for w in windows], dtype=np.float32))
        whi = np.ascontiguousarray(np.asarray([w[1] for w in windows], dtype=np.float32))
        en = _native.EnergyModel(fwhm_frac, e_ref_keV, fwhm_exponent, wlo.size, _fptr(wlo),
                                 _fptr(whi))
        sup = None
        if support is not None:
            sup = np.ascontiguousarray(np.asarray(support).reshape(-1).astype(np.uint8))
        h = ctypes.c_void_p()
        _native.check(lib.lm_create(ctypes.byref(geo), ctypes.byref(att), ctypes.byref(lines),
                                    ctypes.byref(en),
                                    sup.ctypes.data_as(ctypes.c_void_p) if sup is not None else None,
                                    int(n_subsets), ctypes.byref(h)))
        self._h = h
        self.n_subsets = int(n_subsets)
        info = (ctypes.c_int64 * 8)()
        _native.check(lib.lm_model_info(h, info))
        (self.nq, self.np_scatter, self.n_lines, self.n_angles, self.n_bins,
         self.terms_per_event, self.table_bytes, setup_us) = [int(v) for v in info]
        self.setup_ms = setup_us / 1000.0

    @classmethod
    def from_scenario(cls, sc, rho=None, support=None, n_subsets=None) -> "Model":
        if rho is None:
            rho = sc.make_phantom().rho
        return cls(n=sc.n, pixel_cm=sc.pixel_cm, n_angles=sc.n_angles, n_bins=sc.n_bins, rho=rho,
                   knot_keV=sc.knot_keV, mu_water_cm=sc.mu_water_cm, scatter_n=sc.scatter_n,
                   line_keV=sc.line_keV, yields=sc.yields, windows=sc.windows,
                   fwhm_frac=sc.fwhm_frac, e_ref_keV=sc.e_ref_keV,
                   fwhm_exponent=sc.fwhm_exponent, bin_cm=sc.bin_cm, r_det_cm=sc.r_det_cm,
                   coll_fwhm0_cm=sc.coll_fwhm0_cm, coll_fwhm_slope=sc.coll_fwhm_slope,
                   scan_time=sc.scan_time, support=support,
                   n_subsets=sc.n_subsets if n_subsets is None else n_subsets)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _native.load().lm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ calls
    def sensitivity(self, subset=-1, stream=None):
        torch = _torch()
        out = torch.empty(self.n * self.n, dtype=torch.float64, device="cuda")
        _native.check(_native.load().lm_sensitivity(self._h, int(subset),
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    _stream(stream)))
        return out

    def check(self, stream=None):
        """lm_check: wait for the stream and raise LmmewError for what the
        handle's earlier calls found on the device (an event out of range, a
        pipeline wait that ran out of time)."""
        _native.check(_native.load().lm_check(self._h, _stream(stream)))

    def forward(self, events: DeviceEvents, image, out=None, stream=None, check=True):
        """lm_forward.  The library queues its kernels without waiting; with
        check (default) the call then waits and raises for errors found on
        the device, with check=False it returns at once (call check() later)."""
        torch = _torch()
        image = image.to(device="cuda", dtype=torch.float32).contiguous().reshape(-1)
        _require_cuda(image, "image", torch.float32, numel=self.n * self.n)
        if out is None:
            out = torch.empty(len(events), dtype=torch.float32, device="cuda")
        _require_cuda(out, "out", torch.float32, numel=len(events))
        ev = events.struct()
        _native.check(_native.load().lm_forward(self._h, ctypes.byref(ev),
                                                ctypes.c_void_p(image.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr()),
                                                _stream(stream)))
        if check:
            self.check(stream)
        return out

    def forward_noalloc(self, events: DeviceEvents, image, out, stream=None, check=True):
        """lm_forward_noalloc: same result as forward(), no device allocation
        inside the call (``image`` and ``out`` are caller-owned CUDA tensors);
        ``check`` as in forward()."""
        torch = _torch()
        _require_cuda(image, "image", torch.float32, numel=self.n * self.n)
        _require_cuda(out, "out", torch.float32, numel=len(events))
        ev = events.struct()
        _native.check(_native.load().lm_forward_noalloc(self._h, ctypes.byref(ev),
                                                        ctypes.c_void_p(image.data_ptr()),
                                                        ctypes.c_void_p(out.data_ptr()),
                                                        _stream(stream)))
        if check:
            self.check(stream)
        return out

    def backproject(self, events: DeviceEvents, weight, out=None, stream=None, check=True):
        """lm_backproject; ``check`` as in forward()."""
        torch = _torch()
        weight = weight.to(device="cuda", dtype=torch.float32).contiguous().reshape(-1)
        _require_cuda(weight, "weight", torch.float32, numel=len(events))
        if out is None:
            out = torch.empty(self.n * self.n, dtype=torch.float32, device="cuda")
        _require_cuda(out, "out", torch.float32, numel=self.n * self.n)
        ev = events.struct()
        _native.check(_native.load().lm_backproject(self._h, ctypes.byref(ev),
                                                    ctypes.c_void_p(weight.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()),
                                                    _stream(stream)))
        if check:
            self.check(stream)
        return out

    def osem(self, events: DeviceEvents, image, n_subsets, n_iters, start_iter=0, start_subset=0,
             loglik=None, stream=None, check=True):
        """Run LM-OSEM in place on ``image`` (a float32 CUDA tensor of n*n);
        ``check`` as in forward()."""
        torch = _torch()
        _require_cuda(image, "image", torch.float32, numel=self.n * self.n)
        if loglik is not None:
            _require_cuda(loglik, "loglik", torch.float64,
                          min_numel=max(int(n_iters), 0) * max(int(n_subsets), 0))
        ev = events.struct()
        llp = ctypes.c_void_p(loglik.data_ptr()) if loglik is not None else None
        _native.check(_native.load().lm_osem(self._h, ctypes.byref(ev), int(n_subsets),
                                             int(n_iters), int(start_iter), int(start_subset),
                                             ctypes.c_void_p(image.data_ptr()), llp,
                                             _stream(stream)))
        if check:
            self.check(stream)
        return image

    def osem_batch(self, events_list, images, n_subsets, n_iters, loglik=None, stream=None):
        """Batched LM-OSEM: ``images`` is a contiguous float32 CUDA tensor
        [R, n*n] updated in place; ``events_list`` holds R DeviceEvents."""
        torch = _torch()
        R = len(events_list)
        _require_cuda(images, "images", torch.float32, numel=R * self.n * self.n)
        if loglik is not None:
            _require_cuda(loglik, "loglik", torch.float64,
                          min_numel=R * max(int(n_iters), 0) * max(int(n_subsets), 0))
        arr = (_native.Events * R)(*[e.struct() for e in events_list])
        llp = ctypes.c_void_p(loglik.data_ptr()) if loglik is not None else None
        _native.check(_native.load().lm_osem_batch(self._h, R, arr, int(n_subsets), int(n_iters),
                                                   ctypes.c_void_p(images.data_ptr()), llp,
                                                   _stream(stream)))
        return images

    def batch_tuning(self) -> dict:
        out = (ctypes.c_double * 5)()
        _native.check(_native.load().lm_batch_tuning(self._h, out))
        return {"unit_order": int(out[0]), "ctas_per_sm": int(out[1]), "tuned": bool(out[2]),
                "tuned_ms": out[3], "tile_events": int(out[4])}

    def set_tile_events(self, tile_events: int):
        """Events per row-kernel tile (32, 64 or 128) until the next autotune."""
        _native.check(_native.load().lm_set_tile_events(self._h, int(tile_events)))

    def set_energy_pruning(self, enable: bool = True):
        """Evaluate each event's single-scatter terms only for the lines whose
        scatter can reach its recorded energy (default), or for every line."""
        _native.check(_native.load().lm_set_energy_pruning(self._h, 1 if enable else 0))

    def set_table_streaming(self, max_angles: int = 0):
        """Keep the single-scatter path tables of at most max_angles angles on
        the device, rebuilding each block of angles a row launch needs (0:
        every angle resident).  Results are bit-identical either way."""
        _native.check(_native.load().lm_set_table_streaming(self._h, int(max_angles)))

    def table_streaming(self):
        """(angles the streamed table buffer holds, 0 if every angle is
        resident; bytes of the table buffer)."""
        slots = ctypes.c_int(0)
        nbytes = ctypes.c_int64(0)
        _native.check(_native.load().lm_table_streaming(self._h, ctypes.byref(slots),
                                                         ctypes.byref(nbytes)))
        return slots.value, nbytes.value

    PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}

    def set_scatter_precision(self, precision="fp32"):
        """Arithmetic of the single-scatter sum: 'fp32' (exact path), 'fp16' or 'bf16'."""
        _native.check(_native.load().lm_set_scatter_precision(self._h,
                                                              self.PRECISIONS[precision]))

    SCATTER_MODELS = {"exact": _native.SCATTER_EXACT, "surrogate": _native.SCATTER_SURROGATE,
                      "none": _native.SCATTER_NONE,
                      "surrogate_coarse": _native.SCATTER_SURROGATE_COARSE}

    def set_scatter_model(self, model="exact", surrogate: "Surrogate | None" = None):
        """Scatter part of the rows: 'exact' (the single-scatter sum),
        'surrogate' (the learned network at every voxel, which must stay
        alive while used), 'surrogate_coarse' (the network on a
        half-resolution grid of emission positions, interpolated) or 'none'
        (unscattered paths only)."""
        ptr = surrogate._s if surrogate is not None else None
        _native.check(_native.load().lm_set_scatter_model(self._h, self.SCATTER_MODELS[model], ptr))
        self._surrogate_ref = surrogate

    def set_coarse_stride(self, stride: int = 2):
        """Node spacing (2, 3 or 4 pixels) of the 'surrogate_coarse' model."""
        _native.check(_native.load().lm_set_coarse_stride(self._h, int(stride)))

    def surrogate_samples(self, events: DeviceEvents, n, seed=0, stream=None):
        """n training samples (x [n, 32], target [n]) for the surrogate: random
        (event, voxel, line) with the exact ln(S_w + 1e-8) as target."""
        torch = _torch()
        x = torch.empty((int(n), Surrogate.N_IN), dtype=torch.float32, device="cuda")
        t = torch.empty(int(n), dtype=torch.float32, device="cuda")
        ev = events.struct()
        _native.check(_native.load().lm_surrogate_sample(
            self._h, ctypes.byref(ev), int(n), ctypes.c_uint64(seed), ctypes.c_void_p(x.data_ptr()),
            ctypes.c_void_p(t.data_ptr()), _stream(stream)))
        return x, t

    def profile_enable(self, on=True):
        _native.check(_native.load().lm_profile_enable(self._h, 1 if on else 0))

    def profile_read(self) -> dict:
        out = (ctypes.c_double * 5)()
        _native.check(_native.load().lm_profile_read(self._h, out))
        return {"ms": out[0], "launches": int(out[1]), "terms": out[2], "elements": out[3],
                "kernels": int(out[4])}


class Surrogate:
    """The learned single-scatter surrogate (an ``lm_surrogate``): an MLP
    32 -> 128 -> 128 -> 128 -> 1 with GELU, BF16 tensor-core kernels and FP32
    master parameters."""

    N_IN = 32

    def __init__(self, seed=0):
        lib = _native.load()
        s = ctypes.c_void_p()
        _native.check(lib.lm_surrogate_create(ctypes.c_uint64(seed), ctypes.byref(s)))
        self._s = s
        self.n_params = int(lib.lm_surrogate_param_count())

    def _check_inputs(self, x, target=None):
        """x: [rows, 32] float32 CUDA rows; target: one float32 per row."""
        torch = _torch()
        _require_cuda(x, "x", torch.float32)
        if x.dim() != 2 or x.shape[1] != self.N_IN:
            raise ValueError(f"x must have shape [rows, {self.N_IN}], not {tuple(x.shape)}")
        if target is not None:
            _require_cuda(target, "target", torch.float32, numel=x.shape[0])

    def close(self):
        if getattr(self, "_s", None) is not None and self._s.value:
            _native.load().lm_surrogate_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _native.check(_native.load().lm_surrogate_get_params(self._s, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _native.check(_native.load().lm_surrogate_set_params(self._s, p.ctypes.data_as(ctypes.c_void_p)))

    def forward(self, x, stream=None):
        torch = _torch()
        x = x.to(device="cuda", dtype=torch.float32).contiguous()
        self._check_inputs(x)
        out = torch.empty(x.shape[0], dtype=torch.float32, device="cuda")
        _native.check(_native.load().lm_surrogate_forward(self._s, ctypes.c_void_p(x.data_ptr()),
                                                          int(x.shape[0]),
                                                          ctypes.c_void_p(out.data_ptr()),
                                                          _stream(stream)))
        return out

    def gradient(self, x, target, weight=None, stream=None):
        """(grad [n_params] float32 CUDA tensor, weighted mean squared error)."""
        torch = _torch()
        x = x.to(device="cuda", dtype=torch.float32).contiguous()
        target = target.to(device="cuda", dtype=torch.float32).contiguous()
        self._check_inputs(x, target)
        if weight is not None:
            weight = weight.to(device="cuda", dtype=torch.float32).contiguous()
            _require_cuda(weight, "weight", torch.float32, numel=x.shape[0])
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        _native.check(_native.load().lm_surrogate_gradient(
            self._s, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
            ctypes.c_void_p(weight.data_ptr()) if weight is not None else None,
            int(x.shape[0]), ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss), _stream(stream)))
        return g, loss.value

    def train(self, x, target, steps, batch=4096, lr=1e-3, seed=0, weight_power=0.0,
              record_loss=True, stream=None):
        """Adam on minibatches drawn from (x, target), each sample weighted
        by exp(weight_power (t - max t)).  Returns the loss of every
        minibatch before its update (record_loss; this synchronises each
        step), else None."""
        torch = _torch()
        x = x.to(device="cuda", dtype=torch.float32).contiguous()
        target = target.to(device="cuda", dtype=torch.float32).contiguous()
        self._check_inputs(x, target)
        hist = np.zeros(int(steps), dtype=np.float64) if record_loss else None
        _native.check(_native.load().lm_surrogate_train(
            self._s, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(target.data_ptr()),
            int(x.shape[0]) if x.dim() else 0, int(steps), int(batch), ctypes.c_float(lr),
            ctypes.c_float(weight_power), ctypes.c_uint64(seed),
            hist.ctypes.data_as(ctypes.c_void_p) if hist is not None else None, _stream(stream)))
        return hist
