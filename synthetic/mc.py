"""Seeded Monte-Carlo list-mode event generator (stand-in for the paper's MC).

The paper generates its list-mode data with an in-house Monte-Carlo code that
lets photons scatter at most once (Sec. "SPECT simulation").  That code is
not available, so this module is an independent analog photon-transport
simulation of the same 2-D acquisition, used only to make realistic inputs:

* a decay is drawn from the true activity map, uniformly inside its pixel;
  its line is drawn from the yields and its detector angle uniformly;
* the photon either goes straight to the detector (primary) or leaves in a
  uniform in-plane direction, interacts after an exponentially distributed
  optical depth, Compton-scatters into the detector direction with the
  in-plane Klein-Nishina shape as acceptance, and loses energy by the Compton
  formula (forced detection with rejection, so every accepted history is an
  unweighted event);
* attenuation along every leg is marched through the density map in small
  steps;
* the detected position is blurred by a Gaussian whose FWHM grows linearly
  with depth and binned; the energy is blurred by the detector resolution and
  events outside every energy window are dropped.

Every random number comes from numpy's Philox counter-based generator with the
given seed.  Nothing here is shared with the reconstruction code: this module
has its own attenuation-curve interpolation, marching and physics constants,
and it evaluates no system-matrix element.
"""
from __future__ import annotations

import hashlib
import math
import os
from dataclasses import dataclass

import numpy as np

from .presets import Scenario

ME_C2_KEV = 510.99895
FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


@dataclass
class EventList:
    angle: np.ndarray    # uint16
    bin: np.ndarray      # uint16
    energy: np.ndarray   # float32 keV
    origin: np.ndarray   # int32 pixel index of the decay (diagnostic only)
    line: np.ndarray     # uint8 emission line (diagnostic only)
    scattered: np.ndarray  # bool (diagnostic only)

    def __len__(self) -> int:
        return int(self.angle.shape[0])

    def subset(self, idx) -> "EventList":
        return EventList(self.angle[idx], self.bin[idx], self.energy[idx],
                         self.origin[idx], self.line[idx], self.scattered[idx])


def _mu_water(sc: Scenario, e_kev):
    """Water attenuation (1/cm), linear between knots, end segments extended."""
    ek = np.asarray(sc.knot_keV, dtype=np.float64)
    mk = np.asarray(sc.mu_water_cm, dtype=np.float64)
    e = np.asarray(e_kev, dtype=np.float64)
    if ek.size == 1:
        return np.full_like(e, mk[0])
    seg = np.clip(np.searchsorted(ek, e, side="right") - 1, 0, ek.size - 2)
    slope = (mk[seg + 1] - mk[seg]) / (ek[seg + 1] - ek[seg])
    return mk[seg] + slope * (e - ek[seg])


def _kn_shape(cos_t, e_kev):
    """Klein-Nishina angular shape (E'/E)^2 (E'/E + E/E' - sin^2)."""
    ratio = 1.0 / (1.0 + (e_kev / ME_C2_KEV) * (1.0 - cos_t))
    return ratio * ratio * (ratio + 1.0 / ratio - (1.0 - cos_t * cos_t))


def _kn_plane_integral(e_kev: float) -> float:
    th = np.linspace(0.0, 2.0 * np.pi, 20001)
    f = _kn_shape(np.cos(th), e_kev)
    return float(np.sum((f[1:] + f[:-1]) * 0.5) * (th[1] - th[0]))


class _Marcher:
    """Midpoint-rule line integrals of the density map, step ``ds`` cm."""

    def __init__(self, sc: Scenario, rho: np.ndarray, steps_per_pixel: int = 4):
        self.n = sc.n
        self.h = sc.pixel_cm
        self.half = sc.length_cm / 2.0
        self.rho = np.concatenate([rho.reshape(-1).astype(np.float64), [0.0]])
        self.ds = self.h / steps_per_pixel

    def _lookup(self, x, y):
        ix = np.floor((x + self.half) / self.h).astype(np.int64)
        iy = np.floor((y + self.half) / self.h).astype(np.int64)
        ok = (ix >= 0) & (ix < self.n) & (iy >= 0) & (iy < self.n)
        idx = np.where(ok, iy * self.n + ix, self.n * self.n)
        return self.rho[idx]

    def exit_distance(self, x, y, dx, dy):
        """Distance from (x, y) inside the square to its boundary along (dx, dy)."""
        big = 1e30
        with np.errstate(divide="ignore", invalid="ignore"):
            tx = np.where(dx > 0, (self.half - x) / dx,
                          np.where(dx < 0, (-self.half - x) / dx, big))
            ty = np.where(dy > 0, (self.half - y) / dy,
                          np.where(dy < 0, (-self.half - y) / dy, big))
        return np.maximum(np.minimum(tx, ty), 0.0)

    def integral(self, x, y, dx, dy):
        """Integral of rho from (x, y) to the edge of the image along (dx, dy)."""
        total = np.zeros_like(x)
        length = self.exit_distance(x, y, dx, dy)
        t = np.zeros_like(x)
        active = np.nonzero(length > 0)[0]
        while active.size:
            step = np.minimum(self.ds, length[active] - t[active])
            mid = t[active] + 0.5 * step
            total[active] += step * self._lookup(x[active] + mid * dx[active],
                                                 y[active] + mid * dy[active])
            t[active] += step
            active = active[t[active] < length[active] - 1e-12]
        return total

    def interaction(self, x, y, dx, dy, mu, tau_target):
        """Distance at which the optical depth mu*rho reaches ``tau_target``.

        Returns (hit, distance); ``hit`` is False for photons that leave the
        image first.
        """
        length = self.exit_distance(x, y, dx, dy)
        t = np.zeros_like(x)
        tau = np.zeros_like(x)
        hit = np.zeros(x.shape, dtype=bool)
        dist = np.zeros_like(x)
        active = np.nonzero(length > 0)[0]
        while active.size:
            step = np.minimum(self.ds, length[active] - t[active])
            mid = t[active] + 0.5 * step
            r = self._lookup(x[active] + mid * dx[active], y[active] + mid * dy[active])
            dtau = mu[active] * r * step
            cross = tau[active] + dtau >= tau_target[active]
            if np.any(cross):
                ia = active[cross]
                rate = mu[ia] * r[cross]
                dist[ia] = t[ia] + (tau_target[ia] - tau[ia]) / rate
                hit[ia] = True
            tau[active] += dtau
            t[active] += step
            keep = (~cross) & (t[active] < length[active] - 1e-12)
            active = active[keep]
        return hit, dist


def _simulate_chunk(sc: Scenario, rho, act_cdf, marcher, rng, m, z_plane):
    n, h, half = sc.n, sc.pixel_cm, sc.length_cm / 2.0
    n_lines = len(sc.line_keV)
    line_e = np.asarray(sc.line_keV, dtype=np.float64)
    yields = np.asarray(sc.yields, dtype=np.float64)
    yields = yields / yields.sum()

    q = np.searchsorted(act_cdf, rng.random(m), side="right").astype(np.int64)
    q = np.minimum(q, n * n - 1)
    ix, iy = q % n, q // n
    x = (ix + rng.random(m) - n / 2.0) * h
    y = (iy + rng.random(m) - n / 2.0) * h
    w = np.searchsorted(np.cumsum(yields), rng.random(m), side="right")
    w = np.minimum(w, n_lines - 1)
    a = rng.integers(0, sc.n_angles, size=m)
    th = 2.0 * np.pi * a / sc.n_angles
    nx, ny = np.cos(th), np.sin(th)
    e0 = line_e[w]
    mu0 = _mu_water(sc, e0)

    # Proposal split between primary and scattered histories, chosen so that
    # accepted primaries and scatters come out in their physical ratio.
    k_max = 2.0
    p_prim = z_plane[w] / (z_plane[w] + 2.0 * np.pi * k_max)
    prim = rng.random(m) < p_prim

    keep = np.zeros(m, dtype=bool)
    ex, ey, eng = x.copy(), y.copy(), e0.copy()

    ip = np.nonzero(prim)[0]
    if ip.size:
        tau = mu0[ip] * marcher.integral(x[ip], y[ip], nx[ip], ny[ip])
        keep[ip] = rng.random(ip.size) < np.exp(-tau)

    isc = np.nonzero(~prim)[0]
    if isc.size:
        phi = rng.uniform(0.0, 2.0 * np.pi, isc.size)
        dx, dy = np.cos(phi), np.sin(phi)
        tau_t = -np.log1p(-rng.random(isc.size))
        hit, dist = marcher.interaction(x[isc], y[isc], dx, dy, mu0[isc], tau_t)
        sx = x[isc] + dist * dx
        sy = y[isc] + dist * dy
        cos_t = dx * nx[isc] + dy * ny[isc]
        acc = hit & (rng.random(isc.size) * k_max < _kn_shape(cos_t, e0[isc]))
        e1 = e0[isc] / (1.0 + (e0[isc] / ME_C2_KEV) * (1.0 - cos_t))
        surv = np.zeros(isc.size)
        ia = np.nonzero(acc)[0]
        if ia.size:
            mu1 = _mu_water(sc, e1[ia])
            surv[ia] = np.exp(-mu1 * marcher.integral(sx[ia], sy[ia], nx[isc][ia], ny[isc][ia]))
        acc &= rng.random(isc.size) < surv
        keep[isc] = acc
        ex[isc], ey[isc], eng[isc] = sx, sy, e1

    # Detector response: depth-dependent collimator blur, then binning.
    depth = sc.detector_radius_cm - (ex * nx + ey * ny)
    sig_c = (sc.coll_fwhm0_cm + sc.coll_fwhm_slope * depth) / FWHM_PER_SIGMA
    u = (-ex * ny + ey * nx) + sig_c * rng.standard_normal(m)
    bw = sc.bin_width_cm
    b = np.floor((u + 0.5 * sc.n_bins * bw) / bw)
    keep &= (b >= 0) & (b < sc.n_bins)
    # Energy resolution: FWHM/E = frac * (E/E_ref)^exponent.
    sig_e = sc.fwhm_frac * eng * (eng / sc.e_ref_keV) ** sc.fwhm_exponent / FWHM_PER_SIGMA
    e_hat = (eng + sig_e * rng.standard_normal(m)).astype(np.float32)
    inwin = np.zeros(m, dtype=bool)
    for lo, hi in sc.windows:
        inwin |= (e_hat >= np.float32(lo)) & (e_hat < np.float32(hi))
    keep &= inwin
    sel = np.nonzero(keep)[0]
    return EventList(a[sel].astype(np.uint16), b[sel].astype(np.uint16), e_hat[sel],
                     q[sel].astype(np.int32), w[sel].astype(np.uint8), ~prim[sel])


CHUNK_PHOTONS = 200_000       # candidate decays per chunk


def _chunk(args):
    """Chunk ``i`` of a simulation: its own Philox stream (the seed's stream
    jumped i times), so the event list depends on the seed alone, however
    the chunks are spread over processes."""
    sc, act, seed, i = args
    ph = sc.make_phantom()
    cdf = np.cumsum(act)
    cdf = cdf / cdf[-1]
    marcher = _Marcher(sc, ph.rho)
    z_plane = np.array([_kn_plane_integral(e) for e in sc.line_keV])
    rng = np.random.Generator(np.random.Philox(seed).jumped(i))
    return _simulate_chunk(sc, ph.rho, cdf, marcher, rng, CHUNK_PHOTONS, z_plane)


def _pool_map(fn, tasks, processes):
    """fn over tasks in a pool of fresh interpreters (spawn).  The pool starts
    with an empty stand-in for __main__, so the workers import only this
    module and never re-run the caller's script (whose top level may itself
    call simulate)."""
    import multiprocessing as mp
    import sys
    import types
    main = sys.modules.get("__main__")
    sys.modules["__main__"] = types.ModuleType("__main__")
    try:
        pool = mp.get_context("spawn").Pool(processes)
    finally:
        if main is not None:
            sys.modules["__main__"] = main
    with pool:
        return pool.map(fn, tasks)


def _workers() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 32))


def simulate(sc: Scenario, n_events: int | None = None, seed: int | None = None,
             activity: np.ndarray | None = None, workers: int | None = None) -> EventList:
    """Draw ``n_events`` list-mode events (default: the scenario's count/seed).

    Chunks of CHUNK_PHOTONS candidate decays are simulated in order and
    concatenated; with more than a few chunks they run in a pool of worker
    processes, which changes nothing in the result."""
    n_events = sc.n_events if n_events is None else int(n_events)
    seed = sc.seed if seed is None else int(seed)
    ph = sc.make_phantom()
    act = ph.activity if activity is None else np.asarray(activity, dtype=np.float64)
    act = np.asarray(act, dtype=np.float64).reshape(-1)
    parts = [_chunk((sc, act, seed, 0))]
    total = len(parts[0])
    i = 1
    if total < n_events:
        per_chunk = max(total, 1)
        n_more = int(np.ceil((n_events - total) / per_chunk * 1.05)) + 1
        workers = _workers() if workers is None else int(workers)
        if n_more >= 3 and workers > 1:
            more = _pool_map(_chunk, [(sc, act, seed, i + k) for k in range(n_more)],
                             min(workers, n_more))
            parts += more
            total += sum(len(p) for p in more)
            i += n_more
    while total < n_events:
        ev = _chunk((sc, act, seed, i))
        parts.append(ev)
        total += len(ev)
        i += 1
    # keep whole chunks in order, then cut: the result depends only on the seed
    kept, cum = [], 0
    for p in parts:
        kept.append(p)
        cum += len(p)
        if cum >= n_events:
            break
    return EventList(*[np.concatenate([getattr(p, f) for p in kept])[:n_events]
                       for f in ("angle", "bin", "energy", "origin", "line", "scattered")])


def _cache_dir() -> str:
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return os.environ.get("LMMEW_EVENT_CACHE", os.path.join(root, "_cache"))


def simulate_cached(sc: Scenario, n_events: int | None = None,
                    seed: int | None = None) -> EventList:
    """``simulate`` with an on-disk cache keyed by the scenario, count and seed."""
    n_events = sc.n_events if n_events is None else int(n_events)
    seed = sc.seed if seed is None else int(seed)
    key = hashlib.sha1(repr((sc, n_events, seed, "mc-v2")).encode()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"events_{sc.name}_{n_events}_{seed}_{key}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return EventList(z["angle"], z["bin"], z["energy"], z["origin"], z["line"],
                         z["scattered"])
    ev = simulate(sc, n_events, seed)
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, angle=ev.angle, bin=ev.bin, energy=ev.energy, origin=ev.origin,
                 line=ev.line, scattered=ev.scattered)
        os.replace(tmp, path)
    except OSError:
        pass
    return ev
