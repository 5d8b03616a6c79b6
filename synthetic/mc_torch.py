"""The Monte-Carlo event generator of ``synthetic.mc`` on torch tensors.

The same analog photon transport as ``synthetic.mc`` (decay drawn from the
activity map uniformly inside its pixel; primary or scattered history chosen
by the same proposal split; forced detection with rejection on survival and
on the in-plane Klein-Nishina shape; attenuation marched through the density
map at the same midpoint steps; depth-dependent collimator blur, binning,
energy blur and window cut), written with torch operations so that it can
run on a GPU: large event pools (tens of millions of events for batches of
noise realisations) then take seconds instead of many CPU-minutes.

Random numbers come from a torch generator seeded with ``seed`` on the
chosen device (a Philox generator on CUDA devices), so the events depend on
the seed, the device type and the batch size, and differ from
``synthetic.mc``'s for the same seed; both draw independent, identically
distributed events from the same physics.  Nothing here is shared with the
reconstruction code, and it evaluates no system-matrix element.
"""
from __future__ import annotations

import math

import numpy as np

from .mc import ME_C2_KEV, FWHM_PER_SIGMA, EventList, _kn_plane_integral
from .presets import Scenario


def _torch():
    import torch
    return torch


class _Marcher:
    """Midpoint-rule line integrals of the density map, step ``ds`` cm, on
    every photon at once (a photon past its exit takes steps of length 0;
    the march stops once every photon is out)."""

    def __init__(self, sc: Scenario, rho: np.ndarray, device, steps_per_pixel: int = 4):
        torch = _torch()
        self.n = sc.n
        self.h = sc.pixel_cm
        self.half = sc.length_cm / 2.0
        r = np.concatenate([rho.reshape(-1).astype(np.float64), [0.0]])
        self.rho = torch.from_numpy(r).to(device)
        self.ds = self.h / steps_per_pixel
        # the longest chord of the square, in steps
        self.max_steps = int(math.ceil(2.0 * math.sqrt(2.0) * self.half / self.ds)) + 2

    def _lookup(self, x, y):
        torch = _torch()
        ix = torch.floor((x + self.half) / self.h).long()
        iy = torch.floor((y + self.half) / self.h).long()
        ok = (ix >= 0) & (ix < self.n) & (iy >= 0) & (iy < self.n)
        idx = torch.where(ok, iy * self.n + ix, torch.full_like(ix, self.n * self.n))
        return self.rho[idx]

    def exit_distance(self, x, y, dx, dy):
        torch = _torch()
        big = torch.full_like(x, 1e30)
        safe_dx = torch.where(dx != 0, dx, torch.ones_like(dx))
        safe_dy = torch.where(dy != 0, dy, torch.ones_like(dy))
        tx = torch.where(dx > 0, (self.half - x) / safe_dx,
                         torch.where(dx < 0, (-self.half - x) / safe_dx, big))
        ty = torch.where(dy > 0, (self.half - y) / safe_dy,
                         torch.where(dy < 0, (-self.half - y) / safe_dy, big))
        return torch.clamp(torch.minimum(tx, ty), min=0.0)

    def integral(self, x, y, dx, dy):
        torch = _torch()
        total = torch.zeros_like(x)
        length = self.exit_distance(x, y, dx, dy)
        t = torch.zeros_like(x)
        for k in range(self.max_steps):
            step = torch.clamp(torch.clamp(length - t, max=self.ds), min=0.0)
            mid = t + 0.5 * step
            total += step * self._lookup(x + mid * dx, y + mid * dy)
            t += step
            if k % 16 == 15 and not bool((t < length).any()):
                break
        return total

    def interaction(self, x, y, dx, dy, mu, tau_target):
        """(hit, distance) at which the optical depth mu*rho reaches tau_target."""
        torch = _torch()
        length = self.exit_distance(x, y, dx, dy)
        t = torch.zeros_like(x)
        tau = torch.zeros_like(x)
        hit = torch.zeros(x.shape, dtype=torch.bool, device=x.device)
        dist = torch.zeros_like(x)
        for k in range(self.max_steps):
            step = torch.clamp(torch.clamp(length - t, max=self.ds), min=0.0)
            mid = t + 0.5 * step
            r = self._lookup(x + mid * dx, y + mid * dy)
            rate = mu * r
            dtau = rate * step
            cross = (~hit) & (step > 0) & (tau + dtau >= tau_target)
            safe = torch.where(cross, rate, torch.ones_like(rate))
            dist = torch.where(cross, t + (tau_target - tau) / safe, dist)
            hit |= cross
            tau += dtau
            t += step
            if k % 16 == 15 and not bool(((t < length) & ~hit).any()):
                break
        return hit, dist


def _mu_water(sc: Scenario, e, torch):
    ek = torch.tensor(sc.knot_keV, dtype=torch.float64, device=e.device)
    mk = torch.tensor(sc.mu_water_cm, dtype=torch.float64, device=e.device)
    if ek.numel() == 1:
        return torch.full_like(e, float(mk[0]))
    seg = torch.clamp(torch.searchsorted(ek, e, right=True) - 1, 0, ek.numel() - 2)
    slope = (mk[seg + 1] - mk[seg]) / (ek[seg + 1] - ek[seg])
    return mk[seg] + slope * (e - ek[seg])


def _kn_shape(cos_t, e_kev):
    ratio = 1.0 / (1.0 + (e_kev / ME_C2_KEV) * (1.0 - cos_t))
    return ratio * ratio * (ratio + 1.0 / ratio - (1.0 - cos_t * cos_t))


def _simulate_batch(sc, act_cdf, marcher, gen, m, z_plane, device):
    torch = _torch()
    f64 = torch.float64
    n, h = sc.n, sc.pixel_cm
    line_e = torch.tensor(sc.line_keV, dtype=f64, device=device)
    yields = torch.tensor(sc.yields, dtype=f64, device=device)
    ycdf = torch.cumsum(yields / yields.sum(), 0)

    def rand(k):
        return torch.rand(k, generator=gen, dtype=f64, device=device)

    q = torch.clamp(torch.searchsorted(act_cdf, rand(m), right=True), max=n * n - 1)
    ix, iy = q % n, q // n
    x = (ix + rand(m) - n / 2.0) * h
    y = (iy + rand(m) - n / 2.0) * h
    w = torch.clamp(torch.searchsorted(ycdf, rand(m), right=True), max=len(sc.line_keV) - 1)
    a = torch.randint(0, sc.n_angles, (m,), generator=gen, device=device)
    th = 2.0 * math.pi * a.to(f64) / sc.n_angles
    nx, ny = torch.cos(th), torch.sin(th)
    e0 = line_e[w]
    mu0 = _mu_water(sc, e0, torch)

    k_max = 2.0
    zp = z_plane[w]
    p_prim = zp / (zp + 2.0 * math.pi * k_max)
    prim = rand(m) < p_prim

    keep = torch.zeros(m, dtype=torch.bool, device=device)
    ex, ey, eng = x.clone(), y.clone(), e0.clone()
    u_keep = rand(m)   # survival draw of primaries
    # primary histories: survive to the detector along n_a
    ip = torch.nonzero(prim).squeeze(1)
    if ip.numel():
        tau = mu0[ip] * marcher.integral(x[ip], y[ip], nx[ip], ny[ip])
        keep[ip] = u_keep[ip] < torch.exp(-tau)
    # scattered histories: uniform in-plane direction, exponential optical
    # depth, Klein-Nishina acceptance into the detector direction, survival
    isc = torch.nonzero(~prim).squeeze(1)
    phi = rand(m) * (2.0 * math.pi)
    tau_t = -torch.log1p(-rand(m))
    u_kn = rand(m)
    u_surv = rand(m)
    if isc.numel():
        dx, dy = torch.cos(phi[isc]), torch.sin(phi[isc])
        hit, dist = marcher.interaction(x[isc], y[isc], dx, dy, mu0[isc], tau_t[isc])
        sx, sy = x[isc] + dist * dx, y[isc] + dist * dy
        cos_t = dx * nx[isc] + dy * ny[isc]
        e_s = e0[isc]
        acc = hit & (u_kn[isc] * k_max < _kn_shape(cos_t, e_s))
        e1 = e_s / (1.0 + (e_s / ME_C2_KEV) * (1.0 - cos_t))
        ia = torch.nonzero(acc).squeeze(1)
        if ia.numel():
            j = isc[ia]
            surv = torch.exp(-_mu_water(sc, e1[ia], torch) *
                             marcher.integral(sx[ia], sy[ia], nx[j], ny[j]))
            keep[j] = u_surv[j] < surv
        ex[isc], ey[isc], eng[isc] = sx, sy, e1

    depth = sc.detector_radius_cm - (ex * nx + ey * ny)
    sig_c = (sc.coll_fwhm0_cm + sc.coll_fwhm_slope * depth) / FWHM_PER_SIGMA
    u = (-ex * ny + ey * nx) + sig_c * torch.randn(m, generator=gen, dtype=f64, device=device)
    bw = sc.bin_width_cm
    b = torch.floor((u + 0.5 * sc.n_bins * bw) / bw)
    keep &= (b >= 0) & (b < sc.n_bins)
    sig_e = sc.fwhm_frac * eng * (eng / sc.e_ref_keV) ** sc.fwhm_exponent / FWHM_PER_SIGMA
    e_hat = (eng + sig_e * torch.randn(m, generator=gen, dtype=f64, device=device)).float()
    inwin = torch.zeros(m, dtype=torch.bool, device=device)
    for lo, hi in sc.windows:
        inwin |= (e_hat >= lo) & (e_hat < hi)
    keep &= inwin
    sel = torch.nonzero(keep).squeeze(1)
    return (a[sel].to(torch.int32), b[sel].to(torch.int32), e_hat[sel], q[sel].to(torch.int32),
            w[sel].to(torch.uint8), ~prim[sel])


def simulate(sc: Scenario, n_events: int, seed: int, device="cuda", batch: int = 8_000_000,
             activity: np.ndarray | None = None) -> EventList:
    """``n_events`` events drawn in batches of ``batch`` candidate decays,
    kept whole in order and cut at n_events (returned on the host)."""
    torch = _torch()
    ph = sc.make_phantom()
    act = ph.activity if activity is None else activity
    act = np.asarray(act, dtype=np.float64).reshape(-1)
    cdf = np.cumsum(act)
    act_cdf = torch.from_numpy(cdf / cdf[-1]).to(device)
    marcher = _Marcher(sc, ph.rho, device)
    z_plane = torch.tensor([_kn_plane_integral(e) for e in sc.line_keV], dtype=torch.float64,
                           device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    parts, total = [], 0
    while total < n_events:
        out = _simulate_batch(sc, act_cdf, marcher, gen, int(batch), z_plane, device)
        parts.append([t.cpu() for t in out])
        total += int(out[0].numel())
    cols = [torch.cat([p[i] for p in parts])[:n_events].numpy() for i in range(6)]
    return EventList(cols[0].astype(np.uint16), cols[1].astype(np.uint16),
                     cols[2].astype(np.float32), cols[3].astype(np.int32),
                     cols[4].astype(np.uint8), cols[5].astype(bool))
