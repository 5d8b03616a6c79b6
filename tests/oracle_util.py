"""Helpers for building small oracle models in tests."""
from __future__ import annotations

import os

import numpy as np

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            vals = []
            for p in parts[1:]:
                try:
                    vals.append(float(p))
                except ValueError:
                    break
            out[parts[0]] = vals
    return out


def small_model(n=8, pixel_cm=2.0, n_angles=8, n_bins=12, scatter_n=0, rho=None,
                support=None, lines=(82.0, 154.0, 270.0), yields=(0.6, 0.2, 0.2),
                windows=((50.0, 300.0),), knots=(82.0, 154.0, 270.0),
                mu=(0.184, 0.148, 0.121), fwhm0=0.3, slope=0.02, scan_time=1.0,
                bin_cm=0.0, r_det_cm=0.0, fwhm_frac=0.10, e_ref=140.0, expo=-0.5):
    if rho is None:
        rho = np.ones((n, n), dtype=np.float32)
    rho = np.asarray(rho, dtype=np.float32).reshape(n, n)
    if support is None:
        support = np.ones((n, n), dtype=bool)
    return oracle.Model(n=n, pixel_cm=pixel_cm, n_angles=n_angles, n_bins=n_bins,
                        bin_cm=bin_cm, r_det_cm=r_det_cm, coll_fwhm0_cm=fwhm0,
                        coll_fwhm_slope=slope, scan_time=scan_time, rho=rho, knot_keV=knots,
                        mu_water_cm=mu, scatter_n=scatter_n, line_keV=lines, yields=yields,
                        fwhm_frac=fwhm_frac, e_ref_keV=e_ref, fwhm_exponent=expo,
                        windows=windows, support=support)


def events_of(angle, bin_, energy) -> synthetic.EventList:
    a = np.asarray(angle, dtype=np.uint16)
    k = a.shape[0]
    return synthetic.EventList(a, np.asarray(bin_, dtype=np.uint16),
                               np.asarray(energy, dtype=np.float32),
                               np.zeros(k, np.int32), np.zeros(k, np.uint8),
                               np.zeros(k, bool))


def coarse_interpolation(pix, n, stride=2):
    """[nq][nq] interpolation of the coarse-grid surrogate, restated from its
    definition: voxel (ix, iy) takes the bilinear weights of the corners
    (ix - ix % s, iy - iy % s) .. (+s, +s) that lie in the support (s the
    node stride), renormalised to sum 1; with no such corner it is its own
    node."""
    q_of = {int(p): q for q, p in enumerate(pix)}
    M = np.zeros((len(pix), len(pix)))
    s = int(stride)
    for q, p in enumerate(pix):
        ix, iy = int(p) % n, int(p) // n
        x0, y0 = ix - ix % s, iy - iy % s
        tx, ty = (ix - x0) / float(s), (iy - y0) / float(s)
        corners = [(x0, y0, (1 - tx) * (1 - ty)), (x0 + s, y0, tx * (1 - ty)),
                   (x0, y0 + s, (1 - tx) * ty), (x0 + s, y0 + s, tx * ty)]
        keep = [(q_of[cy * n + cx], w) for cx, cy, w in corners
                if w > 0 and cx < n and cy < n and (cy * n + cx) in q_of]
        if not keep:
            M[q, q] = 1.0
        else:
            tot = sum(w for _, w in keep)
            for qq, w in keep:
                M[q, qq] += w / tot
    return M
