"""Model-consistent list-mode event sampler (test infrastructure).

Draws events whose distribution is exactly the path model's event density
(Eq. Aj_expansion with the path sensitivities of Eq. s_p): an event of
detector angle a, bin b and recorded energy E_hat arises with probability
proportional to sum_q lambda_q a(a, b, E_hat; q) over the windows.  It
follows the model's hierarchy, with the oracle's own path sensitivities,
detector masses and window masses:

  1. a path P = (voxel q, line w, unscattered or scattered at point p) of
     angle a with weight
        lambda_q alpha_w s(P, E_0^w) D(u_P, sigma_P) Pi(E_P),
     D the collimator mass that lands on the detector, Pi the energy mass
     inside the windows, E_P the photon energy reaching the detector
     (E_0^w, or the Compton energy after the scatter);
  2. a bin b with probability C(b | u_P, sigma_P) / D;
  3. a recorded energy from the energy-resolution Gaussian at E_P,
     truncated to the windows (drawn again until it lies in one).

Every random number comes from numpy's Philox generator with the given
seed.  Like the rest of ``oracle``, only tests and the benchmark's CPU leg
may use it.  It is pinned by a chi-square test of its histograms over
(angle, bin, energy band) against the expectation the oracle's rows give
(tests/test_oracle_sampler.py).
"""
from __future__ import annotations

import numpy as np

from . import Model


def _masses(model: Model, paths: dict, lines, windows_fn):
    """Detector masses of voxels and scatter points, and window masses of
    every path's detected energy."""
    dmass = np.vectorize(model.detector_mass)
    d_q = dmass(paths["u_q"], paths["sig_q"])
    d_p = dmass(paths["u_p"], paths["sig_p"]) if paths["u_p"].size else paths["u_p"]
    pi_line = np.array([windows_fn(e) for e in lines])
    pi_scat = np.vectorize(windows_fn)(paths["e_scat"]) if paths["e_scat"].size else paths["e_scat"]
    return d_q, d_p, pi_line, pi_scat


def sample_events(model: Model, activity, n_events: int, seed: int):
    """n_events events (angle u16, bin u16, energy f32) drawn from the path
    model for the emission image ``activity`` (n*n, raster order)."""
    p = model.params
    W, A, B = p.n_lines, model.n_angles, p.n_bins
    lines = np.array([p.line_e[w] for w in range(W)])
    alpha = np.array([p.line_yield[w] for w in range(W)])
    win = [(p.win_lo[k], p.win_hi[k]) for k in range(p.n_windows)]
    lam = np.asarray(activity, dtype=np.float64).reshape(-1)[model.voxel_pixels]
    rng = np.random.Generator(np.random.Philox(seed))

    per_angle = []
    totals = np.zeros(A)
    for a in range(A):
        paths = model.angle_paths(a)
        d_q, d_p, pi_line, pi_scat = _masses(model, paths, lines, model.window_mass)
        w_prim = (lam[None, :] * alpha[:, None] * paths["s_prim"] * d_q[None, :]
                  * pi_line[:, None])                                   # [W, nq]
        w_scat = (lam[None, :, None] * alpha[:, None, None] * paths["s_scat"]
                  * d_p[None, None, :] * pi_scat)                       # [W, nq, np]
        weights = np.concatenate([w_prim[:, :, None], w_scat], axis=2).reshape(-1)
        per_angle.append((paths, weights))
        totals[a] = weights.sum()

    counts = rng.multinomial(n_events, totals / totals.sum())
    out_a, out_b, out_e = [], [], []
    nq, npt = model.nq, model.np_scatter
    for a in range(A):
        k = int(counts[a])
        if k == 0:
            continue
        paths, weights = per_angle[a]
        cdf = np.cumsum(weights)
        idx = np.searchsorted(cdf, rng.random(k) * cdf[-1], side="right")
        idx = np.minimum(idx, weights.size - 1)
        w, rest = np.divmod(idx, nq * (npt + 1))
        q, j = np.divmod(rest, npt + 1)
        prim = j == 0
        pt = np.maximum(j - 1, 0)
        u = np.where(prim, paths["u_q"][q], paths["u_p"][pt] if npt else 0.0)
        sig = np.where(prim, paths["sig_q"][q], paths["sig_p"][pt] if npt else 1.0)
        e_det = np.where(prim, lines[w], paths["e_scat"][w, q, pt] if npt else 0.0)
        # bin: C(b | u, sigma) over the detector, by inverse CDF
        cb = np.array([[model.bin_prob(b, uu, ss) for b in range(B)] for uu, ss in zip(u, sig)])
        cb = np.cumsum(cb, axis=1)
        b = np.array([np.searchsorted(row, r * row[-1], side="right")
                      for row, r in zip(cb, rng.random(k))])
        b = np.minimum(b, B - 1)
        # recorded energy: Gaussian at e_det, truncated to the windows
        sig_e = np.array([model.sigma_e(e) for e in e_det])
        e_hat = np.empty(k)
        todo = np.arange(k)
        while todo.size:
            x = e_det[todo] + sig_e[todo] * rng.standard_normal(todo.size)
            x32 = x.astype(np.float32)
            ok = np.zeros(todo.size, dtype=bool)
            for lo, hi in win:
                ok |= (x32 >= np.float32(lo)) & (x32 < np.float32(hi))
            e_hat[todo[ok]] = x[ok]
            todo = todo[~ok]
        out_a.append(np.full(k, a, dtype=np.uint16))
        out_b.append(b.astype(np.uint16))
        out_e.append(e_hat.astype(np.float32))
    return (np.concatenate(out_a), np.concatenate(out_b), np.concatenate(out_e))
