"""The row kernel's collimator floor, checked on the oracle's path data (CPU).

The CUDA path stores a scatter point's collimator probability for a bin as 0
when it is below 1e-7 of the largest point probability of the same (angle,
bin), and skips those points; the oracle keeps every term.  Here the
single-scatter terms of every event are formed in FP64 from the oracle's
path sensitivities, energies and collimator blurs (the n = 1 paths of
Eq. s_p times the detector response), their sum is checked against the
oracle's own rows, and the part the floor drops is bounded against the
event's whole forward value (primary included).  A floor fixed in absolute
terms fails this on events whose value comes from far-tail points, which is
why the floor is relative to each bin's largest factor."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import special

import oracle
from synthetic import preset, simulate

FLOOR_REL = 1e-7     # the CUDA library's relative floor
BOUND = 2e-7         # largest allowed relative change of an event's forward value


def _scatter_terms(orc, sc, a, b, e_hat, lam, ap, sig):
    """[np] per-point single-scatter terms of one event summed over lines and
    voxels (FP64), and the points' collimator probabilities for bin b."""
    w = sc.bin_width_cm
    lo = -0.5 * sc.n_bins * w + b * w
    hi = lo + w
    s2 = math.sqrt(2.0)
    za = (lo - ap["u_p"]) / (s2 * ap["sig_p"])
    zb = (hi - ap["u_p"]) / (s2 * ap["sig_p"])
    # Gaussian mass of the bin, through erfc on whichever side keeps it exact
    c = np.where(za > 0, 0.5 * (special.erfc(za) - special.erfc(zb)),
                 np.where(zb < 0, 0.5 * (special.erfc(-zb) - special.erfc(-za)),
                          0.5 * (special.erf(zb) - special.erf(za))))
    es = ap["e_scat"]
    g = np.exp(-(e_hat - es) ** 2 / (2 * sig ** 2)) / (math.sqrt(2 * math.pi) * sig)
    alpha = np.asarray(sc.yields, dtype=np.float64)
    per_p = np.einsum("wqp,q->p", alpha[:, None, None] * ap["s_scat"] * g, lam)
    return per_p * c, c


@pytest.mark.parametrize("name", ["tiny_8", "small_16", "small_24"])
def test_relative_collimator_floor_moves_forward_values_below_fp32_rounding(name):
    sc = preset(name)
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc)
    rng = np.random.default_rng(1)
    lam_full = rng.uniform(0.2, 3.0, ph.rho.size) * (ph.rho.reshape(-1) > 0)
    lam = lam_full[orc.voxel_pixels]
    fwd = orc.forward(ev, lam_full)
    worst_abs_floor = 0.0
    checked = 0
    for a in range(sc.n_angles):
        idx = np.nonzero(ev.angle == a)[0]
        if idx.size == 0:
            continue
        ap = orc.angle_paths(a)
        es = ap["e_scat"]
        sig = np.vectorize(orc.sigma_e)(es.reshape(-1)).reshape(es.shape)
        for k, i in enumerate(idx):
            b, e_hat = int(ev.bin[i]), float(ev.energy[i])
            terms, c = _scatter_terms(orc, sc, a, b, e_hat, lam, ap, sig)
            if k == 0:
                # the restatement reproduces the oracle's scatter rows
                ref = sum(orc.scatter_line_row(a, b, e_hat, w) @ lam for w in range(len(sc.yields)))
                assert terms.sum() == pytest.approx(ref, rel=1e-5, abs=1e-300)
            dropped = terms[c < FLOOR_REL * c.max()].sum()
            assert dropped / fwd[i] < BOUND, (a, b, e_hat)
            worst_abs_floor = max(worst_abs_floor, terms[c < 1e-8].sum() / fwd[i])
            checked += 1
    assert checked == len(ev)
    if name == "small_16":
        # an absolute floor of 1e-8 moves one of this case's events by ~7e-5
        assert worst_abs_floor > 1e-5
