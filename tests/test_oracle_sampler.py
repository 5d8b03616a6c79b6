"""The model-consistent event sampler (oracle/sampler.py), pinned by a
chi-square test: histograms of its events over (angle, bin, energy band)
against the expectation sum_q lambda_q integral_band a(a, b, E_hat; q) dE_hat
that the oracle's rows give (Eq. Aj_expansion; composite Simpson in energy).
The sampler draws through path sensitivities, detector masses and window
masses; the expectation goes through the rows' bin probabilities and energy
densities, so a dropped term, a flipped detector axis or a wrong window
truncation on either side makes the test fail.  Cases: one 50-300 keV
window and the paper's three photopeak windows (Sec. SPECT simulation)."""
from __future__ import annotations

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle.sampler import sample_events
from oracle_util import events_of
from synthetic import preset

PAPER_WINDOWS = ((68.0, 102.0), (123.0, 184.0), (243.0, 297.0))


def _bands(windows):
    """Energy bands: each window cut in three (one window: at 75, 110 and
    200 keV around the photopeaks; several: in equal thirds, so that events
    piling up at a window's edges show)."""
    if len(windows) == 1:
        lo, hi = windows[0]
        edges = [lo, 75.0, 110.0, 200.0, hi]
        return list(zip(edges[:-1], edges[1:]))
    out = []
    for lo, hi in windows:
        e = np.linspace(lo, hi, 4)
        out += list(zip(e[:-1], e[1:]))
    return out


def _expected(orc, sc, lam, bands, step=0.25):
    """[A, B, bands] model expectation (unnormalised)."""
    A, B = sc.n_angles, sc.n_bins
    out = np.zeros((A, B, len(bands)))
    for k, (lo, hi) in enumerate(bands):
        m = int(round((hi - lo) / step))
        m += m % 2
        x = np.linspace(lo, hi, m + 1)
        w = np.full(m + 1, 2.0)
        w[1::2] = 4.0
        w[0] = w[-1] = 1.0
        w *= (hi - lo) / m / 3.0
        aa = np.repeat(np.arange(A), B * x.size)
        bb = np.tile(np.repeat(np.arange(B), x.size), A)
        ee = np.tile(x, A * B).astype(np.float32)
        y = orc.forward(events_of(aa, bb, ee), lam).reshape(A, B, x.size)
        out[:, :, k] = (y * w).sum(axis=2)
    return out


@pytest.mark.parametrize("windows", [None, PAPER_WINDOWS])
def test_model_sampler_histograms_match_model_expectation(windows):
    sc = preset("tiny_8")
    if windows is not None:
        sc = sc.with_(windows=windows)
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    lam = ph.activity.reshape(-1).astype(np.float64) * (ph.rho.reshape(-1) > 0)
    a, b, e = sample_events(orc, lam, 100000, seed=12)
    assert a.size == 100000
    inwin = np.zeros(e.size, dtype=bool)
    for lo, hi in sc.windows:
        inwin |= (e >= np.float32(lo)) & (e < np.float32(hi))
    assert inwin.all()
    bands = _bands(sc.windows)
    exp = _expected(orc, sc, lam, bands)
    obs = np.zeros_like(exp)
    for k, (lo, hi) in enumerate(bands):
        sel = (e >= np.float32(lo)) & (e < np.float32(hi))
        np.add.at(obs, (a[sel], b[sel], np.full(sel.sum(), k)), 1.0)
    assert obs.sum() == a.size
    expc = exp / exp.sum() * obs.sum()
    keep = expc >= 5.0
    assert keep.sum() >= 60 and expc[keep].sum() > 0.99 * obs.sum()
    chi2 = float((((obs - expc) ** 2) / expc)[keep].sum())
    dof = int(keep.sum()) - 1
    p = float(stats.chi2.sf(chi2, dof))
    assert p > 1e-3, f"chi2 {chi2:.1f} for {dof} dof, p = {p:.2e}"
