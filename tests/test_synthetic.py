"""The seeded input generators (CPU): the Monte-Carlo event list depends on
the seed alone -- not on how its chunks are spread over processes -- and has
the paper's structure (photopeaks plus a Compton continuum inside the window)."""
from __future__ import annotations

import numpy as np
import pytest

from synthetic import preset, simulate


def test_event_list_independent_of_worker_count():
    sc = preset("lmmew_32")
    a = simulate(sc, n_events=130_000, seed=3, workers=1)
    b = simulate(sc, n_events=130_000, seed=3, workers=3)
    for f in ("angle", "bin", "energy", "origin", "line", "scattered"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = simulate(sc, n_events=130_000, seed=4, workers=1)
    assert not np.array_equal(a.energy, c.energy)


def test_event_ranges_and_spectrum():
    sc = preset("lmmew_32")
    ev = simulate(sc, n_events=40_000, seed=5)
    assert len(ev) == 40_000
    assert ev.angle.max() < sc.n_angles and ev.bin.max() < sc.n_bins
    assert ev.energy.min() >= 50.0 and ev.energy.max() < 300.0
    # primaries cluster at their line (within 3 FWHM); scattered events lose energy
    prim = ~ev.scattered
    e0 = np.asarray(sc.line_keV)[ev.line[prim]]
    fwhm = 0.10 * np.sqrt(140.0 * e0)
    assert np.mean(np.abs(ev.energy[prim] - e0) < 3 * fwhm) > 0.99
    sca = ev.scattered
    e0s = np.asarray(sc.line_keV)[ev.line[sca]]
    assert np.mean(ev.energy[sca] < e0s + 3 * 0.10 * np.sqrt(140.0 * e0s)) > 0.99
    assert 0.05 < sca.mean() < 0.8


def test_pooled_generation_from_an_unguarded_script(tmp_path):
    """A script without a main guard may call simulate at its top level: the
    worker processes must not re-run it."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "top_level.py"
    script.write_text(
        "import sys\n"
        f"sys.path.insert(0, {root!r})\n"
        "from synthetic import preset, simulate\n"
        "ev = simulate(preset('lmmew_32'), n_events=130_000, seed=3, workers=2)\n"
        "print('events', len(ev))\n")
    out = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "events 130000" in out.stdout


def test_torch_monte_carlo_matches_numpy_monte_carlo():
    """The torch port of the Monte-Carlo (used for large event pools on the
    GPU) draws from the same distribution as synthetic.mc: two-sample
    chi-square tests on angle, bin and energy-band histograms of 20 000
    events each, and the same scattered fraction within 2 percentage
    points; the same seed gives the same events."""
    pytest.importorskip("torch")
    from scipy import stats
    from synthetic import mc_torch
    sc = preset("small_24")
    ev_t = mc_torch.simulate(sc, 20000, seed=5, device="cpu", batch=200000)
    ev_n = simulate(sc, 20000, seed=5)
    assert len(ev_t) == 20000
    for f, k in ((lambda e: e.angle, sc.n_angles), (lambda e: e.bin, sc.n_bins)):
        a, b = np.bincount(f(ev_t), minlength=k), np.bincount(f(ev_n), minlength=k)
        m = (a + b) > 0
        assert stats.chi2_contingency(np.vstack([a[m], b[m]]))[1] > 1e-3
    bands = np.array([50.0, 75.0, 110.0, 200.0, 300.0])
    a, b = np.histogram(ev_t.energy, bands)[0], np.histogram(ev_n.energy, bands)[0]
    assert stats.chi2_contingency(np.vstack([a, b]))[1] > 1e-3
    assert abs(ev_t.scattered.mean() - ev_n.scattered.mean()) < 0.02
    again = mc_torch.simulate(sc, 5000, seed=5, device="cpu", batch=200000)
    assert np.array_equal(again.energy, ev_t.energy[:5000])
