"""The paper's figures of merit (Sec. "Figure of merit for evaluation"),
pinned to hand-computed values, and the event selections of the comparison
methods.  CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2305_17111_gb300 import studies
from synthetic import preset, simulate


def test_enrmse_bias_std_hand_values():
    truth = np.array([[10.0, 4.0]])                       # S = 1, K = 2
    est = np.array([[[11.0, 4.0], [9.0, 5.0], [12.0, 3.0]]])   # N = 3
    # lesion 0: errors 1, -1, 2 -> rmse sqrt(6/3) = sqrt 2 -> /10
    # lesion 1: errors 0, 1, -1 -> rmse sqrt(2/3) -> /4
    np.testing.assert_allclose(studies.ensemble_nrmse(truth, est),
                               [math.sqrt(2) / 10, math.sqrt(2 / 3) / 4])
    np.testing.assert_allclose(studies.ensemble_bias(truth, est), [2 / 3 / 10, 0.0], atol=1e-15)
    # sample std with N-1: lesion 0 values 11, 9, 12 -> mean 32/3
    sd0 = math.sqrt(((11 - 32 / 3) ** 2 + (9 - 32 / 3) ** 2 + (12 - 32 / 3) ** 2) / 2)
    np.testing.assert_allclose(studies.ensemble_std(truth, est), [sd0 / 10, 1.0 / 4])


def test_perfect_estimates_and_average_over_objects():
    truth = np.array([[2.0], [8.0]])                       # S = 2
    est = np.stack([np.full((5, 1), 2.0), np.full((5, 1), 8.0)])
    assert studies.ensemble_nrmse(truth, est)[0] == 0.0
    assert studies.ensemble_bias(truth, est)[0] == 0.0
    # a 10 % high estimate on one object and exact on the other: mean 5 %
    est2 = est.copy()
    est2[0] *= 1.1
    assert studies.ensemble_bias(truth, est2)[0] == pytest.approx(0.05)
    assert studies.ensemble_nrmse(truth, est2)[0] == pytest.approx(0.05)


def test_method_event_selection():
    sc = preset("paper_study")
    ev = simulate(sc, n_events=2000)
    mew = studies.select(ev, studies.METHODS[0].windows)
    sew = studies.select(ev, studies.METHODS[1].windows)
    binned = studies.select(ev, studies.METHODS[2].windows, studies.METHODS[2].fixed_energy)
    assert len(mew) == len(ev)                 # the generator already cuts to the windows
    assert len(sew) == len(binned) < len(mew)
    assert np.all((sew.energy >= 68.0) & (sew.energy < 102.0))
    assert np.all(binned.energy == np.float32(85.0))
    np.testing.assert_array_equal(sew.bin, binned.bin)
