"""EM invariants of the oracle's LM-OSEM (Eq. os-lm-mlem): non-negativity,
support preservation, count preservation per sub-iteration, monotone
log-likelihood for one subset (the EM ascent property), the one-voxel closed
form and resume.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle_util import events_of, small_model
from synthetic import preset, simulate


@pytest.fixture(scope="module")
def small():
    sc = preset("small_16")
    ph = sc.make_phantom()
    m = oracle.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc)
    lam0 = (ph.rho > 0).astype(np.float64).reshape(-1)
    return sc, m, ev, lam0


def _subset(ev, n_sub, s):
    return ev.subset(np.nonzero((ev.angle % n_sub) == s)[0])


def _explicit_subiteration(m, ev, lam, n_sub, s):
    """Eq. os-lm-mlem for subset s written with the separately pinned
    forward projection, back projection and subset sensitivity."""
    sub = _subset(ev, n_sub, s)
    y = m.forward(sub, lam)
    r = np.where(y > 0, 1.0 / np.where(y > 0, y, 1.0), 0.0)
    num = m.backproject(sub, r)
    sens = m.sensitivity(s, n_sub)
    return np.where(sens > 0, lam * num / np.where(sens > 0, sens, 1.0), 0.0)


def test_osem_matches_explicit_forward_backproject_update(small):
    sc, m, ev, lam0 = small
    n_sub = sc.n_subsets
    lam_osem = m.osem(ev, lam0, n_sub, 2)
    lam = lam0.copy()
    for _ in range(2):
        for s in range(n_sub):
            lam = _explicit_subiteration(m, ev, lam, n_sub, s)
    np.testing.assert_allclose(lam_osem, lam, rtol=1e-11, atol=0)


def test_count_preservation_nonnegativity_support(small):
    sc, m, ev, lam0 = small
    n_sub = sc.n_subsets
    lam = lam0.copy()
    for s in range(n_sub):
        lam = _explicit_subiteration(m, ev, lam, n_sub, s)
        js = int(np.sum(ev.angle % n_sub == s))
        # T sum_q lambda_q^new sens_s[q] = J_s after every sub-iteration
        assert float(np.dot(lam, m.sensitivity(s, n_sub))) == pytest.approx(js, rel=1e-12)
        assert np.all(lam >= 0)
        assert np.all(lam[lam0 == 0] == 0)


def test_mlem_loglik_never_decreases(small):
    sc, m, ev, lam0 = small
    lam, ll = m.osem(ev, lam0, 1, 8, want_loglik=True)
    assert np.all(np.diff(ll) >= -1e-12 * np.abs(ll[1:]))
    assert ll[-1] > ll[0]
    assert np.all(lam >= 0)


def test_loglik_value_matches_definition(small):
    sc, m, ev, lam0 = small
    n_sub = sc.n_subsets
    _, ll = m.osem(ev, lam0, n_sub, 1, want_loglik=True)
    sub = _subset(ev, n_sub, 0)
    ref = np.sum(np.log(m.forward(sub, lam0))) - np.dot(lam0, m.sensitivity(0, n_sub))
    assert ll[0] == pytest.approx(ref, rel=1e-12)


def test_one_voxel_mlem_closed_form():
    """One voxel: y_j = a_j lam, so one MLEM step gives lam = J / sens."""
    n = 8
    sup = np.zeros((n, n), bool)
    sup[3, 4] = True
    m = small_model(n=n, support=sup, scatter_n=4)
    rng = np.random.default_rng(0)
    k = 40
    ev = events_of(rng.integers(0, 8, k), rng.integers(2, 10, k), rng.uniform(60, 290, k))
    lam0 = np.zeros(n * n)
    lam0[3 * n + 4] = 0.37
    lam = m.osem(ev, lam0, 1, 1)
    sens = m.sensitivity(-1, 1)
    assert lam[3 * n + 4] == pytest.approx(k / sens[3 * n + 4], rel=1e-13)


def test_resume_continues_the_same_iteration(small):
    sc, m, ev, lam0 = small
    n_sub = sc.n_subsets
    full = m.osem(ev, lam0, n_sub, 2)
    first = m.osem(ev, lam0, n_sub, 1)
    second = m.osem(ev, first, n_sub, 2, start_iter=1)
    np.testing.assert_allclose(full, second, rtol=1e-13, atol=0)
    # resume in the middle of an iteration
    lam = _explicit_subiteration(m, ev, lam0, n_sub, 0)
    rest = m.osem(ev, lam, n_sub, 1, 0, 1)
    np.testing.assert_allclose(m.osem(ev, lam0, n_sub, 1), rest, rtol=1e-12, atol=0)


def test_thread_count_changes_no_result(small):
    """The CPU baseline times the oracle on one thread and on all of them:
    the thread count is a timing control only.  The forward projection is
    the same on one thread as on all, and the count is restored."""
    sc, m, ev, lam0 = small
    n_all = oracle.max_threads()
    y_all = m.forward(ev, lam0)
    oracle.set_threads(1)
    try:
        assert oracle.max_threads() == 1
        y_one = m.forward(ev, lam0)
    finally:
        oracle.set_threads(n_all)
    assert oracle.max_threads() == n_all
    np.testing.assert_array_equal(y_one, y_all)
