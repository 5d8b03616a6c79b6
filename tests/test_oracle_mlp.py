"""Pins of the FP64 surrogate oracle (oracle/mlp.py) against finite
differences, closed forms and the SplitMix64 reference outputs.  CPU only."""
from __future__ import annotations

import os

import numpy as np
import pytest
from scipy import special

from oracle import mlp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _small_params(seed=3, scale=1.0):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed).astype(np.float64) * scale
    # non-zero biases so that every bias path is exercised
    W1, b1, W2, b2, W3, b3, w4, b4 = mlp.unpack(p.copy())
    b1 = rng.normal(0, 0.3, mlp.N_HID)
    b2 = rng.normal(0, 0.3, mlp.N_HID)
    b3 = rng.normal(0, 0.3, mlp.N_HID)
    return mlp.pack(W1, b1, W2, b2, W3, b3, w4, 0.7)


def _data(n=16, seed=5):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 1, (n, mlp.N_IN)), rng.normal(0, 1, n)


# ---------------------------------------------------------------- GELU
def test_gelu_odd_part_identity_and_limits():
    z = np.linspace(-8, 8, 401)
    # tanh is odd, so 0.5 z (1 + t) - 0.5 (-z)(1 - t) = z exactly
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    assert mlp.gelu(0.0) == 0.0
    np.testing.assert_allclose(mlp.gelu(np.array([30.0, 50.0])), [30.0, 50.0], rtol=1e-15)
    np.testing.assert_allclose(mlp.gelu(np.array([-30.0, -50.0])), [0.0, 0.0], atol=1e-300)


def test_gelu_close_to_erf_form():
    # the tanh form approximates z Phi(z) to better than 1e-3 (Hendrycks and Gimpel 2016)
    z = np.linspace(-6, 6, 1201)
    exact = z * 0.5 * (1 + special.erf(z / np.sqrt(2)))
    assert np.max(np.abs(mlp.gelu(z) - exact)) < 1e-3


def test_gelu_grad_central_difference():
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)


# ---------------------------------------------------------------- network
def test_layout():
    assert mlp.N_PARAMS == 128 * 32 + 128 + 2 * (128 * 128 + 128) + 128 + 1 == 37377
    p = np.arange(mlp.N_PARAMS, dtype=np.float64)
    W1, b1, W2, b2, W3, b3, w4, b4 = mlp.unpack(p)
    np.testing.assert_array_equal(mlp.pack(W1, b1, W2, b2, W3, b3, w4, b4), p)
    assert W1[1, 0] == 32 and b4 == mlp.N_PARAMS - 1


def test_gradient_matches_central_differences_in_every_block():
    p = _small_params()
    x, t = _data()
    g, L = mlp.gradient(p, x, t)
    assert L == pytest.approx(mlp.loss(p, x, t), rel=1e-14)
    rng = np.random.default_rng(7)
    blocks = [(mlp.OFF_W1, mlp.OFF_B1), (mlp.OFF_B1, mlp.OFF_W2), (mlp.OFF_W2, mlp.OFF_B2),
              (mlp.OFF_B2, mlp.OFF_W3), (mlp.OFF_W3, mlp.OFF_B3), (mlp.OFF_B3, mlp.OFF_W4),
              (mlp.OFF_W4, mlp.OFF_B4), (mlp.OFF_B4, mlp.N_PARAMS)]
    h = 1e-5
    for lo, hi in blocks:
        for i in rng.choice(np.arange(lo, hi), size=min(12, hi - lo), replace=False):
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            fd = (mlp.loss(pp, x, t) - mlp.loss(pm, x, t)) / (2 * h)
            assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), (lo, i)


def test_output_bias_gradient_closed_form_and_exact_fit():
    p = _small_params()
    x, _ = _data()
    out = mlp.forward(p, x)
    t = out - 0.25                       # residual 0.25 everywhere
    g, L = mlp.gradient(p, x, t)
    assert L == pytest.approx(0.0625, rel=1e-14)
    assert g[mlp.OFF_B4] == pytest.approx(0.5, rel=1e-14)   # d/db4 mean r^2 = 2 mean r
    g0, L0 = mlp.gradient(p, x, out)
    assert L0 == 0.0 and np.all(g0 == 0.0)


def test_zero_hidden_weights_give_constant_output():
    p = _small_params()
    W1, b1, W2, b2, W3, b3, w4, b4 = mlp.unpack(p.copy())
    p0 = mlp.pack(W1, b1, np.zeros_like(W2), b2, W3, b3, w4, b4)
    x, _ = _data()
    out = mlp.forward(p0, x)
    # with W2 = 0 the output no longer depends on x
    np.testing.assert_allclose(out, out[0], rtol=1e-15)


def test_adam_first_step_is_sign_step():
    rng = np.random.default_rng(1)
    p = rng.normal(size=50)
    g = rng.normal(size=50) * 10 ** rng.uniform(-6, 2, 50)
    p1, m1, m2 = mlp.adam_step(p, np.zeros(50), np.zeros(50), g, step=1, lr=1e-3)
    np.testing.assert_allclose(p - p1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-13)
    np.testing.assert_allclose(m2, 0.001 * g * g, rtol=1e-13)


def test_adam_descends_a_quadratic():
    p = np.array([3.0, -2.0])
    m1 = m2 = np.zeros(2)
    for k in range(1, 3001):
        p, m1, m2 = mlp.adam_step(p, m1, m2, 2 * p, step=k, lr=1e-2)
    assert np.all(np.abs(p) < 1e-2)


# ---------------------------------------------------------------- generator
def _golden_splitmix():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            out[int(line[0])] = [int(v, 0) for v in line[1:]]
    return out


def test_splitmix64_reference_outputs():
    for seed, want in _golden_splitmix().items():
        s, got = seed, []
        for _ in want:
            z, s = mlp.splitmix64(s)
            got.append(z)
        assert got == want


def test_init_params_xavier_ranges():
    p = mlp.init_params(42)
    W1, b1, W2, b2, W3, b3, w4, b4 = mlp.unpack(p)
    for W, fi, fo in ((W1, 32, 128), (W2, 128, 128), (W3, 128, 128), (w4, 128, 1)):
        lim = np.sqrt(6.0 / (fi + fo))
        assert np.max(np.abs(W)) <= lim * (1 + 1e-6)
        # uniform on (-lim, lim): variance lim^2 / 3
        assert np.var(W) == pytest.approx(lim * lim / 3, rel=0.25 if W.size < 200 else 0.06)
    assert np.all(b1 == 0) and np.all(b2 == 0) and np.all(b3 == 0) and b4 == -10.0
    assert not np.array_equal(mlp.init_params(1), mlp.init_params(2))


# ---------------------------------------------------------------- weighted loss
def test_weighted_gradient_matches_central_differences():
    p = _small_params(8)
    x, t = _data(24, 9)
    v = np.random.default_rng(3).uniform(0.1, 3.0, 24)
    g, L = mlp.gradient(p, x, t, v)
    assert L == pytest.approx(mlp.loss(p, x, t, v), rel=1e-14)
    rng = np.random.default_rng(11)
    h = 1e-5
    for i in rng.choice(mlp.N_PARAMS, size=40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss(pp, x, t, v) - mlp.loss(pm, x, t, v)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), i
    # unit weights are the unweighted loss
    g1, L1 = mlp.gradient(p, x, t, np.ones(24))
    g0, L0 = mlp.gradient(p, x, t)
    np.testing.assert_array_equal(g1, g0)
    assert L1 == L0


def test_train_weights_are_powers_of_the_scatter_mass():
    S = np.array([1e-3, 1e-4, 1e-6, 0.0, 2e-3])
    t = np.log(S + mlp.EPS_TARGET)
    for power in (0.0, 0.5, 1.0):
        v = mlp.train_weights(t, power)
        assert v.mean() == pytest.approx(1.0, rel=1e-14)
        want = (S + mlp.EPS_TARGET) ** power
        np.testing.assert_allclose(v, want / want.mean(), rtol=1e-12)


# ---------------------------------------------------------------- inputs
def test_compton_kappa_inverts_the_oracles_compton_energy():
    import oracle
    for e0 in (82.0, 154.0, 270.0):
        for c in np.linspace(-1, 1, 9):
            e1 = oracle.compton_energy(e0, c)
            assert mlp.compton_kappa(e1, e0) == pytest.approx(1.0 - c, abs=1e-12)
    assert mlp.compton_kappa(82.0, 82.0) == 0.0


def test_features_scatter_point_geometry():
    """p* lies on the bin's projection line and is seen from the voxel at the
    Compton angle of the recorded energy; the remaining inputs are the stated
    encodings."""
    n, hpx = 16, 1.2
    rho = np.random.default_rng(0).uniform(0.5, 1.5, (n, n))
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(200):
        x, y = rng.uniform(-8, 8, 2)
        th = rng.uniform(0, 2 * np.pi)
        ub = rng.uniform(-9, 9)
        w = int(rng.integers(3))
        e0 = (82.0, 154.0, 270.0)[w]
        e_hat = rng.uniform(0.45, 1.05) * e0
        od = rng.uniform(0, 3, 8)
        f = mlp.features(x, y, th, ub, e_hat, w, e0, od, rho, hpx)
        ca, sa = np.cos(th), np.sin(th)
        assert f[0] == x * 0.05 and f[1] == y * 0.05 and f[2] == ca and f[3] == sa
        assert f[6 + w] == 1.0 and f[6:9].sum() == 1.0
        np.testing.assert_allclose(f[9:17], od * 0.25)
        xp, yp = f[22] / 0.05, f[23] / 0.05
        # on the line u = u_b
        assert -xp * sa + yp * ca == pytest.approx(ub, abs=1e-9)
        r = f[24] / 0.05
        assert r == pytest.approx(np.hypot(xp - x, yp - y), abs=1e-9)
        kappa = mlp.compton_kappa(e_hat, e0)
        c = 1.0 - kappa
        d = np.array([xp - x, yp - y])
        lim = n * hpx
        depth_off = d @ np.array([ca, sa])
        if -1 < c < 1 and abs(depth_off) < lim * (1 - 1e-9) and np.sqrt(1 - c * c) > 0.05 and r > 0:
            # the angle between p* - q and the detector direction is phi
            assert depth_off / r == pytest.approx(c, abs=1e-9)
            checked += 1
        gx, gy = int(np.floor(xp / hpx + n / 2)), int(np.floor(yp / hpx + n / 2))
        inside = 0 <= gx < n and 0 <= gy < n
        assert f[28] == (rho[gy, gx] if inside else 0.0)
        assert f[27] == (1.0 if e_hat > e0 else 0.0)
    assert checked > 50


def test_scatter_reach_bounds_the_oracles_single_scatter():
    """Outside scatter_reach(line) the oracle's exact single-scatter sum of
    that line is negligible next to its value inside: the surrogate may set it
    to zero there.  The range itself: backscatter (Compton at 180 degrees) to
    the line energy, widened by 8 sigmas."""
    import oracle
    from synthetic import preset
    sc = preset("small_16")
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    rng = np.random.default_rng(3)
    checked = 0
    for w, e0 in enumerate(sc.line_keV):
        lo, hi = mlp.scatter_reach(e0, sc.fwhm_frac, sc.e_ref_keV, sc.fwhm_exponent)
        e_back = oracle.compton_energy(e0, -1.0)
        assert lo < e_back < e0 < hi
        for _ in range(3):
            a, b = int(rng.integers(sc.n_angles)), int(rng.integers(sc.n_bins))
            inside = max(float(orc.scatter_line_row(a, b, e, w).sum())
                         for e in np.linspace(e_back, e0, 9))
            if inside <= 0.0:
                continue
            for e in (lo - 0.5, hi + 0.5):
                if 1.0 < e < 2000.0:
                    out = float(orc.scatter_line_row(a, b, e, w).sum())
                    assert out <= 1e-9 * inside, (w, a, b, e, out, inside)
                    checked += 1
    assert checked >= 8


@pytest.mark.parametrize("stride", [2, 3])
def test_coarse_interpolation_restatement(stride):
    """The coarse-grid surrogate's interpolation as the tests restate it: rows
    sum to 1, only node voxels (both pixel coordinates multiples of the
    stride) or a voxel itself are referenced, nodes map to themselves, and a
    function linear in the pixel coordinates is reproduced exactly wherever
    all four corners lie in the support (bilinear interpolation is exact for
    it)."""
    from oracle_util import coarse_interpolation
    from synthetic import preset
    sc = preset("lmmew_32")
    ph = sc.make_phantom()
    pix = np.nonzero(ph.rho.reshape(-1) > 0)[0]
    n, s = sc.n, stride
    M = coarse_interpolation(pix, n, stride=s)
    np.testing.assert_allclose(M.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    ix, iy = pix % n, pix // n
    node = (ix % s == 0) & (iy % s == 0)
    for q in range(len(pix)):
        cols = np.nonzero(M[q])[0]
        assert np.all(node[cols]) or list(cols) == [q], q
        if node[q]:
            assert M[q, q] == 1.0
    f = 0.7 + 0.3 * ix - 1.1 * iy            # linear in the pixel coordinates
    g = M @ f
    sup = set(int(p) for p in pix)
    full = [q for q in range(len(pix))
            if all((iy[q] - iy[q] % s + dy) * n + (ix[q] - ix[q] % s + dx) in sup
                   for dx in (0, s) for dy in (0, s))]
    assert len(full) > len(pix) // 2
    np.testing.assert_allclose(g[full], f[full], rtol=0, atol=1e-12)
    # at the support edge the renormalised weights still average nearby values
    assert np.all(g >= f.min() - 1e-9) and np.all(g <= f.max() + 1e-9)
