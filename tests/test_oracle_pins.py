"""Pins of the FP64 oracle against closed forms, textbook results, the paper's
printed numbers and brute force -- nothing here re-types the oracle's own
formulas.  CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from oracle_util import events_of, golden, small_model

ME = 510.99895
FWHM = 2.0 * math.sqrt(2.0 * math.log(2.0))


# ---------------------------------------------------------------- KN / Compton
def kn_total_over_pi_re2(e_kev):
    """Textbook Klein-Nishina total cross section per electron / (pi r_e^2)."""
    k = e_kev / ME
    l = math.log1p(2 * k)
    return 2.0 * ((1 + k) / k ** 2 * (2 * (1 + k) / (1 + 2 * k) - l / k)
                  + l / (2 * k) - (1 + 3 * k) / (1 + 2 * k) ** 2)


@pytest.mark.parametrize("e", [30.0, 82.0, 154.0, 270.0, 511.0, 2000.0])
def test_kn_shape_integrates_to_total_cross_section(e):
    # dsigma/dOmega = r_e^2/2 K(cos)  =>  sigma = pi r_e^2 int_{-1}^{1} K dcos
    val = integrate.quad(lambda c: oracle.kn_shape(e, c), -1, 1, epsabs=0, epsrel=1e-13)[0]
    assert val == pytest.approx(kn_total_over_pi_re2(e), rel=1e-10)


def test_kn_thomson_limit_and_forward_value():
    for c in np.linspace(-1, 1, 11):
        assert oracle.kn_shape(1e-7, c) == pytest.approx(1 + c * c, rel=1e-8)
    for e in (82.0, 154.0, 270.0):
        assert oracle.kn_shape(e, 1.0) == pytest.approx(2.0, rel=1e-15)


def kn_plane_closed_form(e_kev):
    """int_0^{2pi} K dtheta from I_n = int dtheta/(a - b cos)^n and
    int sin^2/(a - b cos)^2 = (a I_1 - 2 pi)/b^2 (integration by parts)."""
    k = e_kev / ME
    a, b, d = 1 + k, k, 1 + 2 * k
    i1 = 2 * math.pi / math.sqrt(d)
    i3 = math.pi * (2 * a * a + b * b) * d ** -2.5
    return i3 + i1 - (a * i1 - 2 * math.pi) / b ** 2


@pytest.mark.parametrize("e", [30.0, 82.0, 154.0, 270.0, 2000.0])
def test_kn_plane_norm_closed_form(e):
    assert oracle.kn_plane_norm(e) == pytest.approx(kn_plane_closed_form(e), rel=1e-12)


def test_kn_plane_norm_thomson_limit():
    # K -> 1 + cos^2 whose integral over [0, 2 pi) is 3 pi
    assert oracle.kn_plane_norm(1e-6) == pytest.approx(3 * math.pi, rel=1e-8)


def test_compton_energy_textbook():
    assert oracle.compton_energy(140.0, 1.0) == 140.0
    # backscatter of annihilation photons: 511/3 keV
    assert oracle.compton_energy(ME, -1.0) == pytest.approx(ME / 3.0, rel=1e-14)
    # 90 degrees: E / (1 + E/mc^2)
    assert oracle.compton_energy(270.0, 0.0) == pytest.approx(270.0 / (1 + 270.0 / ME), rel=1e-14)


# ---------------------------------------------------------------- energy axis
def test_energy_resolution_matches_paper():
    m = small_model()
    g = golden("paper_constants.txt")
    assert m.sigma_e(140.0) * FWHM == pytest.approx(g["fwhm_140_keV"][0], rel=1e-13)
    # relative FWHM ~ 1/sqrt(E)  =>  absolute FWHM ~ sqrt(E)
    for e in (60.0, 82.0, 154.0):
        assert m.sigma_e(4 * e) / m.sigma_e(e) == pytest.approx(2.0, rel=1e-13)


@pytest.mark.parametrize("e", [62.0, 82.0, 154.0, 270.0])
def test_energy_density_moments(e):
    m = small_model()
    s = m.sigma_e(e)
    lo, hi = e - 12 * s, e + 12 * s
    m0 = integrate.quad(lambda x: m.energy_density(x, e), lo, hi, epsabs=0, epsrel=1e-12)[0]
    m1 = integrate.quad(lambda x: x * m.energy_density(x, e), lo, hi, epsabs=0, epsrel=1e-12)[0]
    m2 = integrate.quad(lambda x: (x - e) ** 2 * m.energy_density(x, e), lo, hi,
                        epsabs=0, epsrel=1e-12)[0]
    assert m0 == pytest.approx(1.0, rel=1e-11)
    assert m1 == pytest.approx(e, rel=1e-11)
    assert m2 == pytest.approx(s * s, rel=1e-9)


def test_window_mass_symmetric_window_is_erf():
    for z in (0.5, 1.0, 2.0, 3.0):
        e = 140.0
        s = small_model().sigma_e(e)
        m = small_model(windows=((e - z * s, e + z * s),))
        assert m.window_mass(e) == pytest.approx(special.erf(z / math.sqrt(2)), rel=1e-14)


def test_window_mass_equals_integral_of_density_over_windows():
    g = golden("paper_constants.txt")
    wins = (tuple(g["window_EW1"]), tuple(g["window_EW2"]), tuple(g["window_EW3"]))
    m = small_model(windows=wins)
    for e in (70.0, 81.1, 95.0, 144.0, 155.0, 200.0, 270.0):
        ref = sum(integrate.quad(lambda x: m.energy_density(x, e), lo, hi, epsabs=0,
                                 epsrel=1e-12)[0] for lo, hi in wins)
        assert m.window_mass(e) == pytest.approx(ref, rel=1e-10, abs=1e-300)


def test_mu_water_knots_and_extrapolation():
    m = small_model()
    assert m.mu_water(82.0) == 0.184 and m.mu_water(154.0) == 0.148
    assert m.mu_water(270.0) == pytest.approx(0.121, rel=1e-15)
    assert m.mu_water(118.0) == pytest.approx(0.5 * (0.184 + 0.148), rel=1e-14)
    # end segments continue their lines
    for e_out, (e1, e2) in ((60.0, (82.0, 154.0)), (300.0, (154.0, 270.0))):
        slope = (m.mu_water(e2) - m.mu_water(e1)) / (e2 - e1)
        assert m.mu_water(e_out) == pytest.approx(m.mu_water(e1) + slope * (e_out - e1), rel=1e-13)


def _norm_bin(u, s, lo, hi):
    """Gaussian mass on [lo, hi]; upper-tail intervals via the survival function."""
    if lo >= u:
        return stats.norm.sf(lo, u, s) - stats.norm.sf(hi, u, s)
    return stats.norm.cdf(hi, u, s) - stats.norm.cdf(lo, u, s)


# ---------------------------------------------------------------- collimator
def test_bin_probabilities_telescope_and_match_gaussian_integral():
    m = small_model(n_bins=12, pixel_cm=2.0)   # detector spans 16 cm, bins of 16/12 cm
    bw = 16.0 / 12
    for u, sig in ((0.3, 0.4), (-5.1, 1.3), (7.5, 0.8)):
        probs = [m.bin_prob(b, u, sig) for b in range(12)]
        assert sum(probs) == pytest.approx(m.detector_mass(u, sig), rel=1e-13)
        for b in (0, 5, 11):
            lo = -8.0 + b * bw
            ref = _norm_bin(u, sig, lo, lo + bw)
            assert probs[b] == pytest.approx(ref, rel=1e-10, abs=1e-300)
    assert m.detector_mass(0.0, 0.5) == pytest.approx(1.0, rel=1e-15)


def test_collimator_fwhm_linear_in_depth():
    m = small_model(fwhm0=0.3, slope=0.02)
    assert m.sigma_coll(10.0) * FWHM == pytest.approx(0.5, rel=1e-14)
    assert m.sigma_coll(0.0) * FWHM == pytest.approx(0.3, rel=1e-14)


# ---------------------------------------------------------------- line integrals
def _clip_length(x0, y0, x1, y1, bx0, by0, bx1, by1):
    """Length of the segment inside an axis-aligned box (Liang-Barsky)."""
    dx, dy = x1 - x0, y1 - y0
    t0, t1 = 0.0, 1.0
    for p, q in ((-dx, x0 - bx0), (dx, bx1 - x0), (-dy, y0 - by0), (dy, by1 - y0)):
        if p == 0:
            if q < 0:
                return 0.0
            continue
        t = q / p
        if p < 0:
            t0 = max(t0, t)
        else:
            t1 = min(t1, t)
    return max(t1 - t0, 0.0) * math.hypot(dx, dy)


def _brute_integral(rho, h, x0, y0, x1, y1):
    """Sum over every pixel of density x clipped chord length (cm)."""
    n = rho.shape[0]
    half = n * h / 2
    tot = 0.0
    for iy in range(n):
        for ix in range(n):
            if rho[iy, ix] == 0:
                continue
            tot += rho[iy, ix] * _clip_length(x0, y0, x1, y1, ix * h - half, iy * h - half,
                                              (ix + 1) * h - half, (iy + 1) * h - half)
    return tot


def test_line_integrals_random_maps_vs_per_pixel_chords():
    rng = np.random.default_rng(5)
    n, h = 8, 1.5
    rho = rng.uniform(0.0, 2.0, (n, n)).astype(np.float32)
    rho[rng.random((n, n)) < 0.2] = 0.0
    m = small_model(n=n, pixel_cm=h, rho=rho)
    half = n * h / 2
    for _ in range(200):
        x0, y0, x1, y1 = rng.uniform(-1.3 * half, 1.3 * half, 4)
        got = m.line_integral(x0, y0, x1, y1)
        ref = _brute_integral(rho.astype(np.float64), h, x0, y0, x1, y1)
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_line_integral_uniform_map_is_chord_length():
    n, h = 8, 1.0
    m = small_model(n=n, pixel_cm=h)
    assert m.line_integral(-3.2, -1.1, 2.9, 3.3) == pytest.approx(math.hypot(6.1, 4.4), rel=1e-13)
    # from the centre along +x to the edge: 4 cm
    assert m.detector_integral(0.0, 0.0, 0) == pytest.approx(4.0, rel=1e-14)


def test_line_integral_along_grid_line_takes_mean_of_neighbours():
    n, h = 8, 1.0
    rho = np.zeros((n, n), np.float32)
    rho[3, :] = 1.0     # row iy = 3 covers y in [-1, 0)
    rho[4, :] = 3.0     # row iy = 4 covers y in [0, 1)
    m = small_model(n=n, pixel_cm=h, rho=rho)
    # along y = 0 (the edge between rows 3 and 4), x from -4 to 4
    assert m.line_integral(-4.0, 0.0, 4.0, 0.0) == pytest.approx(8 * 2.0, rel=1e-14)
    # along y = 0.5 (centre of row 4)
    assert m.line_integral(-4.0, 0.5, 4.0, 0.5) == pytest.approx(8 * 3.0, rel=1e-14)


def test_detector_integral_random_map_vs_chords():
    rng = np.random.default_rng(7)
    n, h, A = 8, 1.25, 12
    rho = rng.uniform(0.0, 2.0, (n, n)).astype(np.float32)
    m = small_model(n=n, pixel_cm=h, rho=rho, n_angles=A)
    half = n * h / 2
    for a in range(A):
        th = 2 * math.pi * a / A
        for _ in range(10):
            x, y = rng.uniform(-half, half, 2)
            ref = _brute_integral(rho.astype(np.float64), h, x, y, x + 40 * math.cos(th),
                                  y + 40 * math.sin(th))
            assert m.detector_integral(x, y, a) == pytest.approx(ref, rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------- rows
def test_primary_row_point_source_in_uniform_attenuator():
    """One voxel, no scatter, rho = 1 everywhere: the row is
    sum_w alpha_w exp(-mu_w(E_w) D) C(b) g(E_hat; E_w) with D the distance to
    the image edge along the detector direction."""
    n, h, A, B = 8, 2.0, 8, 12
    sup = np.zeros((n, n), bool)
    ix, iy = 5, 2
    sup[iy, ix] = True
    m = small_model(n=n, pixel_cm=h, n_angles=A, n_bins=B, support=sup, scatter_n=0)
    x, y = (ix + 0.5 - n / 2) * h, (iy + 0.5 - n / 2) * h
    half, R, bw = n * h / 2, n * h / 2, n * h / B
    lines, yields = (82.0, 154.0, 270.0), (0.6, 0.2, 0.2)
    mus = (0.184, 0.148, 0.121)
    for a, dist, u, depth in ((0, half - x, y, R - x), (2, half - y, -x, R - y),
                              (4, half + x, -y, R + x), (6, half + y, x, R + y)):
        sig_c = (0.3 + 0.02 * depth) / FWHM
        for b in (0, 3, 7, 11):
            lo = -half + b * bw
            for e_hat in (75.0, 82.0, 150.0, 271.0):
                ref = 0.0
                for e0, al, mu in zip(lines, yields, mus):
                    s_e = 0.1 * math.sqrt(140.0 * e0) / FWHM
                    ref += al * math.exp(-mu * dist) * _norm_bin(u, sig_c, lo, lo + bw) \
                        * stats.norm.pdf(e_hat, e0, s_e)
                got = m.row(a, b, e_hat)[0]
                assert got == pytest.approx(ref, rel=1e-11, abs=1e-300)


def test_single_scatter_row_closed_form():
    """Air everywhere except one dense pixel p: the emission voxel q sits on
    p's row, the detector looks along +y, so the photon turns by 90 degrees at
    p.  Every factor of the single-scatter path is then closed-form."""
    n, h, A, B = 8, 2.0, 4, 16
    rho = np.zeros((n, n), np.float32)
    px, py, qx = 5, 4, 1
    rho[py, px] = 1.25
    sup = np.zeros((n, n), bool)
    sup[py, qx] = True
    lines, yields = (82.0, 154.0, 270.0), (0.6, 0.2, 0.2)
    mus = (0.184, 0.148, 0.121)
    m = small_model(n=n, pixel_cm=h, n_angles=A, n_bins=B, rho=rho, support=sup,
                    scatter_n=n)
    a = 1                                   # theta = 90 degrees, n_a = (0, 1)
    half, R, bw = n * h / 2, n * h / 2, n * h / B
    xq, yq = (qx + 0.5 - n / 2) * h, (py + 0.5 - n / 2) * h
    xp = (px + 0.5 - n / 2) * h
    d = xp - xq
    area = h * h

    def mu_w(e):
        if e >= 154.0:
            return 0.148 + (e - 154.0) * (0.121 - 0.148) / 116.0
        return 0.184 + (e - 82.0) * (0.148 - 0.184) / 72.0

    for b in (2, 7, 12):
        lo = -half + b * bw
        for e_hat in (70.0, 82.0, 126.0, 148.0, 240.0):
            ref = 0.0
            for e0, al, mu0 in zip(lines, yields, mus):
                # primary: q -> +y crosses only air
                sig_q = (0.3 + 0.02 * (R - yq)) / FWHM
                s_e0 = 0.1 * math.sqrt(140.0 * e0) / FWHM
                ref += al * _norm_bin(-xq, sig_q, lo, lo + bw) * stats.norm.pdf(e_hat, e0, s_e0)
                # scatter at p through 90 degrees
                e1 = e0 / (1.0 + e0 / ME)
                k_shape = (e1 / e0) ** 2 * (e1 / e0 + e0 / e1 - 1.0)
                nu = 2 * math.pi * k_shape / kn_plane_closed_form(e0)
                path = (math.exp(-mu0 * 1.25 * h / 2)            # q -> p: half of p's pixel
                        * 1.25 * mu0 * area / (2 * math.pi * d)  # interaction at p
                        * nu
                        * math.exp(-mu_w(e1) * 1.25 * h / 2))    # p -> detector
                sig_p = (0.3 + 0.02 * (R - yq)) / FWHM
                s_e1 = 0.1 * math.sqrt(140.0 * e1) / FWHM
                ref += al * path * _norm_bin(-xp, sig_p, lo, lo + bw) * stats.norm.pdf(e_hat, e1, s_e1)
            got = m.row(a, b, e_hat)[0]
            assert got == pytest.approx(ref, rel=1e-11, abs=1e-300)


def test_sensitivity_is_row_integrated_over_bins_and_window_energies():
    """Brute force on a tiny model with scatter: for every voxel,
    sum_{a in s} sum_b int_window row(a, b, E) dE equals sens_s[q]."""
    from synthetic import preset
    sc = preset("tiny_8")
    ph = sc.make_phantom()
    wins = ((50.0, 120.0), (140.0, 300.0))
    m = oracle.Model.from_scenario(sc.with_(windows=wins), ph.rho)
    n_sub = 2
    # composite Simpson nodes in each window, spaced 1/32 keV so that the
    # float32 event energies hold them exactly
    nodes, wts = [], []
    for lo, hi in wins:
        k = int(round((hi - lo) * 32))
        x = np.linspace(lo, hi, k + 1)
        wgt = np.ones(k + 1)
        wgt[1:-1:2], wgt[2:-1:2] = 4, 2
        nodes.append(x)
        wts.append(wgt * (hi - lo) / (3 * k))
    e_nodes, e_wts = np.concatenate(nodes), np.concatenate(wts)
    for s in range(n_sub):
        ang = [a for a in range(sc.n_angles) if a % n_sub == s]
        A_, B_, E_ = np.meshgrid(ang, np.arange(sc.n_bins), e_nodes, indexing="ij")
        W_ = np.broadcast_to(e_wts, A_.shape)
        ev = events_of(A_.ravel(), B_.ravel(), E_.ravel())
        brute = m.backproject(ev, W_.ravel())
        sens = m.sensitivity(s, n_sub)
        mask = sens > 0
        assert mask.sum() == m.nq
        np.testing.assert_allclose(brute[mask], sens[mask], rtol=2e-7)


def test_backprojection_is_adjoint_of_forward():
    from synthetic import preset, simulate
    sc = preset("small_16")
    ph = sc.make_phantom()
    m = oracle.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc, n_events=150)
    rng = np.random.default_rng(3)
    lam = rng.uniform(0.1, 2.0, sc.n * sc.n) * (ph.rho.reshape(-1) > 0)
    w = rng.uniform(-1.0, 1.0, len(ev))
    lhs = float(np.dot(w, m.forward(ev, lam)))
    rhs = float(np.dot(lam, m.backproject(ev, w)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_forward_is_row_dot_image():
    from synthetic import preset, simulate
    sc = preset("tiny_8")
    ph = sc.make_phantom()
    m = oracle.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc, n_events=20)
    lam = np.linspace(0.5, 1.5, sc.n * sc.n)
    y = m.forward(ev, lam)
    for j in range(len(ev)):
        row = m.row_image(ev.angle[j], ev.bin[j], ev.energy[j])
        assert y[j] == pytest.approx(float(np.dot(row, lam)), rel=1e-13)


def test_no_attenuation_map_gives_blur_only_rows():
    """rho = 0: no scatter points and no attenuation; the row is the bare
    collimator x energy response."""
    n, h, A, B = 8, 2.0, 8, 10
    sup = np.ones((n, n), bool)
    m = small_model(n=n, pixel_cm=h, n_angles=A, n_bins=B, rho=np.zeros((n, n)),
                    support=sup, scatter_n=4)
    assert m.np_scatter == 0
    half, R, bw = n * h / 2, n * h / 2, n * h / B
    row = m.row_image(3, 4, 90.0).reshape(n, n)
    th = 2 * math.pi * 3 / A
    lo = -half + 4 * bw
    for iy in (0, 3, 7):
        for ix in (1, 6):
            x, y = (ix + 0.5 - n / 2) * h, (iy + 0.5 - n / 2) * h
            u = -x * math.sin(th) + y * math.cos(th)
            sig_c = (0.3 + 0.02 * (R - (x * math.cos(th) + y * math.sin(th)))) / FWHM
            ref = sum(al * _norm_bin(u, sig_c, lo, lo + bw)
                      * stats.norm.pdf(90.0, e0, 0.1 * math.sqrt(140 * e0) / FWHM)
                      for e0, al in ((82.0, 0.6), (154.0, 0.2), (270.0, 0.2)))
            assert row[iy, ix] == pytest.approx(ref, rel=1e-11)


# ---------------------------------------------------------------- single-scatter split
def test_scatter_line_rows_are_the_row_minus_the_scatter_free_row():
    """row = primary + sum_w (single-scatter part of line w); the primary part
    is the row of the same object with no scatter points at all, so the split
    is pinned by a model built without the scatter grid."""
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.5, 1.5, (8, 8)).astype(np.float32)
    full = small_model(rho=rho, scatter_n=4)
    prim = small_model(rho=rho, scatter_n=0)
    for a, b, e in ((0, 5, 80.0), (3, 6, 150.0), (6, 2, 265.0), (5, 9, 120.0)):
        split = sum(full.scatter_line_row(a, b, e, w) for w in range(3))
        np.testing.assert_allclose(prim.row(a, b, e) + split, full.row(a, b, e), rtol=1e-12,
                                   atol=1e-300)
        assert np.all(split >= 0) and np.any(split > 0)


def test_scatter_line_row_scales_with_the_line_yield():
    rho = np.ones((8, 8), dtype=np.float32)
    m1 = small_model(rho=rho, scatter_n=4, yields=(0.6, 0.2, 0.2))
    m2 = small_model(rho=rho, scatter_n=4, yields=(0.3, 0.2, 0.8))
    np.testing.assert_allclose(m2.scatter_line_row(2, 6, 100.0, 0),
                               0.5 * m1.scatter_line_row(2, 6, 100.0, 0), rtol=1e-13)
    np.testing.assert_allclose(m2.scatter_line_row(2, 6, 240.0, 2),
                               4.0 * m1.scatter_line_row(2, 6, 240.0, 2), rtol=1e-13)


def _scatter_reach(e_line, fwhm_frac, e_ref, exponent, k=8.0):
    """Recorded energies one Compton scatter of line e_line can produce,
    widened by k energy-resolution sigmas: the union over E' in
    [backscatter energy, e_line] of E' -+ k sigma_E(E'), on a fine grid."""
    e_back = e_line / (1.0 + 2.0 * e_line / 510.99895)
    es = np.linspace(e_back, e_line, 20001)
    sig = fwhm_frac * es * (es / e_ref) ** exponent / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    return float((es - k * sig).min()), float((es + k * sig).max())


@pytest.mark.parametrize("name", ["small_16", "lmmew_32"])
def test_scatter_of_lines_out_of_reach_is_negligible_in_rows(name):
    """The exact row's single-scatter part of a line whose scatter cannot
    reach the recorded energy within 8 sigmas (the energy-window pruning of
    the row kernel) is negligible: below 1e-12 of the event's whole row
    (its forward projection of a uniform image) and below 1e-6 of every
    row element that is not zero.  Energies span the window so that each
    line is out of reach for some of them (Compton's relation, Eq. s_p with
    n = 1)."""
    from synthetic import preset
    sc = preset(name)
    orc = oracle.Model.from_scenario(sc, sc.make_phantom().rho)
    rng = np.random.default_rng(5)
    checked = set()
    for e in (52.0, 60.0, 70.0, 125.0, 160.0, 210.0, 250.0, 290.0):
        for _ in range(3):
            a, b = int(rng.integers(sc.n_angles)), int(rng.integers(sc.n_bins))
            row = orc.row(a, b, e)
            assert row.sum() > 0
            for w, el in enumerate(sc.line_keV):
                lo, hi = _scatter_reach(el, sc.fwhm_frac, sc.e_ref_keV, sc.fwhm_exponent)
                if lo <= e <= hi:
                    continue
                s = orc.scatter_line_row(a, b, e, w)
                assert np.all(s >= 0) and np.all(s <= row)
                assert s.sum() <= 1e-12 * row.sum(), (w, e, s.sum() / row.sum())
                m = row > 0
                assert np.all(s[m] <= 1e-6 * row[m]), (w, e, float((s[m] / row[m]).max()))
                checked.add(w)
    assert checked == set(range(len(sc.line_keV)))
