"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: forward projections within a relative 1e-5 per event, the image
after the stated OSEM iterations within a relative L2 of 1e-4, sensitivities
(accumulated in FP64; the scatter paths' window masses in FP32) within 2e-6,
back projections within 1e-5 per voxel.
Cases span several 32-voxel and 32-point tiles and 128-event tiles with
ragged tails, one to three energy windows and the scatter-free model.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2305_17111_gb300 as lm  # noqa: E402
from synthetic import preset, simulate  # noqa: E402

FWD_RTOL = 1e-5
IMG_RL2 = 1e-4
SENS_RTOL = 2e-6   # FP64 accumulation of terms whose window masses are FP32 (R29)

CASES = ["tiny_8", "small_16", "small_24", "small_32_4w", "noscatter_16", "lmmew_32"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


_cache = {}


def setup_case(name):
    if name in _cache:
        return _cache[name]
    sc = preset(name)
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc)
    out = (sc, ph, orc, gpu, ev, lm.DeviceEvents.from_list(ev))
    _cache[name] = out
    return out


def rand_image(ph, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.2, 3.0, ph.rho.size) * (ph.rho.reshape(-1) > 0)).astype(np.float32)


@pytest.mark.parametrize("name", CASES)
def test_model_sizes_match(name):
    sc, ph, orc, gpu, ev, dev = setup_case(name)
    assert gpu.nq == orc.nq
    assert gpu.np_scatter == orc.np_scatter


@pytest.mark.parametrize("name", CASES)
def test_sensitivity_parity(name):
    sc, ph, orc, gpu, ev, dev = setup_case(name)
    for s in list(range(sc.n_subsets)) + [-1]:
        got = gpu.sensitivity(s).cpu().numpy()
        ref = orc.sensitivity(s, sc.n_subsets)
        np.testing.assert_allclose(got, ref, rtol=SENS_RTOL, atol=0)


@pytest.mark.parametrize("name", CASES)
def test_forward_parity(name):
    sc, ph, orc, gpu, ev, dev = setup_case(name)
    lam = rand_image(ph, 1)
    got = gpu.forward(dev, torch.from_numpy(lam).cuda()).cpu().numpy().astype(np.float64)
    ref = orc.forward(ev, lam.astype(np.float64))
    rel = np.abs(got - ref) / np.abs(ref)
    assert float(rel.max()) < FWD_RTOL, f"max rel {rel.max():.3e} at event {int(rel.argmax())}"


@pytest.mark.parametrize("name", CASES)
def test_backproject_parity(name):
    sc, ph, orc, gpu, ev, dev = setup_case(name)
    rng = np.random.default_rng(2)
    w = rng.uniform(0.1, 1.0, len(ev)).astype(np.float32)
    got = gpu.backproject(dev, torch.from_numpy(w).cuda()).cpu().numpy().astype(np.float64)
    ref = orc.backproject(ev, w.astype(np.float64))
    mask = ref != 0
    assert np.all(got[~mask] == 0)
    rel = np.abs(got[mask] - ref[mask]) / np.abs(ref[mask])
    assert float(rel.max()) < FWD_RTOL


@pytest.mark.parametrize("name", CASES)
def test_osem_image_parity(name):
    sc, ph, orc, gpu, ev, dev = setup_case(name)
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float32)
    img = torch.from_numpy(lam0.copy()).cuda()
    ll = torch.zeros(sc.n_iters * sc.n_subsets, dtype=torch.float64, device="cuda")
    gpu.osem(dev, img, sc.n_subsets, sc.n_iters, loglik=ll)
    got = img.cpu().numpy().astype(np.float64)
    ref, ref_ll = orc.osem(ev, lam0.astype(np.float64), sc.n_subsets, sc.n_iters,
                           want_loglik=True)
    rl2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rl2 < IMG_RL2, f"relative L2 {rl2:.3e}"
    np.testing.assert_allclose(ll.cpu().numpy(), ref_ll, rtol=1e-5)
    assert np.all(got[lam0 == 0] == 0)
    assert np.all(got >= 0)


def test_osem_resume_is_bit_identical():
    sc, ph, orc, gpu, ev, dev = setup_case("small_24")
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    full = lam0.clone()
    gpu.osem(dev, full, sc.n_subsets, 2)
    part = lam0.clone()
    gpu.osem(dev, part, sc.n_subsets, 1)
    gpu.osem(dev, part, sc.n_subsets, 2, start_iter=1)
    assert torch.equal(full, part)
    again = lam0.clone()
    gpu.osem(dev, again, sc.n_subsets, 2)
    assert torch.equal(full, again)          # deterministic


def test_osem_start_subset_matches_oracle():
    """Resume inside an iteration: sub-iterations 1..N-1 on the image the
    oracle produced after sub-iteration 0."""
    sc, ph, orc, gpu, ev, dev = setup_case("small_16")
    n_sub = sc.n_subsets
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float64)
    keep = np.nonzero(ev.angle % n_sub == 0)[0]
    sub0 = ev.subset(keep)
    y = orc.forward(sub0, lam0)
    num = orc.backproject(sub0, np.where(y > 0, 1.0 / y, 0.0))
    sens0 = orc.sensitivity(0, n_sub)
    lam1 = np.where(sens0 > 0, lam0 * num / np.where(sens0 > 0, sens0, 1.0), 0.0)
    img = torch.from_numpy(lam1.astype(np.float32)).cuda()
    gpu.osem(dev, img, n_sub, 1, 0, 1)
    ref = orc.osem(ev, lam0, n_sub, 1)
    got = img.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < IMG_RL2


def test_osem_count_preservation():
    """T sum_q lambda_new[q] sens_s[q] = J_s after a sub-iteration."""
    sc, ph, orc, gpu, ev, dev = setup_case("small_24")
    n_sub = sc.n_subsets
    s = n_sub - 1
    keep = np.nonzero(ev.angle % n_sub == s)[0]
    sub = lm.DeviceEvents.from_list(ev.subset(keep))
    img = torch.from_numpy(rand_image(ph, 7)).cuda()
    gpu.osem(sub, img, n_sub, 1, 0, s)           # exactly one sub-iteration
    sens = gpu.sensitivity(s).cpu().numpy()
    tot = float(np.dot(img.cpu().numpy().astype(np.float64), sens))
    assert tot == pytest.approx(len(keep), rel=1e-5)


def test_mlem_loglik_increases_on_gpu():
    sc, ph, orc, gpu, ev, dev = setup_case("small_16")
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    ll = torch.zeros(6, dtype=torch.float64, device="cuda")
    gpu.osem(dev, lam0, 1, 6, loglik=ll)
    v = ll.cpu().numpy()
    assert np.all(np.diff(v) > -1e-6 * np.abs(v[1:]))


def test_empty_event_list():
    sc, ph, orc, gpu, ev, dev = setup_case("tiny_8")
    empty = lm.DeviceEvents(np.zeros(0, np.uint16), np.zeros(0, np.uint16), np.zeros(0, np.float32))
    y = gpu.forward(empty, torch.ones(sc.n * sc.n, device="cuda"))
    assert y.numel() == 0
    bp = gpu.backproject(empty, torch.zeros(0, device="cuda"))
    assert float(bp.abs().sum()) == 0.0
    img = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    gpu.osem(empty, img, 2, 1)
    ref = orc.osem(ev.subset(np.zeros(0, dtype=np.int64)),
                   (ph.rho.reshape(-1) > 0).astype(np.float64), 2, 1)
    np.testing.assert_array_equal(img.cpu().numpy(), ref.astype(np.float32))


def test_out_of_range_events_rejected():
    sc, ph, orc, gpu, ev, dev = setup_case("tiny_8")
    img = torch.ones(sc.n * sc.n, device="cuda")
    for a, b, e in ((sc.n_angles, 0, 100.0), (0, sc.n_bins, 100.0), (0, 0, 20.0),
                    (0, 0, float("nan"))):
        bad = lm.DeviceEvents([0, a], [0, b], [100.0, e])
        with pytest.raises(lm.LmmewError, match="OUT_OF_RANGE"):
            gpu.forward(bad, img)
    # the handle stays usable
    y = gpu.forward(dev, img)
    assert torch.isfinite(y).all()


def test_invalid_create_arguments():
    sc = preset("tiny_8")
    ph = sc.make_phantom()
    with pytest.raises(lm.LmmewError, match="INVALID_ARG"):
        lm.Model.from_scenario(sc.with_(scatter_n=3), ph.rho)
    with pytest.raises(lm.LmmewError, match="INVALID_ARG"):
        lm.Model.from_scenario(sc.with_(windows=((50.0, 150.0), (100.0, 300.0))), ph.rho)
    with pytest.raises(lm.LmmewError, match="INVALID_ARG"):
        lm.Model.from_scenario(sc, ph.rho, support=np.zeros(sc.n * sc.n, bool))


def test_custom_support_and_single_voxel():
    """A support smaller than the body: parity with the oracle on the same set."""
    sc = preset("small_16")
    ph = sc.make_phantom()
    sup = (ph.rho > 0).copy()
    sup[: sc.n // 2] = False
    orc = oracle.Model.from_scenario(sc, ph.rho, support=sup)
    gpu = lm.Model.from_scenario(sc, ph.rho, support=sup)
    ev = simulate(sc, n_events=300, seed=99)
    dev = lm.DeviceEvents.from_list(ev)
    lam = rand_image(ph, 5)
    got = gpu.forward(dev, torch.from_numpy(lam).cuda()).cpu().numpy().astype(np.float64)
    ref = orc.forward(ev, lam.astype(np.float64) * sup.reshape(-1))
    assert float((np.abs(got - ref) / ref).max()) < FWD_RTOL


def test_energy_model_variants_parity():
    """A relative energy resolution ∝ E^-0.35 (not the square-root law, so
    1/σ(E) takes the general power) at 12 % FWHM at 120 keV, and water
    attenuation through five knots (four interpolation segments, the first
    below the lowest line): sensitivities and forward projections against
    the FP64 oracle at the usual tolerances."""
    sc = preset("small_16").with_(fwhm_exponent=-0.35, fwhm_frac=0.12, e_ref_keV=120.0,
                                  knot_keV=(60.0, 82.0, 154.0, 200.0, 270.0),
                                  mu_water_cm=(0.206, 0.184, 0.148, 0.137, 0.121))
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc)
    for s in (0, -1):
        got = gpu.sensitivity(s).cpu().numpy()
        ref = orc.sensitivity(s, sc.n_subsets)
        np.testing.assert_allclose(got, ref, rtol=SENS_RTOL, atol=0)
    lam = rand_image(ph, 4)
    y = gpu.forward(lm.DeviceEvents.from_list(ev), torch.from_numpy(lam).cuda())
    got = y.cpu().numpy().astype(np.float64)
    ref = orc.forward(ev, lam.astype(np.float64))
    rel = np.abs(got - ref) / np.abs(ref)
    assert float(rel.max()) < FWD_RTOL, f"max rel {rel.max():.3e}"
    gpu.close()


def test_model_beyond_device_memory_is_refused_with_its_size():
    """Path tables of 12 bytes x angles x lines x voxels x scatter points.  A
    model whose tables exceed the free memory is created with streamed tables
    (tests/test_gpu_streaming.py); one whose set-up and the tables of a single
    angle do not fit -- a 1024 x 1024 model with a 1024 x 1024 scatter grid:
    about 0.8 TB of voxel-to-point line integrals and distances and 1.8 TB of
    tables per angle -- is refused before anything large is allocated."""
    sc = preset("lmmew_64").with_(n=1024, pixel_cm=0.0375, n_angles=90, n_bins=256,
                                   scatter_n=1024)
    ph = sc.make_phantom()
    with pytest.raises(lm.LmmewError, match="OOM.*path tables of one angle need"):
        lm.Model.from_scenario(sc, ph.rho)
    # the process keeps a usable device afterwards
    small = preset("tiny_8")
    lm.Model.from_scenario(small, small.make_phantom().rho).close()
