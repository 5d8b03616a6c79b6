"""Parity at the full workload sizes, in the launch configuration bench.py
times (the whole event list through lm_forward / lm_osem), checked on
outputs the FP64 oracle can compute one by one and on properties that hold
at any size."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2305_17111_gb300 as lm  # noqa: E402
from synthetic import preset, simulate_cached  # noqa: E402

FWD_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def sample_indices(ev, n_angles, per_angle_groups, seed, per_angle=3):
    """A few events from spread-out angles (the oracle builds one table per
    angle); per_angle_groups = n_angles takes every angle."""
    rng = np.random.default_rng(seed)
    angles = rng.choice(n_angles, size=per_angle_groups, replace=False)
    out = []
    for a in angles:
        idx = np.nonzero(ev.angle == a)[0]
        out.extend(rng.choice(idx, size=min(per_angle, idx.size), replace=False).tolist())
    return np.array(sorted(out))


def rand_image(ph, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.2, 3.0, ph.rho.size) * (ph.rho.reshape(-1) > 0)).astype(np.float32)


@pytest.mark.parametrize("name,groups,per_angle", [("lmmew_64", 60, 1), ("lmmew_128", 120, 1),
                                                   ("lmmew_128_2m", 4, 3)])
def test_forward_sampled_parity_full_size(name, groups, per_angle):
    """Every angle's point-run table is touched at 64^2 and 128^2 / 1 M
    events (one sampled event per angle)."""
    sc = preset(name)
    ph = sc.make_phantom()
    ev = simulate_cached(sc)
    assert len(ev) == sc.n_events
    gpu = lm.Model.from_scenario(sc, ph.rho)
    lam = rand_image(ph, 11)
    y = gpu.forward(lm.DeviceEvents.from_list(ev), torch.from_numpy(lam).cuda()).cpu().numpy()
    assert np.all(np.isfinite(y)) and np.all(y > 0)
    idx = sample_indices(ev, sc.n_angles, groups, seed=3, per_angle=per_angle)
    orc = oracle.Model.from_scenario(sc, ph.rho)
    ref = orc.forward(ev.subset(idx), lam.astype(np.float64))
    rel = np.abs(y[idx].astype(np.float64) - ref) / ref
    assert float(rel.max()) < FWD_RTOL, f"max rel {rel.max():.3e}"


def test_sensitivity_full_size_128():
    sc = preset("lmmew_128")
    ph = sc.make_phantom()
    gpu = lm.Model.from_scenario(sc, ph.rho)
    orc = oracle.Model.from_scenario(sc, ph.rho)
    s = 5
    got = gpu.sensitivity(s).cpu().numpy()
    ref = orc.sensitivity(s, sc.n_subsets)
    # FP64 accumulation of terms whose window masses are FP32 (R29)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=0)


def test_osem_full_size_invariants_64():
    """One full iteration of the benchmark workload: count preservation in
    every sub-iteration (checked on the last), non-negativity, support, and
    the MLEM log-likelihood ascent at full size."""
    sc = preset("lmmew_64")
    ph = sc.make_phantom()
    ev = simulate_cached(sc)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    img = lam0.clone()
    ll = torch.zeros(sc.n_subsets, dtype=torch.float64, device="cuda")
    gpu.osem(dev, img, sc.n_subsets, 1, loglik=ll)
    got = img.cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got >= 0)
    assert np.all(got[lam0.cpu().numpy() == 0] == 0)
    # one more sub-iteration of the last subset alone: T sum lam sens_s = J_s
    s = sc.n_subsets - 1
    img2 = img.clone()
    gpu.osem(dev, img2, sc.n_subsets, 1, 0, s)
    sens = gpu.sensitivity(s).cpu().numpy()
    js = int(np.sum(ev.angle % sc.n_subsets == s))
    assert float(np.dot(img2.cpu().numpy().astype(np.float64), sens)) == pytest.approx(js, rel=2e-5)
    # MLEM (one subset) ascent over two iterations
    img3 = lam0.clone()
    ll3 = torch.zeros(3, dtype=torch.float64, device="cuda")
    gpu.osem(dev, img3, 1, 3, loglik=ll3)
    v = ll3.cpu().numpy()
    assert v[1] > v[0] and v[2] > v[1]


def test_batching_workload_full_size():
    """The batching workload in the launch configuration bench.py times:
    256 realisations of the 64 x 64 object with U[50k, 500k] events each,
    disjoint slices of one iid pool from the GPU Monte-Carlo, one OSEM
    iteration of 8 subsets in one lm_osem_batch call (71 M events, several
    row blocks per subset).  Sampled realisations equal their own lm_osem
    runs to FP32 rounding (only the back-projection chunk boundaries at
    row-block edges differ), and the first one's forward projections match
    the FP64 oracle."""
    from synthetic import mc_torch
    sc = preset("lmmew_64")
    ph = sc.make_phantom()
    rng = np.random.default_rng(3)
    sizes = rng.integers(50_000, 500_001, size=256)
    off = np.concatenate([[0], np.cumsum(sizes)])
    pool = mc_torch.simulate(sc, int(off[-1]), seed=3, device="cuda")
    evs = [pool.subset(slice(off[r], off[r + 1])) for r in range(256)]
    devs = [lm.DeviceEvents.from_list(e) for e in evs]
    gpu = lm.Model.from_scenario(sc, ph.rho)
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float32)
    imgs = torch.from_numpy(np.stack([lam0] * len(devs))).cuda()
    gpu.osem_batch(devs, imgs, sc.n_subsets, 1)
    torch.cuda.synchronize()
    for i in (0, 97, 255):
        one = torch.from_numpy(lam0.copy()).cuda()
        gpu.osem(devs[i], one, sc.n_subsets, 1)
        a = imgs[i].double().cpu().numpy()
        b = one.double().cpu().numpy()
        assert np.all(np.isfinite(a)) and np.all(a >= 0)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-6, f"realisation {i}"
    # forward projections of realisation 0 at its reconstructed image
    img0 = imgs[0].contiguous()
    y = gpu.forward(devs[0], img0).cpu().numpy()
    idx = sample_indices(evs[0], sc.n_angles, 4, seed=5)
    orc = oracle.Model.from_scenario(sc, ph.rho)
    ref = orc.forward(evs[0].subset(idx), img0.cpu().numpy().astype(np.float64))
    rel = np.abs(y[idx].astype(np.float64) - ref) / ref
    assert float(rel.max()) < FWD_RTOL, f"max rel {rel.max():.3e}"
    gpu.close()
