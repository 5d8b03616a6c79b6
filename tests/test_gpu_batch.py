"""Batched LM-OSEM (many realisations, one persistent row launch per
sub-iteration, the reconstruction replayed as a CUDA graph, autotuned launch
shape): every realisation's image and log-likelihood equal lm_osem's on its
own events bit for bit, including uneven and empty event lists."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2305_17111_gb300 as lm  # noqa: E402
from synthetic import preset, simulate  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_batch_equals_single_reconstructions():
    sc = preset("small_24")
    ph = sc.make_phantom()
    gpu = lm.Model.from_scenario(sc, ph.rho)
    sizes = [300, 0, 700, 451]
    evs = [simulate(sc, n_events=n, seed=100 + i) if n else
           simulate(sc, n_events=1, seed=1).subset(np.zeros(0, dtype=np.int64))
           for i, n in enumerate(sizes)]
    devs = [lm.DeviceEvents.from_list(e) for e in evs]
    rng = np.random.default_rng(0)
    lam0 = np.stack([(rng.uniform(0.5, 2.0, ph.rho.size) * (ph.rho.reshape(-1) > 0))
                     for _ in sizes]).astype(np.float32)
    n_sub, n_it = sc.n_subsets, 2
    imgs = torch.from_numpy(lam0.copy()).cuda()
    ll = torch.zeros(len(sizes), n_it * n_sub, dtype=torch.float64, device="cuda")
    gpu.osem_batch(devs, imgs, n_sub, n_it, loglik=ll)
    torch.cuda.synchronize()
    tune = gpu.batch_tuning()
    assert tune["tuned"] and tune["ctas_per_sm"] >= 1
    for i, d in enumerate(devs):
        one = torch.from_numpy(lam0[i].copy()).cuda()
        l1 = torch.zeros(n_it * n_sub, dtype=torch.float64, device="cuda")
        gpu.osem(d, one, n_sub, n_it, loglik=l1)
        assert torch.equal(imgs[i], one), f"realisation {i}"
        assert torch.equal(ll[i], l1), f"realisation {i}"
    # and one realisation against the FP64 oracle
    orc = oracle.Model.from_scenario(sc, ph.rho)
    ref = orc.osem(evs[2], lam0[2].astype(np.float64), n_sub, n_it)
    got = imgs[2].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-4


def test_batch_rerun_and_retune():
    sc = preset("tiny_8")
    ph = sc.make_phantom()
    gpu = lm.Model.from_scenario(sc, ph.rho)
    devs = [lm.DeviceEvents.from_list(simulate(sc, n_events=n, seed=7 + n)) for n in (50, 90)]
    lam0 = torch.from_numpy(np.stack([(ph.rho.reshape(-1) > 0).astype(np.float32)] * 2)).cuda()
    a = lam0.clone()
    gpu.osem_batch(devs, a, 2, 3)
    b = lam0.clone()
    gpu.osem_batch(devs, b, 2, 3)          # same shape: cached tuning, new graph
    assert torch.equal(a, b)
    c = lam0[:1].clone()
    gpu.osem_batch(devs[:1], c, 2, 3)      # new shape: re-tuned
    assert torch.equal(c[0], a[0])


def test_batch_with_several_row_blocks_per_subset():
    """A batch whose sub-iterations hold more events than one row block (4 GiB
    of rows): each realisation's events of a subset are split over two row
    blocks, so its back-projection chunks restart at the block boundary and
    only the FP32 rounding of those chunk sums may differ from lm_osem.  The
    images and log-likelihoods agree to FP32 rounding."""
    from synthetic import simulate_cached
    sc = preset("lmmew_128")
    ph = sc.make_phantom()
    pool = simulate_cached(sc)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    n_sub, n_real, per_real = 8, 8, 420_000
    row_floats = (gpu.nq + 3) // 4 * 4
    assert n_real * per_real // n_sub * row_floats > 2 ** 30    # > one row block per subset
    rng = np.random.default_rng(21)
    evs = [pool.subset(rng.integers(0, len(pool), size=per_real)) for _ in range(n_real)]
    devs = [lm.DeviceEvents.from_list(e) for e in evs]
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float32)
    imgs = torch.from_numpy(np.stack([lam0] * n_real)).cuda()
    ll = torch.zeros(n_real, n_sub, dtype=torch.float64, device="cuda")
    gpu.osem_batch(devs, imgs, n_sub, 1, loglik=ll)
    torch.cuda.synchronize()
    for i, d in enumerate(devs):
        one = torch.from_numpy(lam0.copy()).cuda()
        l1 = torch.zeros(n_sub, dtype=torch.float64, device="cuda")
        gpu.osem(d, one, n_sub, 1, loglik=l1)
        a = imgs[i].double().cpu().numpy()
        b = one.double().cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-6, f"realisation {i}"
        big = b > 1e-3 * b.max()
        assert float(np.max(np.abs(a[big] - b[big]) / b[big])) < 1e-5, f"realisation {i}"
        assert torch.allclose(ll[i], l1, rtol=1e-9, atol=0.0), f"realisation {i}"
    gpu.close()
