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
