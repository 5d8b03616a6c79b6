"""The reduced-precision form of the single-scatter sum (FP16 / BF16 exponent
arithmetic and ex2, FP32 accumulation): its forward-projection and
reconstruction errors against the FP64 oracle stay within the stated bounds,
and switching back to FP32 restores the exact path bit for bit."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2305_17111_gb300 as lm  # noqa: E402
from synthetic import preset, simulate  # noqa: E402

# stated error bounds of the reduced-precision form (relative to FP64)
BOUNDS = {"fp16": {"fwd_max": 5e-3, "fwd_mean": 1e-3, "img_rl2": 5e-3},
          "bf16": {"fwd_max": 3e-2, "fwd_mean": 1e-2, "img_rl2": 3e-2}}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", ["small_24", "lmmew_32"])
def test_reduced_precision_errors(name):
    sc = preset(name)
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc)
    dev = lm.DeviceEvents.from_list(ev)
    rng = np.random.default_rng(1)
    lam = (rng.uniform(0.2, 3.0, ph.rho.size) * (ph.rho.reshape(-1) > 0)).astype(np.float32)
    ref = orc.forward(ev, lam.astype(np.float64))
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float32)
    ref_img = orc.osem(ev, lam0.astype(np.float64), sc.n_subsets, sc.n_iters)
    y32 = gpu.forward(dev, torch.from_numpy(lam).cuda()).cpu().numpy()
    report = {}
    for prec in ("fp16", "bf16"):
        gpu.set_scatter_precision(prec)
        y = gpu.forward(dev, torch.from_numpy(lam).cuda()).cpu().numpy().astype(np.float64)
        rel = np.abs(y - ref) / ref
        img = torch.from_numpy(lam0.copy()).cuda()
        gpu.osem(dev, img, sc.n_subsets, sc.n_iters)
        got = img.cpu().numpy().astype(np.float64)
        rl2 = float(np.linalg.norm(got - ref_img) / np.linalg.norm(ref_img))
        report[prec] = {"fwd_max": float(rel.max()), "fwd_mean": float(rel.mean()), "img_rl2": rl2}
        b = BOUNDS[prec]
        assert rel.max() < b["fwd_max"] and rel.mean() < b["fwd_mean"] and rl2 < b["img_rl2"], report
    gpu.set_scatter_precision("fp32")
    y_back = gpu.forward(dev, torch.from_numpy(lam).cuda()).cpu().numpy()
    np.testing.assert_array_equal(y_back, y32)
    out = os.environ.get("LMMEW_REPORT_DIR")
    if out:
        with open(os.path.join(out, f"precision_{name}.json"), "w") as f:
            json.dump(report, f)


def test_reduced_precision_forward_full_size_128():
    """The precision form's workload (128 x 128, 120 angles, 1 M events):
    forward projections of FP32, FP16 and BF16 scatter sums on events sampled
    from spread-out angles, against the FP64 oracle event by event."""
    from synthetic import simulate_cached
    sc = preset("lmmew_128")
    ph = sc.make_phantom()
    ev = simulate_cached(sc)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    rng = np.random.default_rng(12)
    lam = (rng.uniform(0.2, 3.0, ph.rho.size) * (ph.rho.reshape(-1) > 0)).astype(np.float32)
    idx = []
    for a in rng.choice(sc.n_angles, size=3, replace=False):
        cand = np.nonzero(ev.angle == a)[0]
        idx.extend(rng.choice(cand, size=3, replace=False).tolist())
    idx = np.array(sorted(idx))
    ref = oracle.Model.from_scenario(sc, ph.rho).forward(ev.subset(idx), lam.astype(np.float64))
    bounds = {"fp32": 1e-5, "fp16": BOUNDS["fp16"]["fwd_max"], "bf16": BOUNDS["bf16"]["fwd_max"]}
    report = {}
    for prec in ("fp32", "fp16", "bf16"):
        gpu.set_scatter_precision(prec)
        y = gpu.forward(dev, torch.from_numpy(lam).cuda()).cpu().numpy().astype(np.float64)
        rel = np.abs(y[idx] - ref) / ref
        report[prec] = float(rel.max())
        assert rel.max() < bounds[prec], report
    gpu.set_scatter_precision("fp32")
    gpu.close()
    out = os.environ.get("LMMEW_REPORT_DIR")
    if out:
        with open(os.path.join(out, "precision_lmmew_128_sampled.json"), "w") as f:
            json.dump(report, f)
