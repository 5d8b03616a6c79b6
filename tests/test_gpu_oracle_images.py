"""Image parity with the FP64 oracle at the study-scale geometries, through
stated OSEM schedules (Eq. os-lm-mlem with z_bar_update_os; Algorithm 1).

The oracle's images and log-likelihoods were written once by
tests/golden/make_oracle_images.py (which calls only the oracle and the
seeded input generators); this test regenerates the same events from their
seeds, checks them against the stored SHA-256, runs lm_osem through the C ABI
with the same schedule and compares:
  image on the support: relative L2 below 1e-4,
  log-likelihood of every sub-iteration run: relative 1e-5.
Cases: the 64 x 64 benchmark workload's whole 300 000-event list (two
sub-iterations), the 64 x 64 geometry through 8 subsets x 10 iterations,
and the 128 x 128 geometry through 8 x 10."""
from __future__ import annotations

import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_17111_gb300 as lm  # noqa: E402
from synthetic import preset  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_oracle_images as mk  # noqa: E402

IMG_RL2 = 1e-4
LL_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("name", list(mk.CASES))
def test_osem_image_matches_stored_oracle_image(name):
    with open(mk.golden_path(name)) as f:
        ref = json.load(f)
    sc, ev = mk.case_events(name)
    assert len(ev) == ref["n_events"]
    assert mk.events_digest(ev) == ref["events_sha256"], "event list differs from the oracle's"
    ph = sc.make_phantom()
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float32)
    sup = np.nonzero(lam0 > 0)[0]
    assert sup.size == ref["support_voxels"]
    gpu = lm.Model.from_scenario(sc, ph.rho)
    img = torch.from_numpy(lam0.copy()).cuda()
    n_sub, n_it, s0 = ref["n_subsets"], ref["n_iters"], ref["start_subset"]
    ll = torch.zeros(n_it * n_sub, dtype=torch.float64, device="cuda")
    gpu.osem(lm.DeviceEvents.from_list(ev), img, n_sub, n_it, ref["start_iter"], s0, loglik=ll)
    got = img.double().cpu().numpy()
    want = np.asarray(ref["image_on_support"])
    rl2 = np.linalg.norm(got[sup] - want) / np.linalg.norm(want)
    ll_rel = np.abs(ll.cpu().numpy()[s0:] / np.asarray(ref["loglik"])[s0:] - 1.0).max()
    print(f"{name}: image relative L2 {rl2:.2e}, log-likelihood max relative {ll_rel:.2e}")
    assert rl2 < IMG_RL2, f"relative L2 {rl2:.3e}"
    assert np.all(got[lam0 == 0] == 0) and np.all(got >= 0)
    run = slice(s0, None)   # sub-iterations before start_subset are not run
    np.testing.assert_allclose(ll.cpu().numpy()[run], np.asarray(ref["loglik"])[run],
                               rtol=LL_RTOL)
    gpu.close()
