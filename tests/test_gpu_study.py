"""The comparison study end to end on the GPU: LM-MEW, LM-SEW and Binned-SEW
reconstructions of the same noise realisations through lm_osem_batch, with
the paper's figures of merit."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2305_17111_gb300 import studies  # noqa: E402
from synthetic import preset  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_small_comparison_study():
    sc = preset("paper_study")
    res = studies.run_study(sc, noise_realisations=4, events_per_realisation=3000, seed=5,
                            n_subsets=4, n_iters=4)
    assert set(res) == {"LM-MEW", "LM-SEW", "Binned-SEW"}
    assert res["LM-MEW"]["events_mean"] > res["LM-SEW"]["events_mean"]
    assert res["LM-SEW"]["events_mean"] == res["Binned-SEW"]["events_mean"]
    for name, r in res.items():
        assert r["estimates"].shape == (4, 4)
        assert np.all(np.isfinite(r["estimates"])) and np.all(r["estimates"] > 0)
        for k in ("enrmse", "bias", "std"):
            assert np.all(np.isfinite(r[k])), (name, k)
        assert np.all(r["enrmse"] >= np.abs(r["bias"]) - 1e-12)
