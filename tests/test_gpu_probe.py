"""The measured exponential rate behind the row kernel's roofline: one MUFU
ex2 per clock per SM lane group, i.e. 32 FP32 exponentials per clock per SM
on GB300, and the packed half forms giving the same number of results."""
from __future__ import annotations

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_17111_gb300 as lm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_ex2_rate_per_sm():
    r = lm.probe_ex2_rate()
    assert 28.0 < r["f32"] < 34.0, r
    # packed halves: no more exponential results per clock than FP32
    assert r["f16x2"] < 1.15 * r["f32"] and r["bf16x2"] < 1.15 * r["f32"], r
    assert r["sm_mhz"] > 1000.0
