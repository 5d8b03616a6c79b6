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


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A wait on an mbarrier that nothing arrives on runs out after its limit
    and is reported as a timeout; the GPU then runs a normal projection."""
    import ctypes

    import numpy as np

    from paper_2305_17111_gb300 import _native
    from synthetic import preset, simulate
    waited = ctypes.c_double()
    rc = _native.load().lm_selftest_wait_timeout(ctypes.byref(waited))
    assert rc == -5, _native.load().lm_last_error()          # LMMEW_ERR_TIMEOUT
    assert 1500.0 < waited.value < 10000.0, waited.value     # the 2 s limit
    sc = preset("tiny_8")
    ph = sc.make_phantom()
    model = lm.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc)
    y = model.forward(lm.DeviceEvents.from_list(ev),
                      torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda())
    assert bool(torch.all(torch.isfinite(y))) and bool(torch.all(y > 0))
