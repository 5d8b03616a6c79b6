"""lm_forward_noalloc, the forward projection for callers that may not
allocate device memory while they run (their device memory belongs to
another allocator, or their steady-state loop forbids the allocation and
synchronisation cudaMalloc brings).  It keeps its scratch in a fixed 16 MiB
static device array of the library.  These tests call it through the C ABI
and compare it with lm_forward, the entry point that allocates, on two calls
in a row (the second call reuses the array the first one left behind), and
check that an oversized request is refused before any work is queued.

The file sorts last so that a failure here stops a -x run only after every
other test has run.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_17111_gb300 as lm  # noqa: E402
from paper_2305_17111_gb300 import _native  # noqa: E402
from synthetic import preset, simulate  # noqa: E402

FWD_RTOL = 1e-5   # the forward-projection tolerance of the parity tests


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    sc = preset("lmmew_32")
    ph = sc.make_phantom()
    model = lm.Model.from_scenario(sc, ph.rho)
    rng = np.random.default_rng(4)
    lam = (rng.uniform(0.2, 3.0, sc.n * sc.n) * (ph.rho.reshape(-1) > 0)).astype(np.float32)
    return sc, model, torch.from_numpy(lam).cuda()


def call_noalloc(model, events, image, out):
    """The raw C-ABI call, no binding logic in between."""
    ev = events.struct()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _native.load().lm_forward_noalloc(model._h, ctypes.byref(ev),
                                             ctypes.c_void_p(image.data_ptr()),
                                             ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_lm_forward_on_two_calls(case):
    sc, model, image = case
    first = lm.DeviceEvents.from_list(simulate(sc, n_events=3000, seed=21))
    second = lm.DeviceEvents.from_list(simulate(sc, n_events=1700, seed=22))
    for events in (first, second):
        ref = model.forward(events, image)
        out = torch.full((len(events),), float("nan"), dtype=torch.float32, device="cuda")
        assert call_noalloc(model, events, image, out) == 0, _native.load().lm_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        want = ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, want, rtol=FWD_RTOL, atol=0)


def test_noalloc_refuses_requests_beyond_its_array(case):
    sc, model, image = case
    n = 400_000   # ~36 MB of scratch for this model, above the 16 MiB array
    rng = np.random.default_rng(0)
    events = lm.DeviceEvents(rng.integers(0, sc.n_angles, n), rng.integers(0, sc.n_bins, n),
                             rng.uniform(60.0, 290.0, n))
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    rc = call_noalloc(model, events, image, out)
    assert rc == -1
    assert b"16777216" in _native.load().lm_last_error()
    assert float(out.abs().sum()) == 0.0
    # the handle and the array stay usable afterwards
    small = lm.DeviceEvents.from_list(simulate(sc, n_events=500, seed=23))
    out2 = torch.empty(len(small), dtype=torch.float32, device="cuda")
    assert call_noalloc(model, small, image, out2) == 0
    np.testing.assert_allclose(out2.cpu().numpy(), model.forward(small, image).cpu().numpy(),
                               rtol=FWD_RTOL)
