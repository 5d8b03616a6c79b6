"""lm_forward_noalloc, the forward projection for callers that may not
allocate device memory while they run (their device memory belongs to
another allocator, or their steady-state loop forbids the allocation and
synchronisation cudaMalloc brings).  It keeps its scratch in a fixed 16 MiB
static device array of the library.  These tests call it through the C ABI
and compare it bit for bit with lm_forward, the entry point that allocates,
on two calls in a row (the second call reuses the array the first one left
behind), with the exact and the scatter-free models; check that an
oversized request and the surrogate models are refused before any work is
queued; and check the Python wrapper's argument checks.

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


def check(model):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _native.load().lm_check(model._h, stream)


@pytest.mark.parametrize("scatter", ["exact", "none"])
def test_noalloc_matches_lm_forward_on_two_calls(case, scatter):
    sc, model, image = case
    model.set_scatter_model(scatter)
    first = lm.DeviceEvents.from_list(simulate(sc, n_events=3000, seed=21))
    second = lm.DeviceEvents.from_list(simulate(sc, n_events=1700, seed=22))
    for events in (first, second):
        ref = model.forward(events, image)
        out = torch.full((len(events),), float("nan"), dtype=torch.float32, device="cuda")
        assert call_noalloc(model, events, image, out) == 0, _native.load().lm_last_error()
        assert check(model) == 0
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        # same kernels in the same order: bit-identical
        np.testing.assert_array_equal(got, ref.cpu().numpy())
    model.set_scatter_model("exact")


def test_noalloc_refuses_the_surrogate_models_before_queueing(case):
    sc, model, image = case
    sur = lm.Surrogate(3)
    events = lm.DeviceEvents.from_list(simulate(sc, n_events=200, seed=24))
    out = torch.zeros(len(events), dtype=torch.float32, device="cuda")
    for kind in ("surrogate", "surrogate_coarse"):
        model.set_scatter_model(kind, sur)
        assert call_noalloc(model, events, image, out) == -6   # LMMEW_ERR_NOT_IMPLEMENTED
        torch.cuda.synchronize()
        assert float(out.abs().sum()) == 0.0
    model.set_scatter_model("exact")
    sur.close()


def test_noalloc_wrapper_checks_its_arguments(case):
    sc, model, image = case
    events = lm.DeviceEvents.from_list(simulate(sc, n_events=300, seed=25))
    with pytest.raises(ValueError):
        model.forward_noalloc(events, image, torch.zeros(len(events) + 1, device="cuda"))
    with pytest.raises(TypeError):
        model.forward_noalloc(events, image, torch.zeros(len(events)))   # host tensor
    out = torch.empty(len(events), dtype=torch.float32, device="cuda")
    model.forward_noalloc(events, image, out)
    assert torch.equal(out, model.forward(events, image))


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
    assert check(model) == 0
    np.testing.assert_array_equal(out2.cpu().numpy(), model.forward(small, image).cpu().numpy())
