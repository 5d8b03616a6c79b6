"""The event-taking entry points queue their work on the caller's stream and
return without waiting for it (after the set-up of a first call): a call
made while a long kernel still runs returns at once, its work completes
later with the same results as a call made on an idle GPU, and an event
that fails validation on the device (an angle outside the model) is
reported by the next synchronising call, lm_check.  Called through the raw
C ABI."""
from __future__ import annotations

import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_17111_gb300 as lm  # noqa: E402
from paper_2305_17111_gb300 import _native  # noqa: E402
from synthetic import preset, simulate  # noqa: E402

SLEEP_CYCLES = 2_000_000_000   # about a second of device time at 2 GHz


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    sc = preset("lmmew_32")
    ph = sc.make_phantom()
    model = lm.Model.from_scenario(sc, ph.rho)
    ev = simulate(sc, n_events=6000, seed=41)
    dev = lm.DeviceEvents.from_list(ev)
    rng = np.random.default_rng(42)
    lam = torch.from_numpy((rng.uniform(0.2, 3.0, sc.n * sc.n)
                            * (ph.rho.reshape(-1) > 0)).astype(np.float32)).cuda()
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    w = torch.from_numpy(rng.uniform(0.1, 1.0, len(ev)).astype(np.float32)).cuda()
    yield sc, model, dev, lam, lam0, w
    model.close()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _forward(model, dev, image, out):
    ev = dev.struct()
    return _native.load().lm_forward(model._h, ctypes.byref(ev), ctypes.c_void_p(image.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), _stream())


def _backproject(model, dev, w, out):
    ev = dev.struct()
    return _native.load().lm_backproject(model._h, ctypes.byref(ev), ctypes.c_void_p(w.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream())


def _osem(model, dev, n_sub, n_it, img, ll):
    ev = dev.struct()
    return _native.load().lm_osem(model._h, ctypes.byref(ev), n_sub, n_it, 0, 0,
                                  ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(ll.data_ptr()),
                                  _stream())


def _check(model):
    return _native.load().lm_check(model._h, _stream())


def test_calls_queue_behind_a_running_kernel_without_a_host_stall(case):
    sc, model, dev, lam, lam0, w = case
    n_sub = sc.n_subsets
    # first calls: set-up (partition tables, scratch, launch-shape tuning)
    ref_y = model.forward(dev, lam).clone()
    ref_bp = model.backproject(dev, w).clone()
    ref_img = lam0.clone()
    ref_ll = torch.zeros(2 * n_sub, dtype=torch.float64, device="cuda")
    model.osem(dev, ref_img, n_sub, 2, loglik=ref_ll)
    torch.cuda.synchronize()

    y = torch.full_like(ref_y, float("nan"))
    bp = torch.full_like(ref_bp, float("nan"))
    img = lam0.clone()
    ll = torch.zeros_like(ref_ll)
    torch.cuda._sleep(SLEEP_CYCLES)
    t0 = time.perf_counter()
    rcs = (_forward(model, dev, lam, y), _backproject(model, dev, w, bp),
           _osem(model, dev, n_sub, 2, img, ll))
    host_s = time.perf_counter() - t0
    queued = torch.cuda.Event()
    queued.record()
    still_running = not queued.query()
    assert rcs == (0, 0, 0), _native.load().lm_last_error()
    assert still_running, "the stream finished before the calls returned"
    assert host_s < 0.25, f"the calls held the host for {host_s:.3f} s"
    assert _check(model) == 0
    assert torch.equal(y, ref_y)
    assert torch.equal(bp, ref_bp)
    assert torch.equal(img, ref_img)
    assert torch.equal(ll, ref_ll)


def test_out_of_range_event_is_reported_by_the_next_check(case):
    sc, model, dev, lam, lam0, w = case
    b = sc.n_bins // 2   # central bins: every valid event there has a positive projection
    bad = lm.DeviceEvents([0, sc.n_angles, 3], [b, b, b + 1], [100.0, 100.0, 150.0])
    y = torch.zeros(3, dtype=torch.float32, device="cuda")
    assert _forward(model, bad, lam, y) == 0
    assert _check(model) == -2          # LMMEW_ERR_OUT_OF_RANGE
    assert b"outside" in _native.load().lm_last_error()
    got = y.cpu().numpy()
    assert np.isnan(got[1]) and np.isfinite(got[0]) and np.isfinite(got[2]) and got[0] > 0
    assert _check(model) == 0          # reported once, then cleared
    # an energy outside every window, through the binding (which checks)
    with pytest.raises(lm.LmmewError, match="OUT_OF_RANGE"):
        model.forward(lm.DeviceEvents([0], [0], [20.0]), lam)
    assert _check(model) == 0
    # the handle keeps working
    assert torch.equal(model.forward(dev, lam), model.forward(dev, lam))
