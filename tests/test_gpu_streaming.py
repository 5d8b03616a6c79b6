"""Streamed single-scatter path tables.  The handle keeps the tables of a
block of detector angles only and rebuilds, with the set-up's own kernel,
each block a row launch needs.  The rebuilt entries are the same bits as the
resident ones and every launch sees the same tiles, so forward projections,
back projections, reconstructions and their log-likelihoods must agree bit
for bit with resident tables, for any block size (including blocks that do
not divide a subset's angles).  The forms that read every angle's tables
refuse streamed tables, and lm_create streams by itself when the tables
exceed the process's table budget."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2305_17111_gb300 as lm  # noqa: E402
from paper_2305_17111_gb300._native import LmmewError  # noqa: E402
from synthetic import preset, simulate  # noqa: E402

NOT_IMPLEMENTED = -6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _case(name, n_events, seed):
    sc = preset(name)
    ph = sc.make_phantom()
    ev = simulate(sc, n_events=n_events, seed=seed)
    rng = np.random.default_rng(seed)
    lam = (rng.uniform(0.2, 3.0, ph.rho.size) * (ph.rho.reshape(-1) > 0)).astype(np.float32)
    return sc, ph, ev, lam


@pytest.mark.parametrize("name", ["lmmew_32", "small_24"])
@pytest.mark.parametrize("max_angles", [1, 3, 7])
def test_streamed_projections_match_resident(name, max_angles):
    sc, ph, ev, lam = _case(name, 2500, 11)
    m = lm.Model.from_scenario(sc, ph.rho)
    assert m.table_streaming()[0] == 0
    dev = lm.DeviceEvents.from_list(ev)
    x = torch.from_numpy(lam).cuda()
    wv = torch.from_numpy(np.random.default_rng(12).uniform(0.1, 1.0, len(ev)).astype(np.float32)).cuda()
    f0 = m.forward(dev, x).cpu()
    b0 = m.backproject(dev, wv).cpu()
    resident_bytes = m.table_streaming()[1]

    m.set_table_streaming(max_angles)
    slots, nbytes = m.table_streaming()
    assert slots == max_angles
    assert nbytes * sc.n_angles == resident_bytes * max_angles
    assert torch.equal(m.forward(dev, x).cpu(), f0)
    assert torch.equal(m.backproject(dev, wv).cpu(), b0)
    out = torch.full((len(ev),), float("nan"), dtype=torch.float32, device="cuda")
    m.forward_noalloc(dev, x, out)
    assert torch.equal(out.cpu(), f0)
    # a second round: blocks resident from the last call are reused or rebuilt
    assert torch.equal(m.forward(dev, x).cpu(), f0)

    m.set_table_streaming(0)
    assert m.table_streaming() == (0, resident_bytes)
    assert torch.equal(m.forward(dev, x).cpu(), f0)
    m.close()


@pytest.mark.parametrize("max_angles", [2, 5])
def test_streamed_osem_matches_resident(max_angles):
    sc, ph, ev, _ = _case("lmmew_32", 3000, 13)
    m = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    n_sub, n_it = 4, 2
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()

    img0 = lam0.clone()
    ll0 = torch.zeros(n_it * n_sub, dtype=torch.float64, device="cuda")
    m.osem(dev, img0, n_sub, n_it, loglik=ll0)

    m.set_table_streaming(max_angles)
    img1 = lam0.clone()
    ll1 = torch.zeros_like(ll0)
    m.osem(dev, img1, n_sub, n_it, loglik=ll1)
    assert torch.equal(img1, img0)
    assert torch.equal(ll1, ll0)
    # resumed from the middle of the schedule
    img2 = lam0.clone()
    m.osem(dev, img2, n_sub, 1)
    m.osem(dev, img2, n_sub, n_it, start_iter=1, start_subset=0)
    assert torch.equal(img2, img0)
    m.close()


def test_streamed_scatter_free_model_needs_no_tables():
    sc, ph, ev, lam = _case("lmmew_32", 1500, 14)
    m = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    x = torch.from_numpy(lam).cuda()
    m.set_scatter_model("none")
    f0 = m.forward(dev, x).cpu()
    m.set_table_streaming(4)
    assert torch.equal(m.forward(dev, x).cpu(), f0)
    m.set_scatter_model("exact")
    f_exact = m.forward(dev, x).cpu()
    m.set_table_streaming(0)
    assert torch.equal(m.forward(dev, x).cpu(), f_exact)
    m.close()


def test_streamed_tables_refuse_forms_that_read_every_angle():
    sc, ph, ev, lam = _case("lmmew_32", 1200, 15)
    m = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    m.set_table_streaming(4)
    with pytest.raises(LmmewError) as e:
        m.set_scatter_precision("bf16")
    assert e.value.code == NOT_IMPLEMENTED
    images = torch.ones((2, sc.n * sc.n), dtype=torch.float32, device="cuda")
    with pytest.raises(LmmewError) as e:
        m.osem_batch([dev, dev], images, 4, 1)
    assert e.value.code == NOT_IMPLEMENTED
    with pytest.raises(LmmewError) as e:
        m.surrogate_samples(dev, 256)
    assert e.value.code == NOT_IMPLEMENTED
    with pytest.raises(LmmewError):
        m.set_table_streaming(-1)
    # resident again: every form works; a reduced precision blocks streaming
    m.set_table_streaming(0)
    m.set_scatter_precision("bf16")
    with pytest.raises(LmmewError) as e:
        m.set_table_streaming(4)
    assert e.value.code == NOT_IMPLEMENTED
    m.set_scatter_precision("fp32")
    m.set_table_streaming(4)
    assert m.table_streaming()[0] == 4
    m.close()


def test_create_streams_above_the_table_budget():
    sc, ph, ev, lam = _case("small_24", 2000, 16)
    ref = lm.Model.from_scenario(sc, ph.rho)
    per_angle = ref.table_streaming()[1] // sc.n_angles
    lm.set_table_budget(per_angle * 5 + per_angle // 2)
    try:
        m = lm.Model.from_scenario(sc, ph.rho)
    finally:
        lm.set_table_budget(0)
    slots, nbytes = m.table_streaming()
    assert slots == 5 and nbytes == 5 * per_angle
    # the sensitivity was summed angle block by angle block: same bits
    assert torch.equal(m.sensitivity(), ref.sensitivity())
    assert torch.equal(m.sensitivity(1), ref.sensitivity(1))
    dev = lm.DeviceEvents.from_list(ev)
    x = torch.from_numpy(lam).cuda()
    assert torch.equal(m.forward(dev, x), ref.forward(dev, x))
    # later models are resident again
    again = lm.Model.from_scenario(sc, ph.rho)
    assert again.table_streaming()[0] == 0
    for h in (m, ref, again):
        h.close()
