"""Energy-window pruning of the row kernel: events sorted by (angle, energy
class, bin), each tile evaluating the single-scatter terms of the lines
whose scatter can reach its recorded energies only.  A skipped term's energy
factor is below exp(-32) of its path's peak (the oracle pin
test_scatter_of_lines_out_of_reach_is_negligible_in_rows), so pruned and
unpruned projections agree to a few FP32 roundings, and both stay within the
parity tolerance of the FP64 oracle.  Covered: one 50-300 keV window, the
paper's three windows, 32- to 128-event tiles, and an OSEM run."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2305_17111_gb300 as lm  # noqa: E402
from synthetic import preset, simulate  # noqa: E402

FWD_RTOL = 1e-5        # parity with the FP64 oracle
PRUNE_RTOL = 1e-6      # pruned vs unpruned FP32 sums: a few roundings


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


@pytest.mark.parametrize("name,tile", [("lmmew_32", 64), ("small_32_4w", 128), ("small_16", 32)])
def test_pruned_projections_match_unpruned_and_oracle(name, tile):
    sc, ph, ev, lam = _case(name, 1500, 8)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    gpu.set_tile_events(tile)
    dev = lm.DeviceEvents.from_list(ev)
    x = torch.from_numpy(lam).cuda()
    wv = torch.from_numpy(np.random.default_rng(9).uniform(0.1, 1.0, len(ev)).astype(np.float32)).cuda()
    gpu.profile_enable(True)
    y_on = gpu.forward(dev, x).cpu().numpy().astype(np.float64)
    terms_on = gpu.profile_read()["terms"]
    bp_on = gpu.backproject(dev, wv).cpu().numpy().astype(np.float64)
    gpu.set_energy_pruning(False)
    gpu.set_tile_events(tile)
    y_off = gpu.forward(dev, x).cpu().numpy().astype(np.float64)
    terms_off = gpu.profile_read()["terms"]
    bp_off = gpu.backproject(dev, wv).cpu().numpy().astype(np.float64)
    gpu.profile_enable(False)
    assert 0 < terms_on < terms_off
    assert float((np.abs(y_on - y_off) / y_off).max()) < PRUNE_RTOL
    m = bp_off != 0
    assert np.all(bp_on[~m] == 0)
    assert float((np.abs(bp_on[m] - bp_off[m]) / bp_off[m]).max()) < PRUNE_RTOL
    idx = np.arange(0, len(ev), 7)
    ref = oracle.Model.from_scenario(sc, ph.rho).forward(ev.subset(idx), lam.astype(np.float64))
    rel = np.abs(y_on[idx] - ref) / ref
    assert float(rel.max()) < FWD_RTOL, f"max rel {rel.max():.3e}"
    gpu.close()


def test_pruned_osem_matches_unpruned():
    sc, ph, ev, lam = _case("lmmew_32", 2000, 10)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float32)
    a = torch.from_numpy(lam0.copy()).cuda()
    gpu.osem(dev, a, 4, 3)
    gpu.set_energy_pruning(False)
    b = torch.from_numpy(lam0.copy()).cuda()
    gpu.osem(dev, b, 4, 3)
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < PRUNE_RTOL
    gpu.close()


def test_tiles_of_every_size_stay_bit_identical_with_pruning():
    sc, ph, ev, lam = _case("small_24", 1700, 11)
    gpu = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    x = torch.from_numpy(lam).cuda()
    out = {}
    for ts in (128, 64, 32):
        gpu.set_tile_events(ts)
        out[ts] = gpu.forward(dev, x).cpu()
    assert torch.equal(out[64], out[128]) and torch.equal(out[32], out[128])
    gpu.close()
