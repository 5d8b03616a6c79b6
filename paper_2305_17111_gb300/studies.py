"""The paper's comparison study on top of the GB300 path (Sec. "Experiments").

Three reconstructions of the same list-mode data, all with the same kernels:

* LM-MEW -- the proposed method: events from the three photopeak windows
  EW1 68-102 keV, EW2 123-184 keV, EW3 243-297 keV with their energies;
* LM-SEW -- EW1 only, with their energies;
* Binned-SEW -- EW1 only, every event's energy set to 85 keV.

Uptake in a lesion = sum of the reconstructed activity over the lesion's
pixels (Sec. "Procedure to perform quantification task").  The figures of
merit are the paper's ensemble normalised RMSE, bias and standard deviation
over S object realisations x N noise realisations (Sec. "Figure of merit for
evaluation").  Everything here is host-side orchestration and statistics;
the reconstructions run through the C ABI (lm_osem_batch).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EW1 = (68.0, 102.0)
EW2 = (123.0, 184.0)
EW3 = (243.0, 297.0)
BINNED_SEW_KEV = 85.0


def ensemble_nrmse(truth, est):
    """ENRMSE_k = 1/S sum_s (1/y_sk) sqrt(sum_n (yhat_skn - y_sk)^2 / N).

    truth: [S, K]; est: [S, N, K].  Returns [K]."""
    truth = np.asarray(truth, dtype=np.float64)
    est = np.asarray(est, dtype=np.float64)
    err = est - truth[:, None, :]
    return np.mean(np.sqrt(np.mean(err * err, axis=1)) / truth, axis=0)


def ensemble_bias(truth, est):
    """Ens. norm. bias_k = 1/(S N) sum_s sum_n (yhat_skn - y_sk) / y_sk."""
    truth = np.asarray(truth, dtype=np.float64)
    est = np.asarray(est, dtype=np.float64)
    return np.mean(np.mean(est - truth[:, None, :], axis=1) / truth, axis=0)


def ensemble_std(truth, est):
    """Ens. norm. std_k = 1/S sum_s (1/y_sk) sqrt(sum_n (yhat_skn - mean_n)^2 / (N-1))."""
    truth = np.asarray(truth, dtype=np.float64)
    est = np.asarray(est, dtype=np.float64)
    sd = np.std(est, axis=1, ddof=1)
    return np.mean(sd / truth, axis=0)


@dataclass
class Method:
    name: str
    windows: tuple
    fixed_energy: float | None = None


METHODS = (
    Method("LM-MEW", (EW1, EW2, EW3)),
    Method("LM-SEW", (EW1,)),
    Method("Binned-SEW", (EW1,), BINNED_SEW_KEV),
)


def select(events, windows, fixed_energy=None):
    """Events inside the windows; optionally every energy replaced."""
    e = np.asarray(events.energy)
    keep = np.zeros(e.shape, dtype=bool)
    for lo, hi in windows:
        keep |= (e >= np.float32(lo)) & (e < np.float32(hi))
    sub = events.subset(np.nonzero(keep)[0])
    if fixed_energy is not None:
        sub.energy = np.full(len(sub), fixed_energy, dtype=np.float32)
    return sub


def roi_uptake(images, masks):
    """[R, n*n] images -> [R, K] lesion sums."""
    imgs = np.asarray(images, dtype=np.float64).reshape(len(images), -1)
    return np.stack([imgs[:, m.reshape(-1)].sum(axis=1) for m in masks], axis=1)


def run_study(scenario, noise_realisations, events_per_realisation, seed=0, n_subsets=None,
              n_iters=None, methods=METHODS):
    """One object (S = 1), N noise realisations drawn by the Monte-Carlo
    generator over all three windows, reconstructed by each method.

    The true uptake of a lesion is its true activity sum rescaled to the
    reconstruction's units: lambda is in expected detected events per unit
    T*sens, so truth = sum_lesion(lambda*) * J_expected / sum_q lambda*_q sens_q,
    with each method's own sensitivity and the mean event count it sees."""
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import simulate

    sc = scenario.with_(windows=(EW1, EW2, EW3))
    ph = sc.make_phantom()
    n_subsets = sc.n_subsets if n_subsets is None else n_subsets
    n_iters = sc.n_iters if n_iters is None else n_iters
    pool = simulate(sc, n_events=events_per_realisation * noise_realisations, seed=seed)
    reals = [pool.subset(np.arange(i * events_per_realisation, (i + 1) * events_per_realisation))
             for i in range(noise_realisations)]
    out = {}
    for meth in methods:
        model = lm.Model.from_scenario(sc.with_(windows=meth.windows), ph.rho, n_subsets=n_subsets)
        evs = [select(r, meth.windows, meth.fixed_energy) for r in reals]
        devs = [lm.DeviceEvents.from_list(e) for e in evs]
        lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
        imgs = lam0.repeat(len(devs), 1).contiguous()
        model.osem_batch(devs, imgs, n_subsets, n_iters)
        est = roi_uptake(imgs.cpu().numpy(), ph.lesion_masks)
        sens = model.sensitivity(-1).cpu().numpy()
        act = ph.activity.reshape(-1).astype(np.float64)
        mean_j = float(np.mean([len(e) for e in evs]))
        scale = mean_j / float(np.dot(act, sens))
        truth = np.array([act[m.reshape(-1)].sum() * scale for m in ph.lesion_masks])
        out[meth.name] = {
            "events_mean": mean_j,
            "truth": truth,
            "estimates": est,
            "enrmse": ensemble_nrmse(truth[None, :], est[None, :, :]),
            "bias": ensemble_bias(truth[None, :], est[None, :, :]),
            "std": ensemble_std(truth[None, :], est[None, :, :]),
        }
        model.close()
    return out
