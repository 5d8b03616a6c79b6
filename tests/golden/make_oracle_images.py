"""Write the FP64-oracle LM-OSEM images that the GPU parity tests compare with.

Each case runs the oracle's LM-OSEM (Eq. os-lm-mlem with z_bar_update_os,
the subsets and iterations of Algorithm 1) on a workload geometry from
``synthetic`` with seeded Monte-Carlo events and stores the image and the
per-sub-iteration log-likelihood (Eq. lll_med without its constants) as
JSON beside this script.  Only ``oracle`` and ``synthetic`` are called: no
value here comes from the CUDA path.

The events are not stored.  They are regenerated from their seed by
``synthetic`` wherever the files are used; the SHA-256 of the event arrays
(angle u16, bin u16, energy f32, little-endian) is stored so that a test
can first check that it reconstructs the same list.

Cases (each takes the oracle tens of minutes on 8 cores):

  lmmew_64_full_2sub  64 x 64, 60 angles, 64 bins, 64 x 64 scatter grid,
                      the workload's whole 300 000-event list (seed 1), two
                      sub-iterations from 1 on rho > 0: subsets 6 and 7 of 8
                      (start_subset = 6), about 70 000 event rows
  lmmew_64_sched      the same geometry, 4 000 events (seed 101), the
                      stated schedule of 8 subsets x 10 iterations
  lmmew_128_sched     128 x 128, 120 angles, 128 bins, 64 x 64 scatter grid,
                      four lesions, 1 000 events (seed 102), 8 x 10

Usage:  python tests/golden/make_oracle_images.py [case ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synthetic import preset, simulate, simulate_cached  # noqa: E402

CASES = {
    # name: (preset, events (None = the workload's own list), seed, subsets,
    #        iterations, first subset)
    "lmmew_64_full_2sub": ("lmmew_64", None, None, 8, 1, 6),
    "lmmew_64_sched": ("lmmew_64", 4000, 101, 8, 10, 0),
    "lmmew_128_sched": ("lmmew_128", 1000, 102, 8, 10, 0),
}


def events_digest(ev) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(ev.angle, dtype="<u2").tobytes())
    h.update(np.ascontiguousarray(ev.bin, dtype="<u2").tobytes())
    h.update(np.ascontiguousarray(ev.energy, dtype="<f4").tobytes())
    return h.hexdigest()


def case_events(name):
    pre, n_ev, seed = CASES[name][:3]
    sc = preset(pre)
    if n_ev is None:
        return sc, simulate_cached(sc)
    return sc, simulate(sc, n_events=n_ev, seed=seed)


def golden_path(name: str) -> str:
    return os.path.join(HERE, f"oracle_osem_{name}.json")


def make(name: str) -> dict:
    pre, n_ev, seed, n_sub, n_it, s0 = CASES[name]
    sc, ev = case_events(name)
    ph = sc.make_phantom()
    orc = oracle.Model.from_scenario(sc, ph.rho)
    lam0 = (ph.rho.reshape(-1) > 0).astype(np.float64)
    t0 = time.time()
    img, ll = orc.osem(ev, lam0, n_sub, n_it, start_subset=s0, want_loglik=True)
    wall = time.time() - t0
    sup = np.nonzero(lam0 > 0)[0]
    return {
        "case": name,
        "what": "FP64 oracle LM-OSEM image and per-sub-iteration log-likelihood",
        "cite": "Eq. os-lm-mlem with z_bar_update_os; Algorithm 1; Eq. lll_med",
        "preset": pre,
        "n_events": len(ev),
        "event_seed": sc.seed if seed is None else seed,
        "events_sha256": events_digest(ev),
        "n_subsets": n_sub,
        "n_iters": n_it,
        "start_iter": 0,
        "start_subset": s0,
        "initial_image": "1 on rho > 0, 0 elsewhere",
        "support_voxels": int(sup.size),
        "image_on_support": [float(v) for v in img[sup]],
        # entry it * n_subsets + s; sub-iterations before start_subset stay 0
        "loglik": [float(v) for v in ll],
        "oracle_threads": oracle.max_threads(),
        "oracle_wall_s": round(wall, 1),
    }


def main(argv):
    names = argv or list(CASES)
    for name in names:
        out = make(name)
        with open(golden_path(name), "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(f"{name}: {out['n_events']} events, {out['oracle_wall_s']} s, "
              f"{out['oracle_threads']} threads", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
