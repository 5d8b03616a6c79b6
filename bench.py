#!/usr/bin/env python
"""Benchmark of the LM-MEW OSEM hot path on GB300.

One step = one full LM-OSEM iteration (every subset: system-matrix rows
computed on the fly, forward projection, ratio, back projection, update) over
the 64x64 study-scale workload (300k events, 60 angles, 64 bins, 64x64
scatter grid, 3 emission lines, 8 subsets), through the C ABI.  The K timed
steps are K iterations of one lm_osem call (the events are sorted once per
call); the end-to-end measure makes one call per step, with that step's host
copies.

Metric: system-matrix elements per second (events x support voxels per
step / step time), plus seconds per OSEM iteration.  With --gpus N under
torchrun every rank reconstructs its own independent noise realisation
(replicas; the path has no cross-GPU exchange), the value is the whole job's
elements / the slowest rank's time.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (its forward projection of a subset of events) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "lmmew_64"
METRIC = "sys-matrix elems/s"
UNIT = "elem/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--events", type=int, default=None,
                    help="override the workload's event count (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the forms section (precision, batching with the combined form, comparison, surrogate)")
    ap.add_argument("--forms", default="precision,batching,comparison,surrogate,streamed",
                    help="comma-separated forms to measure")
    ap.add_argument("--case", default=None, choices=["row", "row_rows", "surrogate_rows", "surrogate_train", "surrogate_coarse_osem", "setup"],
                    help="run one small kernel case (for profiling) instead of the benchmark")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload_config(sc, nq=None, npts=None):
    cfg = {"workload": f"{sc.name}: {sc.n}x{sc.n} image {sc.pixel_cm} cm, {sc.n_angles} angles, "
                       f"{sc.n_bins} bins, {sc.scatter_n}x{sc.scatter_n} scatter grid, "
                       f"{len(sc.line_keV)} lines {'/'.join(str(int(e)) for e in sc.line_keV)} keV, "
                       f"{sc.n_events} events, {sc.n_subsets} subsets",
           "events": sc.n_events, "subsets": sc.n_subsets, "step": "one LM-OSEM iteration"}
    if nq is not None:
        cfg["support_voxels"] = nq
    if npts is not None:
        cfg["scatter_points"] = npts
    return cfg


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ peaks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return None


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# current k_row revision on this workload.  Measured on the small case
# `--case row_rows` (60 000 events of subset 0's 8 angles, rows stored as
# lm_osem does, 64-event tiles): 217 606 144 B read (the 8 angles' path
# tables) + 175 658 496 B written (the row block), in a one-launch capture;
# scaled to one OSEM launch of this workload by angles for the reads (7.5 of
# 8) and by events for the writes (37 500 of 60 000).  Emptied whenever
# k_row or the tables it streams change until the counters are taken again.
ROW_TRAFFIC_BYTES_PER_LAUNCH = {"lmmew_64": 204_005_760 + 109_786_560}

# Exponential (MUFU ex2) issue rate of one GB300 SM per clock.  The roofline
# of the exact path is the SFU rate: every path term needs one ex2.
EX2_PER_SM_PER_CLK = 32


def ex2_peak(sm_count, mhz):
    return sm_count * EX2_PER_SM_PER_CLK * mhz * 1e6


# ------------------------------------------------------------------ CPU baseline
class OracleSample:
    """The FP64 oracle, as it stands, timed on bounded samples of the workload."""

    def __init__(self, sc):
        import numpy as np

        import oracle
        from synthetic import simulate_cached
        self.sc = sc
        ph = sc.make_phantom()
        self.ev = simulate_cached(sc)
        self.orc = oracle.Model.from_scenario(sc, ph.rho)
        self.lam = (ph.rho.reshape(-1) > 0).astype(np.float64)
        self.cores = oracle.max_threads()

    def run(self, n_sample, seed=0):
        import numpy as np
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(len(self.ev), size=min(n_sample, len(self.ev)), replace=False))
        sub = self.ev.subset(idx)
        t0 = time.perf_counter()
        self.orc.forward(sub, self.lam)
        dt = time.perf_counter() - t0
        return len(sub) * self.orc.nq, dt


def host_cpu_model():
    """The host's core model (lscpu's 'Model name'; else /proc/cpuinfo's x86
    'model name' or Arm implementer / part numbers), for the CPU baseline's
    record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.processor() or "unknown"
    for line in info:
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    impl = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU implementer")]
    part = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU part")]
    if impl and part:
        return f"{platform.machine()} implementer {impl[0]} part {part[0]}"
    return platform.machine() or "unknown"


def cpu_baseline(sc, n_sample=None):
    import oracle
    o = OracleSample(sc)
    if n_sample is None:
        n_sample = 400 if sc.n <= 64 else 60
    elems, dt = o.run(n_sample)
    # the same oracle on one core, on a tenth of the sample
    n_one = max(n_sample // 10, 1)
    oracle.set_threads(1)
    try:
        elems1, dt1 = o.run(n_one, seed=1)
    finally:
        oracle.set_threads(o.cores)
    return {"value": elems / dt, "unit": UNIT, "cores": o.cores, "kind": "oracle",
            "sample": f"{n_sample} random events of {sc.name}: FP64 oracle row + forward "
                      f"projection ({elems:.3e} elements in {dt:.1f} s)",
            "value_1core": elems1 / dt1,
            "sample_1core": f"{n_one} other random events, one thread ({dt1:.1f} s)",
            "cpu_model": host_cpu_model()}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from synthetic import preset
    sc = preset(args.workload)
    n_per_step = 100 if sc.n <= 64 else 16
    o = OracleSample(sc)
    tot_e, tot_t = 0.0, 0.0
    for step in range(args.warmup + args.steps):
        elems, dt = o.run(n_per_step, seed=step)
        if step >= args.warmup:
            tot_e += elems
            tot_t += dt
    value = tot_e / tot_t
    base = {"cores": o.cores}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(sc),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"],
                             "kind": "oracle",
                             "sample": f"each step: {n_per_step} random events of "
                                       f"{sc.name}, FP64 oracle row + forward projection"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(value, dist=None, device="cpu"):
    """The slowest rank's time (or any value): MAX all-reduce when distributed."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank_step, steps, world, ms_max):
    """Units all ranks processed / the slowest rank's time (replicas: every
    rank processes the same number of units per step)."""
    return world * units_per_rank_step * steps / (ms_max / 1e3)


def run_e2e(model, ev, img, sc, n_sub, it, steps, stream, barrier, dist):
    """Same steps through the same call with host buffers: each step copies
    its events from pinned host memory and reads the image back."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    h_ang = torch.from_numpy(np.asarray(ev.angle, np.uint16).view(np.int16).copy()).pin_memory()
    h_bin = torch.from_numpy(np.asarray(ev.bin, np.uint16).view(np.int16).copy()).pin_memory()
    h_en = torch.from_numpy(np.asarray(ev.energy, np.float32).copy()).pin_memory()
    h_img = torch.empty(sc.n * sc.n, dtype=torch.float32).pin_memory()
    d_ang = torch.empty_like(h_ang, device="cuda")
    d_bin = torch.empty_like(h_bin, device="cuda")
    d_en = torch.empty_like(h_en, device="cuda")
    dev2 = lm.DeviceEvents(d_ang, d_bin, d_en)
    img2 = img.clone()
    barrier()
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(steps):
        d_ang.copy_(h_ang, non_blocking=True)
        d_bin.copy_(h_bin, non_blocking=True)
        d_en.copy_(h_en, non_blocking=True)
        model.osem(dev2, img2, n_sub, it + 1, start_iter=it)
        h_img.copy_(img2, non_blocking=True)
        it += 1
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1), dist, "cuda")
    h2d = h_ang.numel() * 2 + h_bin.numel() * 2 + h_en.numel() * 4
    d2h = h_img.numel() * 4

    return ms_e2e, h2d, d2h, it


# ------------------------------------------------------------------ chosen forms
def roi_sums(img, masks):
    import numpy as np
    v = np.asarray(img, dtype=np.float64).reshape(-1)
    return [float(v[m.reshape(-1)].sum()) for m in masks]


def run_precision_form(workload="lmmew_128", iters=None):
    """The reduced-precision scatter sum against the exact FP32 path on the
    same GPU: seconds per OSEM iteration, and the deviation of forward
    projections and lesion (ROI) activities after the stated iterations from
    the FP32 result (the FP32 path's own parity with the FP64 oracle is
    established by the test suite)."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate_cached
    sc = preset(workload)
    ph = sc.make_phantom()
    ev = simulate_cached(sc)
    model = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    rng = np.random.default_rng(5)
    lam_r = torch.from_numpy((rng.uniform(0.2, 3.0, ph.rho.size)
                              * (ph.rho.reshape(-1) > 0)).astype(np.float32)).cuda()
    n_it = sc.n_iters if iters is None else iters
    out = {"workload": f"{sc.name}: {sc.n}x{sc.n}, {sc.n_angles} angles, {sc.n_bins} bins, "
                       f"{sc.scatter_n}x{sc.scatter_n} scatter grid, {len(ev)} events, "
                       f"{sc.n_subsets} subsets x {n_it} iterations"}
    res = {}
    for prec in ("fp32", "fp16", "bf16"):
        model.set_scatter_precision(prec)
        y = model.forward(dev, lam_r).cpu().numpy().astype(np.float64)
        img = lam0.clone()
        model.osem(dev, img, sc.n_subsets, 1)             # warm-up iteration
        img = lam0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        model.osem(dev, img, sc.n_subsets, n_it)
        e1.record()
        torch.cuda.synchronize()
        res[prec] = {"y": y, "img": img.cpu().numpy(), "s_per_iter": e0.elapsed_time(e1) / 1e3 / n_it}
    model.set_scatter_precision("fp32")
    ref = res["fp32"]
    roi_ref = roi_sums(ref["img"], ph.lesion_masks)
    out["fp32"] = {"s_per_iter": ref["s_per_iter"],
                   "elems_per_s": len(ev) * model.nq / ref["s_per_iter"],
                   "roi_activity": roi_ref}
    for prec in ("fp16", "bf16"):
        r = res[prec]
        dev_y = np.abs(r["y"] - ref["y"]) / ref["y"]
        roi = roi_sums(r["img"], ph.lesion_masks)
        out[prec] = {"s_per_iter": r["s_per_iter"],
                     "speedup_vs_fp32": ref["s_per_iter"] / r["s_per_iter"],
                     "fwd_rel_dev_vs_fp32": {"max": float(dev_y.max()), "mean": float(dev_y.mean())},
                     "roi_rel_dev_vs_fp32": [abs(a - b) / b for a, b in zip(roi, roi_ref)],
                     "image_rel_l2_vs_fp32": float(np.linalg.norm(r["img"] - ref["img"])
                                                   / np.linalg.norm(ref["img"]))}
    model.close()
    return out


def _object_events(args):
    """Events of one random training object (a process-pool task)."""
    k, seed, workload, n_events = args
    from synthetic import preset, random_water_bone_object, simulate
    sc = preset(workload).with_(phantom=random_water_bone_object(seed, k))
    return simulate(sc, n_events=n_events, seed=seed * 1000 + k, workers=1)


def train_surrogate_on_random_objects(sc, n_objects, n_samples, object_events, seed):
    """A surrogate trained on n_samples exact single-scatter sums drawn from
    n_objects random water/bone objects on the workload's grid (never the
    workload's own object).  Returns (surrogate, sampling s, training s,
    schedule, batch)."""
    import multiprocessing as mp

    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import random_water_bone_object

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    with mp.get_context("spawn").Pool(min(n_objects, os.cpu_count() or 1)) as pool:
        obj_events = pool.map(_object_events,
                              [(k, seed, sc.name, object_events) for k in range(n_objects)])
    xs, ts, t_sample = [], [], 0.0
    for k in range(n_objects):
        sck = sc.with_(phantom=random_water_bone_object(seed, k))
        mk = lm.Model.from_scenario(sck, sck.make_phantom().rho)
        dk = lm.DeviceEvents.from_list(obj_events[k])
        (x, t), dt = timed(lambda: mk.surrogate_samples(dk, n_samples // n_objects,
                                                        seed=seed * 100 + k))
        xs.append(x)
        ts.append(t)
        t_sample += dt
        mk.close()
        del dk
    x, t = torch.cat(xs), torch.cat(ts)
    del xs, ts
    sur = lm.Surrogate(seed)
    batch = 16384
    schedule = ((2000, 2e-3), (1500, 6e-4), (500, 2e-4))

    def train():
        for steps, lr in schedule:
            sur.train(x, t, steps=steps, batch=batch, lr=lr, seed=seed * 10 + steps,
                      weight_power=0.5, record_loss=False)
    _, t_train = timed(train)
    return sur, t_sample, t_train, schedule, batch


def run_surrogate_form(workload="lmmew_128_2m", n_objects=8, n_samples=10_000_000,
                       object_events=20_000, iters=10, seed=5):
    """The learned single-scatter surrogate against the exact FP32 path on the
    same GPU, on the 128 x 128, 2 M-event workload.  The network is trained
    on 10^7 exact single-scatter sums drawn (lm_surrogate_sample) from eight
    random water/bone objects on the same grid -- never from the workload's
    own object -- with the loss weighted by the square root of the scatter
    mass.  Reported: sampling and training time, the mass-weighted error of
    the scatter sum on samples of the workload's object, seconds per OSEM
    iteration and network throughput, and the deviation of forward
    projections, images and lesion activities from the exact path -- next to
    the same deviations of the model without scatter, which is what the
    surrogate has to beat."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate_cached
    sc = preset(workload)
    ph = sc.make_phantom()
    ev = simulate_cached(sc)

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    sur, t_sample, t_train, schedule, batch = train_surrogate_on_random_objects(
        sc, n_objects, n_samples, object_events, seed)

    model = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    xv, tv = model.surrogate_samples(dev, 200_000, seed=8)
    sv = torch.exp(tv.double()) - 1e-8
    pe = torch.clamp(torch.exp(sur.forward(xv).double()) - 1e-8, min=0)
    mass_err = float(torch.sum(torch.abs(pe - sv)) / torch.sum(sv))
    mass_ratio = float(torch.sum(pe) / torch.sum(sv))
    del xv, tv

    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    lam_true = torch.from_numpy(ph.activity.reshape(-1).astype(np.float32)).cuda()
    res = {}
    kinds = ("exact", "surrogate", "surrogate_coarse", "surrogate_coarse_s3", "surrogate_coarse_s4",
             "none")
    for kind in kinds:
        # the coarse grid's node stride in pixels: 2, or the suffix's
        stride = int(kind[-1]) if kind[-3:-1] == "_s" else 2
        model.set_coarse_stride(stride)
        model.set_scatter_model(kind[:-3] if kind[-3:-1] == "_s" else kind,
                                sur if kind.startswith("surrogate") else None)
        y = model.forward(dev, lam_true).cpu().numpy().astype(np.float64)   # also warms up
        model.osem(dev, lam0.clone(), sc.n_subsets, 0)   # untimed: the row-kernel autotune
        img = lam0.clone()
        _, sec = timed(lambda: model.osem(dev, img, sc.n_subsets, iters))
        res[kind] = {"y": y, "img": img.cpu().numpy().astype(np.float64), "s_per_iter": sec / iters}
    model.set_scatter_model("exact")
    model.set_coarse_stride(2)
    ex = res["exact"]
    roi_ex = roi_sums(ex["img"], ph.lesion_masks)
    samples_per_iter = surrogate_samples_in_reach(sc, ev.energy, model.nq)
    dense_samples_per_iter = len(ev) * model.nq * len(sc.line_keV)
    flop_per_sample = 2 * (32 * 128 + 2 * 128 * 128) + 2 * 128
    out = {"workload": f"{sc.name}: {sc.n}x{sc.n}, {sc.n_angles} angles, {sc.n_bins} bins, "
                       f"{sc.scatter_n}x{sc.scatter_n} scatter grid, {len(ev)} events, "
                       f"{sc.n_subsets} subsets x {iters} iterations",
           "training": {"objects": f"{n_objects} random water/bone ellipses (seed {seed}), "
                                    f"{object_events} MC events each; the workload's object "
                                    "is not among them",
                        "samples": n_samples, "sample_s": t_sample, "train_s": t_train,
                        "steps": sum(k for k, _ in schedule), "batch": batch,
                        "loss_weight": "(S + 1e-8)^0.5",
                        "heldout_object_mass_rel_err": mass_err,
                        "heldout_object_mass_ratio": mass_ratio},
           "exact": {"s_per_iter": ex["s_per_iter"], "roi_activity": roi_ex}}
    for kind in kinds[1:]:
        r = res[kind]
        roi = roi_sums(r["img"], ph.lesion_masks)
        out[kind] = {"s_per_iter": r["s_per_iter"],
                     "speedup_vs_exact": ex["s_per_iter"] / r["s_per_iter"],
                     "fwd_rel_l2_vs_exact": float(np.linalg.norm(r["y"] - ex["y"])
                                                  / np.linalg.norm(ex["y"])),
                     "image_rel_l2_vs_exact": float(np.linalg.norm(r["img"] - ex["img"])
                                                    / np.linalg.norm(ex["img"])),
                     "roi_rel_dev_vs_exact": [abs(a - b) / b for a, b in zip(roi, roi_ex)]}
    out["surrogate"]["network_samples_per_iter"] = samples_per_iter
    out["surrogate"]["samples_in_reach_fraction"] = samples_per_iter / dense_samples_per_iter
    out["surrogate"]["network_samples_per_s"] = samples_per_iter / res["surrogate"]["s_per_iter"]
    out["surrogate"]["network_tflops"] = (samples_per_iter * flop_per_sample
                                          / res["surrogate"]["s_per_iter"] / 1e12)
    sur.close()
    model.close()
    return out


def run_batch_forms():
    """The batching form on two workloads: the scope's 256 realisations of
    U[50k, 500k] events at 64^2 through 8 subsets x 10 iterations each
    (run_c3_forms, with the combined form on the same realisations), and
    256 realisations of the paper's own study (64^2 of 4.6 mm, 120 angles,
    three windows, U[8k, 12k] events around its ~10^4 per realisation,
    4 subsets x 16 iterations), where every single reconstruction is too
    small to fill the GPU."""
    return {"lmmew_64_256": run_c3_forms(),
            "paper_study_256": run_batch_form(workload="paper_study", lo=8_000, hi=12_000,
                                              iters=None, repeats=2, seed=31)}


def run_c3_forms(workload="lmmew_64", n_real=256, lo=50_000, hi=500_000, seed=3,
                 n_objects=8, n_samples=4_000_000, sur_seed=6):
    """256 independent noise realisations of the 64 x 64 object with event
    counts drawn uniformly from [50k, 500k] (seed 3), each through 8 subsets x
    10 iterations.  The realisations are disjoint consecutive slices of one
    pool of iid Monte-Carlo events (the torch port of the MC on the GPU,
    seed 3): independent noise realisations.  Timed on the same GPU:
      exact FP32 one realisation at a time (each reconstruction's own time:
        p50 / p99 over the 256);
      exact FP32 batched: all realisations in one lm_osem_batch call (one
        persistent row launch per row block and sub-iteration over every
        realisation, the reconstruction replayed as one CUDA graph, autotuned
        launch shape); every reconstruction completes when the call does;
      the combined form: the same batched call with the scatter part from
        the BF16 tensor-core surrogate on the coarse grid, trained on random
        water/bone objects (not this object), with every realisation's
        lesion activities against its exact reconstruction.
    Each batched call is preceded by an untimed one-iteration call that
    tunes the launch shape and warms up."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import mc_torch, preset
    sc = preset(workload)
    ph = sc.make_phantom()
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=n_real)
    off = np.concatenate([[0], np.cumsum(sizes)])
    t0 = time.time()
    pool = mc_torch.simulate(sc, int(off[-1]), seed=seed, device="cuda")
    t_pool = time.time() - t0
    devs = [lm.DeviceEvents(pool.angle[off[r]:off[r + 1]], pool.bin[off[r]:off[r + 1]],
                            pool.energy[off[r]:off[r + 1]]) for r in range(n_real)]
    del pool
    model = lm.Model.from_scenario(sc, ph.rho)
    n_it = sc.n_iters
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    # exact FP32, one realisation at a time (the untimed calls with no
    # iteration sort and run the row-kernel autotune of each class: set-up)
    for d in devs:
        model.osem(d, lam0.clone(), sc.n_subsets, 0)
    seq, exact_roi = [], []
    for d in devs:
        img = lam0.clone()
        seq.append(timed(lambda: model.osem(d, img, sc.n_subsets, n_it)))
        exact_roi.append(roi_sums(img.cpu().numpy().astype(np.float64), ph.lesion_masks))
    seq = np.asarray(seq)

    def batched():
        imgs = lam0.repeat(n_real, 1).contiguous()
        model.osem_batch(devs, imgs, sc.n_subsets, 1)          # tunes, warms up
        imgs = lam0.repeat(n_real, 1).contiguous()
        sec = timed(lambda: model.osem_batch(devs, imgs, sc.n_subsets, n_it))
        return sec, imgs.cpu().numpy().astype(np.float64)

    t_batch, imgs_b = batched()
    tune = model.batch_tuning()
    dev_b = max(abs(a - b) / b for r in range(n_real)
                for a, b in zip(roi_sums(imgs_b[r], ph.lesion_masks), exact_roi[r]))
    elems = float(off[-1]) * model.nq * n_it
    out = {"workload": f"{n_real} realisations of {sc.name} with U[{lo}, {hi}] events (seed "
                       f"{seed}, {int(off[-1])} events: disjoint slices of one iid MC pool), "
                       f"{sc.n_subsets} subsets x {n_it} iterations each",
           "pool": {"generator": "synthetic.mc_torch on the GPU", "events": int(off[-1]),
                    "generation_s": t_pool},
           "one_at_a_time": {"realisations_per_s": n_real / float(seq.sum()),
                             "elements_per_s": elems / float(seq.sum()),
                             "recon_s_p50": float(np.percentile(seq, 50)),
                             "recon_s_p99": float(np.percentile(seq, 99)),
                             "total_s": float(seq.sum())},
           "batched": {"realisations_per_s": n_real / t_batch,
                       "elements_per_s": elems / t_batch,
                       "batch_s": t_batch,
                       "recon_latency_s": t_batch,
                       "roi_max_rel_dev_vs_one_at_a_time": float(dev_b),
                       "tuning": tune},
           "speedup_batched_vs_one_at_a_time": float(seq.sum()) / t_batch}
    # the combined form on the same realisations
    sur, t_sample, t_train, _, _ = train_surrogate_on_random_objects(
        sc, n_objects, n_samples, 20_000, sur_seed)
    out["combined"] = {"form": "BF16 tensor-core surrogate on the coarse grid (node stride 2 "
                               "or 3 pixels) + batched realisations in one CUDA graph",
                       "surrogate_training": {"objects": n_objects, "samples": n_samples,
                                              "sample_s": t_sample, "train_s": t_train}}
    for stride in (2, 3):
        model.set_coarse_stride(stride)
        model.set_scatter_model("surrogate_coarse", sur)
        t_comb, imgs_c = batched()
        model.set_scatter_model("exact")
        dev = np.asarray([[abs(a - b) / b for a, b in zip(roi_sums(imgs_c[r], ph.lesion_masks),
                                                           exact_roi[r])] for r in range(n_real)])
        out["combined"][f"stride_{stride}"] = {
            "batch_s": t_comb,
            "speedup_vs_exact_fp32_one_at_a_time": float(seq.sum()) / t_comb,
            "speedup_vs_exact_fp32_batched": t_batch / t_comb,
            "roi_rel_dev_vs_exact": {"mean": float(dev.mean()), "max": float(dev.max()),
                                     "per_lesion_mean": dev.mean(axis=0).tolist()}}
    model.set_coarse_stride(2)
    sur.close()
    model.close()
    return out


def run_batch_form(workload="lmmew_64", n_real=256, lo=50_000, hi=500_000, iters=1, repeats=2,
                   seed=3):
    """Many noise realisations with uneven event counts in one batched call
    (persistent row launch per sub-iteration over all realisations, the whole
    reconstruction replayed as one CUDA graph, autotuned launch shape) against
    the same realisations reconstructed one call at a time.  256 realisations
    of U[50k, 500k] events (~70 M events); one full OSEM iteration (all
    subsets) per realisation keeps the form within a minute, and the
    per-iteration cost is what the 8 x 10 schedule repeats."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate_cached
    sc = preset(workload)
    ph = sc.make_phantom()
    pool = simulate_cached(sc, n_events=max(sc.n_events, 100_000))
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=n_real)
    # realisations drawn from one iid Monte-Carlo pool (with replacement)
    evs = [pool.subset(rng.integers(0, len(pool), size=int(k))) for k in sizes]
    devs = [lm.DeviceEvents.from_list(e) for e in evs]
    model = lm.Model.from_scenario(sc, ph.rho)
    n_it = sc.n_iters if iters is None else iters
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # one realisation at a time; the row-kernel autotune of each event count's
    # class is set-up (once per handle and class, like the tables), so it runs
    # untimed first: lm_osem with no iteration only sorts and tunes
    for d in devs:
        model.osem(d, lam0.clone(), sc.n_subsets, 0)
    seq = []
    for d in devs:
        img = lam0.clone()
        torch.cuda.synchronize()
        e0.record()
        model.osem(d, img, sc.n_subsets, n_it)
        e1.record()
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1) / 1e3)
    # batched
    imgs = lam0.repeat(n_real, 1).contiguous()
    model.osem_batch(devs, imgs, sc.n_subsets, n_it)      # tunes + warms up
    torch.cuda.synchronize()
    batch = []
    for _ in range(repeats):
        imgs = lam0.repeat(n_real, 1).contiguous()
        torch.cuda.synchronize()
        e0.record()
        model.osem_batch(devs, imgs, sc.n_subsets, n_it)
        e1.record()
        torch.cuda.synchronize()
        batch.append(e0.elapsed_time(e1) / 1e3)
    tune = model.batch_tuning()
    model_nq = model.nq
    model.close()
    return {"workload": f"{n_real} realisations of {sc.name} with U[{lo}, {hi}] events "
                        f"(seed {seed}, {int(sizes.sum())} events, drawn from one MC pool), "
                        f"{sc.n_subsets} subsets x {n_it} iterations each",
            "batched": {"realisations_per_s": n_real / float(np.median(batch)),
                        "realisation_iterations_per_s": n_real * n_it / float(np.median(batch)),
                        "elements_per_s": float(sizes.sum()) * model_nq * n_it / float(np.median(batch)),
                        "batch_s_p50": float(np.percentile(batch, 50)),
                        "batch_s_p99": float(np.percentile(batch, 99)),
                        "tuning": tune},
            "one_at_a_time": {"realisations_per_s": n_real / float(np.sum(seq)),
                              "recon_s_p50": float(np.percentile(seq, 50)),
                              "recon_s_p99": float(np.percentile(seq, 99))},
            "speedup_batched_vs_one_at_a_time": float(np.sum(seq) / np.median(batch))}


def run_streamed_form(workload="lmmew_64", iters=2, blocks=(8, 1)):
    """Streamed path tables (the fallback for models whose tables exceed the
    device memory) against resident tables at the benchmark's workload:
    seconds per OSEM iteration with the tables of `blocks` angles kept at a
    time, and whether the image equals the resident one bit for bit."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate_cached
    sc = preset(workload)
    ph = sc.make_phantom()
    ev = simulate_cached(sc)
    model = lm.Model.from_scenario(sc, ph.rho)
    model.set_tile_events(64)
    dev = lm.DeviceEvents.from_list(ev)
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()

    def timed():
        img = lam0.clone()
        model.osem(dev, img, sc.n_subsets, 1)   # warm-up (resident: tunes once)
        img = lam0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        model.osem(dev, img, sc.n_subsets, iters)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / iters, img
    t_res, img_res = timed()
    out = {"workload": f"{sc.name}: {len(ev)} events, {sc.n_subsets} subsets x {iters} iterations",
           "resident": {"s_per_iter": t_res, "table_bytes": model.table_streaming()[1]}}
    for k in blocks:
        model.set_table_streaming(k)
        t, img = timed()
        out[f"blocks_of_{k}"] = {"s_per_iter": t, "table_bytes": model.table_streaming()[1],
                                 "slowdown": t / t_res,
                                 "image_bit_identical": bool(torch.equal(img, img_res))}
    model.close()
    return out


def run_comparison_form(noise_realisations=16, events=10_000, seed=21):
    """The paper's comparison (LM-MEW vs LM-SEW vs Binned-SEW) on its study
    object and protocol: ensemble normalised RMSE, bias and standard
    deviation of the four lesions' uptake."""
    import time as _time

    from paper_2305_17111_gb300 import studies
    from synthetic import preset
    sc = preset("paper_study")
    t0 = _time.perf_counter()
    res = studies.run_study(sc, noise_realisations, events, seed=seed)
    wall = _time.perf_counter() - t0
    out = {"workload": f"paper_study: 64x64 of 4.6 mm, 120 angles, EW1-EW3, lesions r = "
                       f"7/10/12/14 mm at SBR 4:1, {noise_realisations} noise realisations x "
                       f"{events} events (seed {seed}), {sc.n_subsets} subsets x {sc.n_iters} "
                       f"iterations", "wall_s_incl_event_generation": wall}
    for name, r in res.items():
        out[name] = {"events_mean": r["events_mean"],
                     "enrmse": [float(v) for v in r["enrmse"]],
                     "bias": [float(v) for v in r["bias"]],
                     "std": [float(v) for v in r["std"]]}
    # the other signal-to-background ratios of the study (ENRMSE per lesion)
    from synthetic.phantom import paper_study_phantom
    out["sbr_sweep_enrmse"] = {}
    for sbr in (2.0, 6.0):
        rs = studies.run_study(sc.with_(phantom=paper_study_phantom(sbr)), noise_realisations,
                               events, seed=seed)
        out["sbr_sweep_enrmse"][f"{sbr:g}:1"] = {name: [float(v) for v in r["enrmse"]]
                                                 for name, r in rs.items()}
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, local_rank, world):
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate_cached

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    sc = preset(args.workload)
    if args.events:
        sc = sc.with_(n_events=args.events)
    ph = sc.make_phantom()
    # every rank reconstructs its own noise realisation (seed + rank)
    ev = simulate_cached(sc, seed=sc.seed + rank)
    model = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    img = lam0.clone()
    n_sub = sc.n_subsets
    J, nq = len(ev), model.nq

    def barrier():
        if dist is not None:
            dist.barrier()

    it = 0
    for _ in range(args.warmup):
        model.osem(dev, img, n_sub, it + 1, start_iter=it)
        it += 1
    torch.cuda.synchronize()
    model.profile_read()                      # reset counters
    model.profile_enable(True)
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # the K timed steps are K LM-OSEM iterations of one lm_osem call, as a
    # reconstruction runs them (the events are sorted once per call)
    model.osem(dev, img, n_sub, it + args.steps, start_iter=it)
    it += args.steps
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = model.profile_read()
    model.profile_enable(False)
    row_tuning = model.batch_tuning()           # the launch shape the timed steps ran
    ms = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms / args.steps
    elems_step = J * nq
    value = whole_job_throughput(elems_step, args.steps, world, ms)

    ms_e2e, h2d, d2h = None, 0, 0
    if not args.no_e2e:
        ms_e2e, h2d, d2h, it = run_e2e(model, ev, img, sc, n_sub, it, args.steps, stream, barrier,
                                       dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(local_rank)
    sm_count = props.multi_processor_count
    peaks = measured_peaks() or {}
    sm_max = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    peak = ex2_peak(sm_count, sm_max)
    achieved = prof["terms"] / (prof["ms"] / 1e3) if prof["ms"] > 0 else 0.0
    probe = lm.probe_ex2_rate()          # measured exponential rate of this GPU
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(sc, nq, model.np_scatter),
                       l2="inputs larger than L2: %.2f GB of path tables stream every step"
                          % (model.table_bytes / 1e9),
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       timed="the K steps as K iterations of one lm_osem call (events sorted "
                             "once per call); e2e: one call per step with the step's host "
                             "copies"),
        "s_per_osem_iter": ms_per_step / 1e3,
        "terms_per_s": prof["terms"] / (ms / 1e3) if ms > 0 else None,
        "terms_evaluated_per_step": prof["terms"] / args.steps,
        "terms_dense_per_step": float(model.terms_per_event) * J,
        "setup_ms": model.setup_ms,
        "clocks": clk,
        "e2e": ({"value": whole_job_throughput(elems_step, args.steps, world, ms_e2e), "unit": UNIT,
                 "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h} if ms_e2e else None),
        "gpu_launches": int(prof["kernels"]),
        "roofline": {"bound": "alu", "kernel": "k_row (fused row + forward)",
                     "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tex2/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": (ROW_TRAFFIC_BYTES_PER_LAUNCH.get(sc.name)
                                 if not args.events else None),
                     "peak_basis": f"{sm_count} SMs x {EX2_PER_SM_PER_CLK} ex2/clk x "
                                   f"{sm_max:.0f} MHz",
                     "peak_probe": probe["f32"] * sm_count * probe["sm_mhz"] * 1e6 / 1e12,
                     "probe_ex2_per_clk_per_sm": {k: probe[k] for k in ("f32", "f16x2", "bf16x2")},
                     "row_kernel_share": prof["ms"] / ms if ms > 0 else None,
                     "row_tuning": row_tuning},
    }
    if world == 1 and not args.no_forms and not args.events:
        model.close()
        runners = {"precision": run_precision_form, "batching": run_batch_forms,
                   "comparison": run_comparison_form, "surrogate": run_surrogate_form,
                   "streamed": run_streamed_form}
        line["forms"] = {k: runners[k]() for k in args.forms.split(",") if k in runners}
        # the metric's third part: the chosen forms against the plain FP32
        # path on the same GPU, at the stated ROI-activity error, at the
        # forms' own workloads
        chosen = {"form": "BF16 tensor-core surrogate on the coarse grid (+ batched "
                          "realisations in one CUDA graph where there are several)"}
        c3 = line["forms"].get("batching", {}).get("lmmew_64_256", {}).get("combined")
        if c3:
            chosen["realisations_256"] = {
                "workload": line["forms"]["batching"]["lmmew_64_256"]["workload"]}
            for k in ("stride_2", "stride_3"):
                chosen["realisations_256"][k] = {
                    "speedup_vs_plain_fp32_one_at_a_time": c3[k]["speedup_vs_exact_fp32_one_at_a_time"],
                    "speedup_vs_plain_fp32_batched": c3[k]["speedup_vs_exact_fp32_batched"],
                    "roi_rel_dev_vs_plain_fp32": c3[k]["roi_rel_dev_vs_exact"]}
        c4 = line["forms"].get("surrogate")
        if c4:
            chosen["single_128_2m"] = {"workload": c4["workload"]}
            for k, kind in (("stride_2", "surrogate_coarse"), ("stride_3", "surrogate_coarse_s3"),
                            ("stride_4", "surrogate_coarse_s4")):
                chosen["single_128_2m"][k] = {
                    "speedup_vs_plain_fp32": c4[kind]["speedup_vs_exact"],
                    "roi_rel_dev_vs_plain_fp32": c4[kind]["roi_rel_dev_vs_exact"]}
        if len(chosen) > 1:
            line["chosen_form"] = chosen
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def surrogate_samples_in_reach(sc, energies, nq):
    """(event, voxel, line) samples the surrogate evaluates: the recorded
    energy inside the line's single-scatter reach (backscatter energy to E_w,
    widened by 8 energy-resolution sigmas, the library's rule), times nq."""
    import numpy as np

    def sigma_e(e):
        return (sc.fwhm_frac * e * (e / sc.e_ref_keV) ** sc.fwhm_exponent
                / (2 * np.sqrt(2 * np.log(2))))
    e_hat = np.asarray(energies, dtype=np.float64)
    reachable = 0
    for e_w in sc.line_keV:
        e_back = e_w / (1 + 2 * e_w / 510.99895)
        reachable += int(np.count_nonzero((e_hat >= e_back - 8 * sigma_e(e_back))
                                          & (e_hat <= e_w + 8 * sigma_e(e_w))))
    return reachable * nq


def run_surrogate_rows_case(n_events=20_000, repeats=3):
    """Small case for profiling the surrogate row kernel: the 64 x 64 object,
    20 000 MC events, lm_forward with the surrogate scatter model (untrained
    weights: the work does not depend on them).  Prints one JSON line."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate
    sc = preset("lmmew_64")
    ph = sc.make_phantom()
    ev = simulate(sc, n_events=n_events, seed=3)
    model = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    sur = lm.Surrogate(1)
    model.set_scatter_model("surrogate", sur)
    lam = torch.from_numpy(ph.activity.reshape(-1).astype(np.float32)).cuda()
    times = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        model.forward(dev, lam)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    model.set_scatter_model("exact")
    samples = surrogate_samples_in_reach(sc, ev.energy, model.nq)
    ms = min(times)
    print(json.dumps({"case": "surrogate_rows", "events": len(ev), "samples": samples,
                      "samples_dense": len(ev) * model.nq * len(sc.line_keV),
                      "ms": ms, "samples_per_s": samples / ms * 1e3,
                      "tflops": samples * (2 * (32 * 128 + 2 * 128 * 128) + 256) / ms / 1e9}),
          flush=True)
    sur.close()
    model.close()
    return 0


def run_row_case(n_events=60_000, tile_events=64, repeats=3, store_rows=False):
    """Small case for profiling the exact row kernel in the launch shape the
    benchmark's workload uses: the 64 x 64 object (its 1.6 GB of path
    tables), n_events MC events of the subset-0 angles (8 angles, about one
    lm_osem sub-iteration's work), tiles of tile_events; lm_forward (forward
    sums only) or, with store_rows, lm_backproject (the row block written, as
    lm_osem's launches do).  One row-kernel launch per call.  Prints one
    JSON line."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate
    sc = preset("lmmew_64")
    ph = sc.make_phantom()
    ev = simulate(sc, n_events=8 * n_events, seed=3)
    ev = ev.subset(np.nonzero(ev.angle % sc.n_subsets == 0)[0][:n_events])
    model = lm.Model.from_scenario(sc, ph.rho)
    model.set_tile_events(tile_events)
    dev = lm.DeviceEvents.from_list(ev)
    lam = torch.from_numpy(ph.activity.reshape(-1).astype(np.float32)).cuda()
    wt = torch.ones(len(ev), dtype=torch.float32, device="cuda")

    def call():
        if store_rows:
            model.backproject(dev, wt)
        else:
            model.forward(dev, lam)
    model.profile_enable(True)
    call()
    model.profile_read()
    for _ in range(repeats):
        call()
    prof = model.profile_read()
    model.profile_enable(False)
    print(json.dumps({"case": "row_rows" if store_rows else "row", "events": len(ev),
                      "tile_events": tile_events,
                      "row_ms": prof["ms"] / repeats, "terms": prof["terms"] / repeats,
                      "Tterms_per_s": prof["terms"] / (prof["ms"] / 1e3) / 1e12}), flush=True)
    model.close()
    return 0


def run_surrogate_coarse_osem_case(n_events=200_000, repeats=2):
    """Small case for the launch list of the coarse-grid surrogate form: the
    128 x 128 object, 200 000 MC events, OSEM iterations of 8 subsets with
    the surrogate evaluated on the half-resolution node grid (untrained
    weights: the work does not depend on them).  One untimed iteration tunes
    the row kernel; then `repeats` iterations are timed one by one.  Prints
    one JSON line."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    from synthetic import preset, simulate
    sc = preset("lmmew_128")
    ph = sc.make_phantom()
    ev = simulate(sc, n_events=n_events, seed=3)
    model = lm.Model.from_scenario(sc, ph.rho)
    dev = lm.DeviceEvents.from_list(ev)
    sur = lm.Surrogate(1)
    model.set_scatter_model("surrogate_coarse", sur)
    lam0 = torch.from_numpy((ph.rho.reshape(-1) > 0).astype(np.float32)).cuda()
    img = lam0.clone()
    model.osem(dev, img, sc.n_subsets, 1)
    times = []
    for _ in range(repeats):
        img.copy_(lam0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        model.osem(dev, img, sc.n_subsets, 1)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"case": "surrogate_coarse_osem", "events": len(ev), "voxels": model.nq,
                      "subsets": sc.n_subsets, "ms_per_iter": times}), flush=True)
    model.set_scatter_model("exact")
    sur.close()
    model.close()
    return 0


def run_setup_case(workload, repeats=2):
    """Small case for profiling the set-up kernels: `lm_create` of the named
    workload's model `repeats` times (no events).  Prints one JSON line."""
    import paper_2305_17111_gb300 as lm
    from synthetic import preset
    sc = preset(workload)
    ph = sc.make_phantom()
    times = []
    for _ in range(repeats):
        model = lm.Model.from_scenario(sc, ph.rho)
        times.append(model.setup_ms)
        model.close()
    print(json.dumps({"case": "setup", "workload": workload, "setup_ms": times}), flush=True)
    return 0


def run_surrogate_train_case(steps=10, batch=16_384, n=200_000):
    """Small case for profiling one surrogate training step: Adam on
    minibatches of 16 384 of 200 000 random inputs (2 warm-up steps, then
    `steps` steps without per-step loss read-back).  Prints one JSON line."""
    import numpy as np
    import torch

    import paper_2305_17111_gb300 as lm
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.normal(0, 1, (n, 32)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(-10, 2, n).astype(np.float32)).cuda()
    sur = lm.Surrogate(seed=3)
    sur.train(x, t, steps=2, batch=batch, lr=1e-3, record_loss=False)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    sur.train(x, t, steps=steps, batch=batch, lr=1e-3, record_loss=False)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"case": "surrogate_train", "batch": batch, "steps": steps,
                      "ms_per_step": e0.elapsed_time(e1) / steps}), flush=True)
    sur.close()
    return 0


def main():
    args = parse_args()
    rank, local_rank, world = dist_env()
    if args.case in ("row", "row_rows"):
        return run_row_case(n_events=args.events or 60_000, store_rows=args.case == "row_rows")
    if args.case == "surrogate_rows":
        return run_surrogate_rows_case()
    if args.case == "surrogate_train":
        return run_surrogate_train_case()
    if args.case == "surrogate_coarse_osem":
        return run_surrogate_coarse_osem_case()
    if args.case == "setup":
        return run_setup_case(args.workload)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, local_rank, world)


if __name__ == "__main__":
    sys.exit(main())
