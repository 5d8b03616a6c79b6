"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
keeps the JSON contract: one line with the arm's metric, unit and direction,
the oracle as its CPU baseline and a zero-copy end-to-end figure.  CPU only,
on the small 32 x 32 workload."""
from __future__ import annotations

import argparse
import json

import bench


def test_reference_arm_json_line(capsys):
    args = argparse.Namespace(workload="lmmew_32", steps=1, warmup=1)
    assert bench.run_reference(args, rank=0, world=1) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"],
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("lmmew_32")


def test_reference_arm_other_ranks_do_no_work(capsys):
    args = argparse.Namespace(workload="lmmew_32", steps=1, warmup=1)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
