"""profiles/traffic.json: each record names an existing kernel source and the workload it
was captured on, keyed as bench.py looks it up ("<kernel form> @ <workload>"), and every
form bench.py can report for its default workload has a key of that shape."""
import json
import os

import bench
from paper_2401_12890_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def records():
    return json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))


def test_record_structure():
    for key, rec in records().items():
        name, _, wl = key.partition(" @ ")
        assert name and wl == rec["bench_workload"], key
        assert wl in synth.WORKLOADS or wl == synth.B1_WORKLOAD.name, key
        assert os.path.exists(os.path.join(ROOT, rec["source"])), key
        assert rec["dram_bytes_per_launch_full"] == rec["dram_read"] + rec["dram_write"]
        assert len(rec["source_sha"]) == 16 and "ncu" in rec["command"]
        assert "--clock-control none" in rec["command"]


def test_lookup_keys_match_bench():
    keys = set(records())
    for form, prec, fused in [("dense", "bf16x3", 0), ("dense", "bf16x3", 1),
                              ("lowrank", "fp32", 0)]:
        name, kfile, *_, tkey = bench.dominant_kernel(form, prec, 2500, 16384, 20, fused)
        assert f"{tkey} @ {bench.WORKLOAD}" in keys, tkey
        assert os.path.exists(os.path.join(ROOT, "paper_2401_12890_gb300", "csrc", kfile))
