"""bench.py's reference arm (the FP64 oracle on the host cores) keeps the JSON-line
contract. No GPU: the arm never touches one. It is run as a subprocess, once on a small
workload (--workload, for speed) and once on the default workload the metric is quoted
on, with one step each."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e"}


def run(*extra):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0", *extra], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


@pytest.mark.parametrize("extra,name", [(("--workload", "dr2d_tiny"), "dr2d_tiny"),
                                        ((), "dr2d_slice")])
def test_reference_line(extra, name):
    line = run(*extra)
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["metric"] == line["unit"]
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith(name + ":")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
