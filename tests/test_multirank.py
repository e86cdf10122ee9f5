"""The N > 1 path of bench.py on CPU: world size 2 over gloo on 127.0.0.1, no GPU.

Under torchrun every rank solves its own seeded problem with no collective on the data
path; the ranks meet only at barriers around the timed region and in the max over their
step times, and rank 0 alone prints. These tests run that host logic as two real
processes: the barrier and max of bench.Dist, the whole-job value built from the max, the
per-rank seeds, and the reference arm under torch.distributed.run (rank 0 prints one
line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
d = bench.Dist("gloo")
d.barrier()
local_ms = 10.0 * (d.rank + 1)            # rank 1 is the slower one
ms_max = d.max(local_ms)
d.barrier()
out = {{"rank": d.rank, "world": d.world, "ms_max": ms_max,
        "value": bench.weak_value(d.world, 1000, 50, ms_max / 1e3),
        "seed": bench.rank_seed(17, d.rank)}}
d.close()
print(json.dumps(out))
"""


def run_ranks(world):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e
        outs.append(json.loads([l for l in o.splitlines() if l.startswith("{")][-1]))
    return sorted(outs, key=lambda x: x["rank"])


def test_dist_barrier_and_max_over_two_ranks():
    outs = run_ranks(2)
    assert [o["rank"] for o in outs] == [0, 1] and all(o["world"] == 2 for o in outs)
    # every rank sees the slowest rank's time, so every rank reports the same value
    assert all(o["ms_max"] == 20.0 for o in outs)
    expect = 2 * 1000 * 50 * 100 / 0.020
    assert all(o["value"] == pytest.approx(expect, rel=1e-12) for o in outs)
    # distinct problems per rank
    assert outs[0]["seed"] != outs[1]["seed"]


def test_weak_value_and_single_rank():
    import bench
    # one rank: the plain rate of its own problem
    assert bench.weak_value(1, 16384, 2500, 0.012) == pytest.approx(
        16384 * 2500 * bench.ITERS_PER_STEP / 0.012)
    # weak scaling: N ranks at the same step time do N times the work
    assert bench.weak_value(4, 10, 10, 1.0) == 4 * bench.weak_value(1, 10, 10, 1.0)
    d = bench.Dist("gloo")   # WORLD_SIZE unset: no process group, max is the identity
    assert d.world == 1 and d.max(3.5) == 3.5
    d.barrier()
    d.close()


def test_rank_seeds_give_distinct_reproducible_problems():
    import bench
    from paper_2401_12890_gb300 import synth
    w = synth.WORKLOADS["dr2d_tiny"]
    _, M0, _ = synth.make_problem("dr2d_tiny", seed=bench.rank_seed(w.seed, 0))
    _, M1, _ = synth.make_problem("dr2d_tiny", seed=bench.rank_seed(w.seed, 1))
    _, M0b, _ = synth.make_problem("dr2d_tiny", seed=bench.rank_seed(w.seed, 0))
    assert M0.shape == M1.shape
    assert not (M0 == M1).all()
    assert (M0 == M0b).all()
    assert bench.rank_seed(w.seed, 0) == w.seed


def test_reference_arm_under_torchrun_two_ranks():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload",
           "dr2d_tiny"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout            # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"].startswith("dr2d_tiny:")
