"""Write tests/golden/longrun.json from the FP64 oracle only: long runs of Algorithm 2.

Algorithm 2's objective on these problems approaches its minimum very slowly: the
components of z in the null space of K are shaped only by the smoothness term, so the
last stretch of the iteration contracts by a factor close to 1. On the 32x32 workload the
objective still falls by ~5e-8 (of ~0.95) per 1000 iterations after 128000 iterations,
with a ratio of ~0.996 between consecutive 1000-iteration decreases; running to a change
of 1e-12 would take millions of FP64 iterations. So the reference values are the
oracle's objective after fixed, long iteration counts from the zero start -- which the
GPU forms reproduce iteration for iteration -- plus, for the 32x32 workload, an estimate
of the limit from the geometric tail of the last blocks.

  dr2d_tiny (32x32, P = 30, Q = 225): the full-rank (Eq. 26, objective with K) and the
      low-rank (Eq. 28, rank rule, objective with K_r) iterations, in blocks of 1000
      iterations each continuing from the previous block's state (z, d): J at 300, 3000,
      30000 and 100000 iterations; the decrease over the last two blocks; J_limit_est =
      J_100000 - delta * rho / (1 - rho) with delta the last block's decrease and rho the
      ratio of the last two decreases.
  dr2d_slice (128x128, P = 120, Q = 2500): the full-rank iteration for 2000 iterations
      (past the residual stopping rule at 3e-4, which stops near 1070), in blocks of 100.

Run:  python tests/golden/make_longrun.py [dr2d_tiny|dr2d_slice ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ladmm as L  # noqa: E402
from paper_2401_12890_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "longrun.json")


def objective_for(K, M, z, w, dense, r):
    Kf = K if dense else L.truncated_dictionary(K, r)
    return L.objective(Kf, M, z, w.dims, w.lam)


def long_run(name, dense, marks, block):
    """J after each count in `marks` (ascending), continuing block by block."""
    w = synth.WORKLOADS[name]
    K = synth.dictionary_for(name)
    M = synth.make_problem(name)[1].astype(np.float64)
    z = d = None
    k, r = 0, None
    at, trail = {}, []
    t0 = time.time()
    todo = list(marks)
    while todo:
        step = min(block, todo[0] - k)
        res = L.ladmm(K, M, w.dims, w.lam, w.beta, dense=dense, iters=step, check_every=0,
                      z0=z, d0=d)
        z, d, r = res["z"], res["d"], res["r"]
        k += step
        if step == block or k == todo[0]:
            J = objective_for(K, M, z, w, dense, r)
            trail.append((k, J))
            print(f"{name} dense={dense} k={k} J={J!r} ({time.time() - t0:.0f} s)", flush=True)
        if k == todo[0]:
            at[str(k)] = trail[-1][1]
            todo.pop(0)
    return {"J_at": at, "rank": int(r), "dense": dense, "trail_tail": trail[-3:],
            "znorm": float(np.linalg.norm(z))}


def main():
    which = sys.argv[1:] or ["dr2d_tiny", "dr2d_slice"]
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if "dr2d_tiny" in which:
        rec = {}
        for key, dense in (("dense", True), ("lowrank", False)):
            run = long_run("dr2d_tiny", dense, [300, 3000, 30000, 100000], 1000)
            (k1, J1), (k2, J2), (k3, J3) = run["trail_tail"]
            d1, d2 = J1 - J2, J2 - J3
            rho = d2 / d1
            run["last_block_decrease"] = d2
            run["decrease_ratio"] = rho
            run["J_limit_est"] = J3 - d2 * rho / (1.0 - rho)
            rec[key] = run
        out["dr2d_tiny"] = rec
        json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)
    if "dr2d_slice" in which:
        out["dr2d_slice"] = {"dense": long_run("dr2d_slice", True, [300, 2000], 100)}
        json.dump(out, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
