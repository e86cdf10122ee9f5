"""Write tests/golden/workloads.json from the FP64 oracle only.

For each benchmark workload (paper_2401_12890_gb300.synth.WORKLOADS) it records:
  beta      -- the paper's heuristic (Sec. III-E): tuned once on the centre 3x3 (x3)
               patch, lowest objective after 300 iterations (oracle.tune)
  rank      -- the rank rule of Sec. III-E (||K - K_r||_F < 5e-5 ||K||_F)
  sigma1    -- largest singular value of K
  dtd_norm  -- ||D^T D|| of the grid (literal Eq. 8), xi_p -- Eq. 32
and, for the small 32x32 workload, the oracle's objective after 300 iterations of
Algorithm 2 (and of the full-rank Eq. 26 variant) with those parameters. For the
spatially varying dictionary workload (synth.B1_WORKLOAD, one dictionary per B1 level)
the heuristic runs on the centre 3x3 patch with the centre voxel's dictionary, and the
record holds each dictionary's rank.

Run:  python tests/golden/make_golden.py [workload ...]   (default: all)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import grid, ladmm as L, tune  # noqa: E402
from paper_2401_12890_gb300 import synth  # noqa: E402


def b1_record():
    w = synth.B1_WORKLOAD
    Ks, labels, M, _ = synth.make_b1_problem()
    centre = (w.dims[1] // 2) * w.dims[0] + w.dims[0] // 2
    c = int(labels[centre])
    beta, table = tune.tune_beta(Ks[c], M.astype(np.float64), w.dims, w.lam)
    ranks = [L.rank_rule(L.svd_factors(K)[1]) for K in Ks]
    return {
        "dims": list(w.dims), "P": w.P, "Q": w.Q, "lambda": w.lam, "levels": len(Ks),
        "beta": beta, "centre_label": c, "ranks": ranks,
        "sigma1": max(float(L.svd_factors(K)[1][0]) for K in Ks),
        "dtd_norm": grid.dtd_norm(w.dims, 2), "xi_p": grid.xi_p_rule(w.lam, w.dims, 2),
        "beta_table": {f"{b:.6g}": v for b, v in table.items()},
    }


def main():
    path = os.path.join(HERE, "workloads.json")
    which = sys.argv[1:] or list(synth.WORKLOADS) + [synth.B1_WORKLOAD.name]
    out = json.load(open(path)) if os.path.exists(path) else {}
    if synth.B1_WORKLOAD.name in which:
        out[synth.B1_WORKLOAD.name] = b1_record()
        print(synth.B1_WORKLOAD.name, out[synth.B1_WORKLOAD.name]["beta"], flush=True)
    for name, w in synth.WORKLOADS.items():
        if name not in which:
            continue
        K = synth.dictionary_for(name)
        _, M, _ = synth.make_problem(name)
        beta, table = tune.tune_beta(K, M.astype(np.float64), w.dims, w.lam)
        _, s, _ = L.svd_factors(K)
        rec = {
            "dims": list(w.dims), "P": w.P, "Q": w.Q, "lambda": w.lam,
            "beta": beta, "rank": L.rank_rule(s), "sigma1": float(s[0]),
            "dtd_norm": grid.dtd_norm(w.dims, 2), "xi_p": grid.xi_p_rule(w.lam, w.dims, 2),
            "beta_table": {f"{b:.6g}": v for b, v in table.items()},
        }
        if name == "dr2d_tiny":
            M64 = M.astype(np.float64)
            for key, dense in (("lowrank", False), ("dense", True)):
                res = L.ladmm(K, M64, w.dims, w.lam, beta, dense=dense, iters=300,
                              check_every=0)
                Kf = K if dense else L.truncated_dictionary(K, res["r"])
                rec[f"J300_{key}"] = L.objective(Kf, M64, res["z"], w.dims, w.lam)
                rec[f"znorm300_{key}"] = float(np.linalg.norm(res["z"]))
        out[name] = rec
        print(name, {k: v for k, v in rec.items() if k != "beta_table"}, flush=True)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
