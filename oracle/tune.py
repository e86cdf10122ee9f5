"""The paper's beta heuristic (Sec. III-E), FP64 (test infrastructure).

beta is tuned once on a small image patch (3 x 3 voxels, 3 x 3 x 3 in 3D) for the
fastest convergence and then reused on the full image. "Fastest" is read here as the
lowest objective J(z^k) (Eq. 7, with the dictionary the iteration uses) after a fixed
budget of k iterations from the zero start. Candidates are sigma_1^2 times a
log-spaced grid; sigma_1 is the largest singular value of K.
"""
from __future__ import annotations

import numpy as np

from . import ladmm as L


def centre_patch(M, dims, size=3):
    """Columns of M for the centre patch (size per axis) and the patch's dims."""
    dims = tuple(int(d) for d in dims)
    starts = [max(0, d // 2 - size // 2) for d in dims]
    sizes = [min(size, d) for d in dims]
    cols = []
    for n in np.ndindex(*reversed(sizes)):          # n = (z, y, x) or (y, x)
        coord = list(reversed(n))                    # (x, y[, z]) within the patch
        flat, stride = 0, 1
        for ax in range(len(dims)):
            flat += (starts[ax] + coord[ax]) * stride
            stride *= dims[ax]
        cols.append(flat)
    return np.asarray(M)[:, cols], tuple(sizes)


def tune_beta(K, M, dims, lam, iters=300, grid_lo=-6.0, grid_hi=1.0, n_grid=15,
              rank=None):
    """Returns (best beta, {beta: J(z^iters)}) on the centre patch."""
    Mp, pdims = centre_patch(M, dims)
    _, s, _ = L.svd_factors(K)
    r = L.rank_rule(s) if rank is None else int(rank)
    Kr = L.truncated_dictionary(K, r)
    table = {}
    for b in s[0] ** 2 * np.logspace(grid_lo, grid_hi, n_grid):
        res = L.ladmm(K, Mp, pdims, lam, float(b), rank=r, iters=iters, check_every=0)
        table[float(b)] = L.objective(Kr, Mp, res["z"], pdims, lam)
    best = min(table, key=lambda b: (table[b], b))
    return best, table
