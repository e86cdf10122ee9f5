"""Voxel-by-voxel nonnegative least squares (Eq. 6 with R = 0), test infrastructure.

At lambda = 0 the spatially regularised problem of Eq. 7 separates into one NNLS
problem per voxel, so its minimiser can be checked voxel by voxel against
  * the Lawson-Hanson active-set method (Sec. II-B), through scipy.optimize.nnls,
    which implements that algorithm, and
  * brute force over every active set on tiny Q: for each subset S of columns, solve
    the unconstrained least-squares problem on S and keep the feasible candidate
    with the smallest residual (the NNLS minimiser is one of these candidates).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.optimize


def nnls_lawson_hanson(K, M):
    """Column-wise NNLS: returns F (Q x N) with F[:, n] = argmin_{f>=0} ||m_n - K f||."""
    K = np.asarray(K, np.float64)
    M = np.asarray(M, np.float64)
    F = np.empty((K.shape[1], M.shape[1]))
    for n in range(M.shape[1]):
        F[:, n], _ = scipy.optimize.nnls(K, M[:, n], maxiter=50 * K.shape[1])
    return F


def nnls_brute_force(K, m):
    """Exact NNLS for one voxel by enumerating active sets (Q <= 12)."""
    K = np.asarray(K, np.float64)
    m = np.asarray(m, np.float64)
    Q = K.shape[1]
    if Q > 12:
        raise ValueError("brute force NNLS is for tiny Q only")
    best = np.zeros(Q)
    best_res = float(m @ m)
    for size in range(1, Q + 1):
        for S in itertools.combinations(range(Q), size):
            KS = K[:, S]
            sol, *_ = np.linalg.lstsq(KS, m, rcond=None)
            if np.all(sol >= -1e-12):
                f = np.zeros(Q)
                f[list(S)] = np.maximum(sol, 0.0)
                res = float(np.sum((m - K @ f) ** 2))
                if res < best_res - 1e-15:
                    best_res = res
                    best = f
    return best
