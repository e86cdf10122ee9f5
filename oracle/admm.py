"""Algorithm 1 of the paper: the previous three-split ADMM, FP64 (test infrastructure).

Splitting f = x = y = z of Eq. 9; per iteration (all variables start at 0):
    f   = (beta x + d_x + beta y + d_y + beta z + d_z) / (3 beta)
    x   = (I kron M)(g + beta f - d_x),   M = (K^T K + beta I)^{-1},  g = (I kron K^T) m
    y   = max(0, f - d_y / beta)
    z   = (lambda D^T D + beta I)^{-1} (beta f - d_z)
    d_x = d_x - beta (f - x);  d_y = d_y - beta (f - y);  d_z = d_z - beta (f - z)
It is a second, structurally different solver of the same problem (Eq. 7). The z-step's
sparse system is solved by a sparse LU factorisation (one per run).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import grid
from .ladmm import dense_inverse


def admm(K, M, dims, lam, beta, iters=1000, pairs=2):
    K = np.asarray(K, np.float64)
    M = np.asarray(M, np.float64)
    Q, N = K.shape[1], M.shape[1]
    Minv = dense_inverse(K, beta)
    g = K.T @ M
    DtD = grid.dtd(dims, pairs)
    solve_z = spla.factorized((lam * DtD + beta * sp.identity(N, format="csr")).tocsc())
    x = np.zeros((Q, N)); y = np.zeros((Q, N)); z = np.zeros((Q, N))
    dx = np.zeros((Q, N)); dy = np.zeros((Q, N)); dz = np.zeros((Q, N))
    f = np.zeros((Q, N))
    for _ in range(iters):
        f = (beta * x + dx + beta * y + dy + beta * z + dz) / (3.0 * beta)
        x = Minv @ (g + beta * f - dx)
        y = np.maximum(0.0, f - dy / beta)
        rhs = beta * f - dz
        z = np.stack([solve_z(rhs[q]) for q in range(Q)])
        dx = dx - beta * (f - x)
        dy = dy - beta * (f - y)
        dz = dz - beta * (f - z)
    return {"f": f, "x": x, "y": y, "z": z}
