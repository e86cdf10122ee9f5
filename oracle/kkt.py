"""First-order optimality (KKT) residuals of Eq. 7 under Z >= 0, FP64.

For the convex problem min_{Z>=0} J(Z) the point Z is optimal iff
  Z >= 0,   grad J(Z) >= 0,   Z * grad J(Z) = 0   (elementwise),
with grad J(Z) = K^T K Z - K^T M + lambda Z D^T D. Residuals are scaled by
||K^T M||_inf so they are comparable across problems.
"""
from __future__ import annotations

import numpy as np

from . import grid


def gradient(K, M, Z, dims, lam, pairs=2):
    K = np.asarray(K, np.float64)
    Z = np.asarray(Z, np.float64)
    DtD = grid.dtd(dims, pairs)
    return K.T @ (K @ Z) - K.T @ np.asarray(M, np.float64) + lam * grid.apply_dtd(Z, DtD)


def kkt_residuals(K, M, Z, dims, lam, pairs=2):
    """(negativity, dual infeasibility, complementarity), each relative to ||K^T M||_inf."""
    Z = np.asarray(Z, np.float64)
    g = gradient(K, M, Z, dims, lam, pairs)
    scale = max(float(np.max(np.abs(np.asarray(K, np.float64).T @ np.asarray(M, np.float64)))), 1e-300)
    neg = float(max(0.0, -Z.min())) / scale
    dual = float(max(0.0, -g.min())) / scale
    comp = float(np.max(np.abs(Z * g))) / (scale * max(float(Z.max()), 1e-300))
    return neg, dual, comp
