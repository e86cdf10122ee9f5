"""An independent solver of Eq. 7: accelerated projected gradient (FISTA), FP64.

    J(Z) = 1/2 ||M - K Z||_F^2 + lambda/2 ||D Z||^2,   Z >= 0
    grad J(Z) = K^T K Z - K^T M + lambda Z (D^T D)

The step is 1/L with L the largest eigenvalue of the Hessian Z -> K^T K Z +
lambda Z D^T D, found by power iteration. Momentum restarts when the objective rises
(adaptive restart), which keeps FISTA monotone on these ill-conditioned problems.
Test infrastructure: it shares nothing with LADMM except the problem definition.
"""
from __future__ import annotations

import numpy as np

from . import grid


def hessian_norm(K, dims, lam, pairs=2, iters=500, seed=0):
    """Power iteration for lambda_max of Z -> K^T K Z + lambda Z D^T D."""
    K = np.asarray(K, np.float64)
    KtK = K.T @ K
    DtD = grid.dtd(dims, pairs)
    N = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((K.shape[1], N))
    X /= np.linalg.norm(X)
    lam_max = 0.0
    for _ in range(iters):
        Y = KtK @ X + lam * grid.apply_dtd(X, DtD)
        lam_new = float(np.sum(X * Y))
        X = Y / np.linalg.norm(Y)
        if abs(lam_new - lam_max) <= 1e-13 * abs(lam_new):
            lam_max = lam_new
            break
        lam_max = lam_new
    return lam_max


def fista(K, M, dims, lam, iters=20000, pairs=2, tol=1e-15, Z0=None):
    """Projected FISTA with adaptive restart; returns (Z, objective)."""
    K = np.asarray(K, np.float64)
    M = np.asarray(M, np.float64)
    KtK = K.T @ K
    KtM = K.T @ M
    DtD = grid.dtd(dims, pairs)
    L = hessian_norm(K, dims, lam, pairs) * 1.01
    Q, N = K.shape[1], M.shape[1]

    def J(Z):
        R = M - K @ Z
        return 0.5 * float(np.sum(R * R)) + lam * 0.5 * float(np.sum(Z * grid.apply_dtd(Z, DtD)))

    Z = np.zeros((Q, N)) if Z0 is None else np.array(Z0, np.float64)
    Y = Z.copy()
    t = 1.0
    J_old = J(Z)
    for _ in range(iters):
        grad = KtK @ Y - KtM + lam * grid.apply_dtd(Y, DtD)
        Z_new = np.maximum(0.0, Y - grad / L)
        J_new = J(Z_new)
        if J_new > J_old:           # restart momentum
            t = 1.0
            Y = Z.copy()
            continue
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        Y = Z_new + ((t - 1.0) / t_new) * (Z_new - Z)
        done = abs(J_old - J_new) <= tol * max(abs(J_new), 1e-300)
        Z, t, J_old = Z_new, t_new, J_new
        if done:
            break
    return Z, J_old
