"""Algorithm 2 with a spatially varying dictionary, FP64, plain numpy (test infrastructure).

The paper's fingerprinting experiment (Sec. IV-D) models each voxel with the dictionary of
its own B1 level (a few dozen quantised levels). Each voxel n then has a label c(n) and
the problem of Eq. 7 becomes

    min_{F >= 0}  sum_n 1/2 || m_n - K_{c(n)} f_n ||^2 + lambda/2 || D F ||^2 .

The splitting of Algorithm 2 is unchanged: the f-step is per voxel, so it takes the
voxel's own factors, and the z-step and the dual step do not involve K at all:

    g_n       = sum_{i<=r_c} sigma_{c,i} v_{c,i} u_{c,i}^T m_n          (Eq. 27, c = c(n))
    c_n       = g_n + beta z_n - d_n
    f_n       = c_n/beta - sum_i W_{c,i} v_{c,i} (v_{c,i}^T c_n)          (Eq. 28)
    z'        = max(0, (xi_p z - lambda D^T D z + beta f + d) / (xi_p + beta))   (Eq. 31)
    d'        = d - beta (z' - f)

with W_{c,i} = sigma_{c,i}^2 / (beta^2 + beta sigma_{c,i}^2), each dictionary's rank r_c
chosen by the rank rule of Sec. III-E (or fixed), and xi_p from Eq. 32 (it depends on D
alone). The full-rank variant uses f_n = (K_c^T K_c + beta I)^{-1} c_n (Eq. 26) with
g_n = K_c^T m_n. All dictionaries share P and Q.

Independent routes for the pins: `fista_multi` (projected gradient on the same
objective) and per-voxel NNLS at lambda = 0 (scipy).
"""
from __future__ import annotations

import numpy as np

from . import grid
from .ladmm import dense_inverse, lowrank_weights, rank_rule, svd_factors


def _check(Ks, labels, M, dims):
    Ks = [np.asarray(K, np.float64) for K in Ks]
    P, Q = Ks[0].shape
    assert all(K.shape == (P, Q) for K in Ks), "dictionaries must share P and Q"
    labels = np.asarray(labels).ravel().astype(np.int64)
    N = int(np.prod(dims))
    assert labels.shape == (N,) and labels.min() >= 0 and labels.max() < len(Ks)
    M = np.asarray(M, np.float64)
    assert M.shape == (P, N)
    return Ks, labels, M, P, Q, N


def objective_multi(Ks, labels, M, Z, dims, lam, pairs=2):
    """The objective above for a Q x N map Z."""
    Ks, labels, M, P, Q, N = _check(Ks, labels, M, dims)
    Z = np.asarray(Z, np.float64)
    fit = 0.0
    for c, K in enumerate(Ks):
        sel = labels == c
        if sel.any():
            R = M[:, sel] - K @ Z[:, sel]
            fit += 0.5 * float(np.sum(R * R))
    return fit + lam * grid.roughness(Z, dims, pairs)


def ladmm_multi(Ks, labels, M, dims, lam, beta, *, rank=None, dense=False, xi_p=None,
                iters=300, tol_primal=0.0, tol_change=0.0, check_every=10, pairs=2,
                rank_tol=5e-5):
    """Algorithm 2 with the voxel's own dictionary in the f-step (dense=True: Eq. 26).

    rank: None -> the rank rule per dictionary; int -> that r for every dictionary.
    Stopping rule and returned values as `oracle.ladmm.ladmm`.
    """
    Ks, labels, M, P, Q, N = _check(Ks, labels, M, dims)
    if xi_p is None:
        xi_p = grid.xi_p_rule(lam, dims, pairs)
    DtD = grid.dtd(dims, pairs)
    groups = [np.flatnonzero(labels == c) for c in range(len(Ks))]

    # steps 1-4 per dictionary: factors, weights (or the Eq. 26 inverse), and g
    G = np.zeros((Q, N))
    fstep = []
    ranks = []
    for K, idx in zip(Ks, groups):
        if dense:
            Minv = dense_inverse(K, beta)
            fstep.append(("dense", Minv))
            ranks.append(min(P, Q))
            if idx.size:
                G[:, idx] = K.T @ M[:, idx]
        else:
            U, sigma, V = svd_factors(K)
            r = rank_rule(sigma, rank_tol) if rank is None else int(rank)
            Ur, sr, Vr = U[:, :r], sigma[:r], V[:, :r]
            fstep.append(("lowrank", Vr, lowrank_weights(sr, beta)))
            ranks.append(r)
            if idx.size:
                G[:, idx] = Vr @ (sr[:, None] * (Ur.T @ M[:, idx]))

    z = np.zeros((Q, N))
    d = np.zeros((Q, N))
    f = np.zeros((Q, N))
    history = []
    k = 0
    while k < iters:
        c_all = G + beta * z - d
        # steps 6-8: each voxel's f-step with its dictionary's factors
        for step, idx in zip(fstep, groups):
            if not idx.size:
                continue
            c = c_all[:, idx]
            if step[0] == "dense":
                f[:, idx] = step[1] @ c
            else:
                _, Vr, W = step
                f[:, idx] = c / beta - Vr @ (W[:, None] * (Vr.T @ c))
        # step 10: the z-step (Eq. 31)
        z_new = np.maximum(0.0, (xi_p * z - lam * grid.apply_dtd(z, DtD) + beta * f + d)
                           / (xi_p + beta))
        # step 11: the dual step
        d = d - beta * (z_new - f)
        z_old = z
        z = z_new
        k += 1
        if check_every > 0 and k % check_every == 0:
            zn = max(np.linalg.norm(z), 1e-300)
            rp = np.linalg.norm(z - f) / zn
            rc = np.linalg.norm(z - z_old) / zn
            history.append((k, rp, rc))
            used = [(t, v) for t, v in ((tol_primal, rp), (tol_change, rc)) if t > 0]
            if used and all(v <= t for t, v in used):
                break
    return {"z": z, "f": f, "d": d, "iters": k, "ranks": ranks, "xi_p": xi_p,
            "history": history}


def fista_multi(Ks, labels, M, dims, lam, iters=20000, pairs=2, tol=1e-15):
    """Projected FISTA with adaptive restart on the objective above; returns (Z, J).

    The gradient is K_c^T (K_c f_n - m_n) per voxel plus lambda Z D^T D; the step is
    1/L with L = max_c ||K_c||_2^2 + lambda ||D^T D|| (an upper bound of the Hessian's
    norm). Shares nothing with `ladmm_multi` but the objective's definition.
    """
    Ks, labels, M, P, Q, N = _check(Ks, labels, M, dims)
    DtD = grid.dtd(dims, pairs)
    L = max(float(np.linalg.norm(K, 2)) ** 2 for K in Ks) + lam * grid.dtd_norm(dims, pairs)
    groups = [np.flatnonzero(labels == c) for c in range(len(Ks))]
    KtK = [K.T @ K for K in Ks]
    KtM = np.zeros((Q, N))
    for K, idx in zip(Ks, groups):
        if idx.size:
            KtM[:, idx] = K.T @ M[:, idx]

    def grad(Z):
        g = lam * grid.apply_dtd(Z, DtD) - KtM
        for A, idx in zip(KtK, groups):
            if idx.size:
                g[:, idx] += A @ Z[:, idx]
        return g

    def J(Z):
        return objective_multi(Ks, labels, M, Z, dims, lam, pairs)

    Z = np.zeros((Q, N))
    Y = Z.copy()
    t = 1.0
    j_old = J(Z)
    for _ in range(iters):
        Z_new = np.maximum(0.0, Y - grad(Y) / L)
        j_new = J(Z_new)
        if j_new > j_old:               # adaptive restart: drop the momentum
            t = 1.0
            Y = Z.copy()
            continue
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        Y = Z_new + ((t - 1.0) / t_new) * (Z_new - Z)
        converged = j_old - j_new <= tol * max(abs(j_new), 1e-300)
        Z, t, j_old = Z_new, t_new, j_new
        if converged:
            break
    return Z, j_old
