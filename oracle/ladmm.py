"""Algorithm 2 of the paper (proposed LADMM), FP64, plain numpy (test infrastructure).

Problem (Eq. 7 with the Tikhonov roughness of Eq. 8):

    min_{f >= 0}  1/2 || m - (I_N kron K) f ||^2 + lambda * 1/2 || D f ||^2

Splitting f = z (Eq. 20), with Q = 0 for the f-step and P = xi_p I - lambda D^T D for
the z-step (Sec. III-C, III-D), gives the iteration of Algorithm 2:

    c_n^k     = g_n + beta z_n^k - d_n^k                               (every voxel n)
    f_n^{k+1} = c_n^k / beta - sum_i sigma_i^2/(beta^2 + beta sigma_i^2) v_i (v_i^T c_n^k)
    z^{k+1}   = max(0, (xi_p z^k - lambda D^T D z^k + beta f^{k+1} + d^k) / (xi_p + beta))
    d^{k+1}   = d^k - beta (z^{k+1} - f^{k+1})

with g_n = sum_{i<=r} sigma_i v_i u_i^T m_n from the rank-r truncated SVD of K (Eq. 27),
and f, z, d initialised to 0. The full-rank variant replaces the f-step by Eq. 26,
f_n = (K^T K + beta I)^{-1} (K^T m_n + beta z_n - d_n), with the unapproximated K.

Arrays are map-major: Z, F, Dual, G are Q x N, M is P x N.

Readings where the paper is silent (shared with the CUDA path):
  * "while not converged": a fixed iteration budget plus an optional test every
    `check_every` iterations, stop when ||z^{k+1} - f^{k+1}|| <= tol_primal ||z^{k+1}||
    and ||z^{k+1} - z^k|| <= tol_change ||z^{k+1}|| (a tolerance <= 0 is not used; with
    both unused the budget is spent in full).
  * the returned estimate is z (it satisfies z >= 0); f and d are returned too.
  * D^T D per the literal Eq. 8 (pairs=2), see oracle.grid.
"""
from __future__ import annotations

import numpy as np

from . import grid


def svd_factors(K):
    """Step 3 of Algorithm 2: thin SVD K = sum_i sigma_i u_i v_i^T (sigma descending).

    Returns U (P x s), sigma (s,), V (Q x s) with s = min(P, Q).
    """
    U, s, Vt = np.linalg.svd(np.asarray(K, np.float64), full_matrices=False)
    return U, s, Vt.T


def rank_rule(sigma, tol=5e-5):
    """Sec. III-E: the smallest r whose truncation error is below `tol` (Frobenius).

    By Eckart-Young, ||K - K_r||_F^2 = sum_{i > r} sigma_i^2, and the paper's
    "0.005% approximation error" is read relative to ||K||_F.
    """
    sigma = np.asarray(sigma, np.float64)
    total = float(np.sum(sigma ** 2))
    if total == 0.0:
        return 0
    for r in range(0, sigma.size + 1):
        tail = float(np.sum(sigma[r:] ** 2))
        if np.sqrt(tail / total) < tol:
            return r
    return int(sigma.size)


def lowrank_weights(sigma_r, beta):
    """The scalar weights of Eq. 28: sigma_i^2 / (beta^2 + beta sigma_i^2)."""
    s2 = np.asarray(sigma_r, np.float64) ** 2
    return s2 / (beta * beta + beta * s2)


def dense_inverse(K, beta):
    """Eq. 26: M = (K^T K + beta I_Q)^{-1}, through a Cholesky factorisation."""
    K = np.asarray(K, np.float64)
    A = K.T @ K + beta * np.eye(K.shape[1])
    L = np.linalg.cholesky(A)
    Linv = np.linalg.solve(L, np.eye(K.shape[1]))
    return Linv.T @ Linv


def ladmm(K, M, dims, lam, beta, *, rank=None, dense=False, xi_p=None, iters=300,
          tol_primal=0.0, tol_change=0.0, check_every=10, pairs=2, rank_tol=5e-5,
          return_history=False, mask=None, z0=None, d0=None):
    """Run Algorithm 2 (or its full-rank Eq. 26 variant with dense=True).

    rank: None -> the rank rule of Sec. III-E with `rank_tol`; int -> that r.
    xi_p: None -> Eq. 32, 0.75 lambda ||D^T D|| + 1e-10, with ||D^T D|| of the box grid
    (with a mask this bounds the masked operator's norm from above: removing edges
    from a graph cannot raise its Laplacian's eigenvalues).
    mask: voxels inside the object (True); the problem is posed on them alone, with the
    pairs of the induced grid graph, and z, f, d are 0 outside.
    z0, d0: the state (z^k, d^k) to continue from (Q x N each); None starts from zero as
    Algorithm 2 does. f^{k+1} depends only on z^k and d^k, so continuing from the state
    after k1 iterations for k2 more repeats a run of k1 + k2 iterations exactly.
    Returns a dict with z, f, d (Q x N), iterations run, r, xi_p and the check history.
    """
    if mask is not None:
        inside = np.flatnonzero(np.asarray(mask, bool).ravel())
        if xi_p is None:
            xi_p = grid.xi_p_rule(lam, dims, pairs)
        sub_dtd = grid.dtd(dims, pairs, mask)[inside][:, inside]
        sub = (lambda a: None if a is None else np.asarray(a, np.float64)[:, inside])
        res = _ladmm_core(K, np.asarray(M, np.float64)[:, inside], sub_dtd, lam, beta,
                          rank=rank, dense=dense, xi_p=xi_p, iters=iters,
                          tol_primal=tol_primal, tol_change=tol_change,
                          check_every=check_every, rank_tol=rank_tol, z0=sub(z0), d0=sub(d0))
        for key in ("z", "f", "d"):
            full = np.zeros((res[key].shape[0], int(np.prod(dims))))
            full[:, inside] = res[key]
            res[key] = full
        if not return_history:
            res.pop("history", None)
        return res
    if xi_p is None:
        xi_p = grid.xi_p_rule(lam, dims, pairs)
    K_ = np.asarray(K, np.float64)
    assert np.asarray(M).shape[0] == K_.shape[0] and int(np.prod(dims)) == np.asarray(M).shape[1]
    res = _ladmm_core(K, M, grid.dtd(dims, pairs), lam, beta, rank=rank, dense=dense,
                      xi_p=xi_p, iters=iters, tol_primal=tol_primal, tol_change=tol_change,
                      check_every=check_every, rank_tol=rank_tol, z0=z0, d0=d0)
    if not return_history:
        res.pop("history", None)
    return res


def _ladmm_core(K, M, DtD, lam, beta, *, rank, dense, xi_p, iters, tol_primal, tol_change,
                check_every, rank_tol, z0=None, d0=None):
    """Algorithm 2 on the voxels of M (columns) coupled by the given D^T D."""
    K = np.asarray(K, np.float64)
    M = np.asarray(M, np.float64)
    P, Q = K.shape
    N = M.shape[1]
    assert M.shape[0] == P and DtD.shape == (N, N)

    if dense:
        # Eq. 26 with the unapproximated K: g_n = K^T m_n, M_mat = (K^T K + beta I)^-1
        Minv = dense_inverse(K, beta)
        G = K.T @ M
        r = min(P, Q)
    else:
        U, sigma, V = svd_factors(K)
        r = rank_rule(sigma, rank_tol) if rank is None else int(rank)
        Ur, sr, Vr = U[:, :r], sigma[:r], V[:, :r]
        # step 4: g_n = sum_i sigma_i v_i u_i^T m_n
        G = Vr @ (sr[:, None] * (Ur.T @ M))
        W = lowrank_weights(sr, beta)

    z = np.zeros((Q, N)) if z0 is None else np.array(z0, np.float64)
    d = np.zeros((Q, N)) if d0 is None else np.array(d0, np.float64)
    f = np.zeros((Q, N))
    history = []
    k = 0
    while k < iters:
        # steps 6-8: per-voxel f-step
        c = G + beta * z - d
        if dense:
            f = Minv @ c
        else:
            f = c / beta - Vr @ (W[:, None] * (Vr.T @ c))
        # step 10: z-step (Eq. 31) with the projection onto z >= 0
        z_new = np.maximum(0.0, (xi_p * z - lam * grid.apply_dtd(z, DtD) + beta * f + d)
                           / (xi_p + beta))
        # step 11: dual update
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
    return {"z": z, "f": f, "d": d, "iters": k, "r": r, "xi_p": xi_p, "history": history}


def objective(K, M, Z, dims, lam, pairs=2, mask=None):
    """Eq. 7 with Eq. 8: 1/2 ||M - K Z||_F^2 + lambda * 1/2 ||D Z||^2 (over the voxels
    inside `mask` and the pairs of its induced grid graph when a mask is given)."""
    K = np.asarray(K, np.float64)
    R = np.asarray(M, np.float64) - K @ np.asarray(Z, np.float64)
    if mask is not None:
        R = R[:, np.asarray(mask, bool).ravel()]
    return 0.5 * float(np.sum(R * R)) + lam * grid.roughness(np.asarray(Z, np.float64),
                                                             dims, pairs, mask)


def truncated_dictionary(K, r):
    """K_r of Eq. 27 (the dictionary the low-rank iteration actually fits)."""
    U, s, V = svd_factors(K)
    return (U[:, :r] * s[:r]) @ V[:, :r].T


def residual_norms(z, f, z_prev):
    """The two relative residuals of the stopping rule, in FP64."""
    zn = max(np.linalg.norm(z), 1e-300)
    return np.linalg.norm(z - f) / zn, np.linalg.norm(z - z_prev) / zn
