"""The spatial finite-difference operator D of Eq. 8 (oracle; test infrastructure).

Eq. 8 defines the roughness penalty as a sum over every voxel n and every voxel m
adjacent to n of 1/2 ||f_n - f_m||^2, and names that 1/2 ||D f||^2. Read literally,
each unordered neighbour pair is visited twice (once from each end), so D has one row
per ORDERED adjacent pair and D^T D = 2 L with L the grid-graph Laplacian. The
alternative reading (one row per unordered edge, D^T D = L) is `pairs=1`.

Adjacency is axis-aligned: 2 neighbours per axis, so 4 in 2D and 6 in 3D. The image
boundary is free: voxels on the edge have fewer neighbours, there is no wrap-around
and no ghost voxel (the paper's maskless form, footnote to Algorithm 1).

Voxel index n = x + nx*(y + ny*z).

Masks: the paper's maskless form estimates only the voxels inside the object and
imposes no smoothness across the object boundary (footnote to Algorithm 1). With a
voxel mask (True = inside), the adjacent pairs are those with both voxels inside, i.e.
the grid graph induced by the mask; voxels outside belong to no pair.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def neighbor_pairs(dims, mask=None):
    """All ordered pairs (n, m) with m adjacent to n (both inside `mask` when given),
    as two int64 arrays."""
    dims = tuple(int(d) for d in dims)
    N = int(np.prod(dims))
    idx = np.arange(N).reshape(tuple(reversed(dims)))  # [z][y][x] (x fastest)
    src, dst = [], []
    nd = len(dims)
    for ax in range(nd):
        arr_ax = nd - 1 - ax          # axis 0 (x) is the last array axis
        if dims[ax] < 2:
            continue
        a = np.take(idx, np.arange(dims[ax] - 1), axis=arr_ax).ravel()
        b = np.take(idx, np.arange(1, dims[ax]), axis=arr_ax).ravel()
        src += [a, b]
        dst += [b, a]
    if not src:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    n, m = np.concatenate(src), np.concatenate(dst)
    if mask is not None:
        inside = np.asarray(mask, bool).ravel()
        keep = inside[n] & inside[m]
        n, m = n[keep], m[keep]
    return n, m


def difference_operator(dims, pairs=2, mask=None):
    """Sparse D (rows = adjacent pairs, cols = N voxels) with (D f)_row = f_n - f_m.

    pairs=2: one row per ordered pair (literal Eq. 8). pairs=1: one row per edge.
    """
    n, m = neighbor_pairs(dims, mask)
    if pairs == 1:
        keep = n < m
        n, m = n[keep], m[keep]
    elif pairs != 2:
        raise ValueError("pairs must be 1 or 2")
    N = int(np.prod(dims))
    rows = np.arange(n.size)
    data = np.concatenate([np.ones(n.size), -np.ones(n.size)])
    D = sp.csr_matrix((data, (np.concatenate([rows, rows]), np.concatenate([n, m]))),
                      shape=(n.size, N))
    return D


def dtd(dims, pairs=2, mask=None):
    """D^T D as a sparse N x N matrix (symmetric)."""
    D = difference_operator(dims, pairs, mask)
    return (D.T @ D).tocsr()


def apply_dtd(Z, DtD):
    """(D^T D) applied to every compartment map: Z is Q x N (map-major)."""
    return (DtD @ Z.T).T


def roughness(Z, dims, pairs=2, mask=None):
    """R(Z) = 1/2 ||D Z||^2 summed over all Q maps (Eq. 8)."""
    D = difference_operator(dims, pairs, mask)
    DZ = D @ Z.T
    return 0.5 * float(np.sum(DZ * DZ))


def dtd_norm(dims, pairs=2):
    """Spectral norm ||D^T D|| on a free-boundary box grid.

    D^T D = s * L with s = 2 (pairs=2) or 1 (pairs=1). L is the Cartesian product of
    path-graph Laplacians, whose eigenvalues are 2 - 2 cos(pi k / n_d), k = 0..n_d-1,
    and the product's eigenvalues are sums over axes, so the largest is
    s * sum_d (2 - 2 cos(pi (n_d - 1) / n_d)).
    """
    s = 2.0 if pairs == 2 else 1.0
    tot = 0.0
    for nd in dims:
        nd = int(nd)
        if nd >= 2:
            tot += 2.0 - 2.0 * np.cos(np.pi * (nd - 1) / nd)
    return s * tot


def xi_p_rule(lam, dims, pairs=2, eps=1e-10):
    """Eq. 32: xi_p = 0.75 * lambda * ||D^T D|| + eps (eps = 1e-10 in the paper)."""
    return 0.75 * lam * dtd_norm(dims, pairs) + eps
