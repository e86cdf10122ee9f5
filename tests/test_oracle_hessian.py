"""Pins of the oracle's power iteration for the Hessian of Eq. 7 (oracle.pg.hessian_norm).

The Hessian of J(Z) = 1/2 ||M - K Z||^2 + lambda/2 ||D Z||^2 over the Q x N maps is
H = I_N (x) K^T K + lambda D^T D (x) I_Q. Its largest eigenvalue is checked against
  * a dense eigensolve of H built explicitly with np.kron (tiny problems), and
  * the closed form sigma_1^2 + lambda ||D^T D|| (a Kronecker sum's eigenvalues are the
    sums of its factors'; ||D^T D|| is the path-Laplacian closed form pinned in
    test_oracle_grid.py).
"""
import numpy as np
import pytest

from oracle import grid, pg

CASES = [((4, 3), 6, 4, 0.3, 2), ((5,), 3, 7, 1.1, 2), ((3, 2, 2), 8, 5, 0.05, 1),
         ((6, 5), 9, 9, 0.7, 2)]


@pytest.mark.parametrize("dims,P,Q,lam,pairs", CASES)
def test_hessian_norm_matches_dense_eigensolve_and_closed_form(dims, P, Q, lam, pairs):
    rng = np.random.default_rng(P * 31 + Q)
    K = rng.uniform(0.0, 1.0, (P, Q))
    N = int(np.prod(dims))
    H = np.kron(np.eye(N), K.T @ K) + lam * np.kron(grid.dtd(dims, pairs).toarray(), np.eye(Q))
    dense = float(np.linalg.eigvalsh(H)[-1])
    closed = float(np.linalg.svd(K, compute_uv=False)[0] ** 2) + lam * grid.dtd_norm(dims, pairs)
    got = pg.hessian_norm(K, dims, lam, pairs, iters=5000)
    assert dense == pytest.approx(closed, rel=1e-12)
    assert got == pytest.approx(dense, rel=1e-10)
