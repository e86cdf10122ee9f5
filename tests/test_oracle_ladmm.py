"""Pins for the oracle's Algorithm 2 (and its full-rank Eq. 26 variant).

Nothing here re-types the oracle's own formulas: each check compares against an
independent route to the same mathematical object --
  * Eq. 28 at full rank against a Cholesky inverse (Woodbury identity),
  * lambda = 0 against per-voxel NNLS (Lawson-Hanson and brute-force enumeration),
  * lambda > 0 against an independent FISTA solver and the KKT conditions,
  * Algorithm 1 (three-split ADMM) as a third solver,
  * closed-form special cases: noise-free recovery, a single voxel, a single
    compartment with an interior solution (a plain linear system).
"""
import numpy as np
import pytest
import scipy.optimize

from oracle import admm, grid, kkt, ladmm as L, nnls, pg
from paper_2401_12890_gb300 import synth


def small_problem(P=8, Q=5, dims=(3, 2), seed=0, snr=None, full_rank=True):
    return synth.random_problem(P, Q, dims, seed, snr=snr, full_rank=full_rank)


def test_lowrank_f_step_matches_cholesky_inverse_at_full_rank():
    rng = np.random.default_rng(3)
    for P, Q in [(6, 10), (12, 7), (9, 9)]:
        K = rng.standard_normal((P, Q))
        for beta in (1e-3, 0.7, 25.0):
            U, s, V = L.svd_factors(K)
            W = L.lowrank_weights(s, beta)
            Mlr = np.eye(Q) / beta - (V * W) @ V.T
            Mchol = L.dense_inverse(K, beta)
            np.testing.assert_allclose(Mlr, Mchol, rtol=0, atol=1e-10 * np.abs(Mchol).max())
            # and it really is (K^T K + beta I)^{-1}
            np.testing.assert_allclose(Mchol @ (K.T @ K + beta * np.eye(Q)), np.eye(Q),
                                       atol=1e-9)


def test_svd_factors_reconstruct_and_are_orthonormal():
    K = synth.dictionary_for("dr2d_tiny")
    U, s, V = L.svd_factors(K)
    np.testing.assert_allclose((U * s) @ V.T, K, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-12)
    assert np.all(np.diff(s) <= 0)


def test_rank_rule_on_prescribed_spectrum():
    rng = np.random.default_rng(0)
    s = np.array([10.0, 3.0, 1.0, 1e-2, 1e-4, 1e-6])
    Uq, _ = np.linalg.qr(rng.standard_normal((8, 6)))
    Vq, _ = np.linalg.qr(rng.standard_normal((9, 6)))
    K = (Uq * s) @ Vq.T
    _, sig, _ = L.svd_factors(K)
    tot = np.sqrt(np.sum(s ** 2))
    # tail after r=3 is sqrt(1e-4 + 1e-8 + 1e-12) ~ 1e-2 -> 1e-2/10.49 ~ 9.5e-4
    assert L.rank_rule(sig, 1e-3) == 3
    assert L.rank_rule(sig, 5e-4) == 4
    assert L.rank_rule(sig, 5e-5) == 4      # tail 1e-4/tot ~ 9.5e-6
    assert L.rank_rule(sig, 5e-6) == 5
    assert L.rank_rule(sig, 1e-9) == 6
    assert tot > 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lambda_zero_converges_to_voxelwise_nnls(seed):
    K, M, _ = small_problem(seed=seed, snr=20.0)
    dims = (3, 2)
    out = L.ladmm(K, M, dims, 0.0, beta=2.0, rank=K.shape[1], iters=6000, check_every=0)
    F_lh = nnls.nnls_lawson_hanson(K, M)
    np.testing.assert_allclose(out["z"], F_lh, atol=1e-8)
    for n in range(M.shape[1]):
        np.testing.assert_allclose(out["z"][:, n], nnls.nnls_brute_force(K, M[:, n]),
                                   atol=1e-8)
    # the dense (Eq. 26) variant agrees too
    outd = L.ladmm(K, M, dims, 0.0, beta=2.0, dense=True, iters=6000, check_every=0)
    np.testing.assert_allclose(outd["z"], F_lh, atol=1e-8)


def test_single_voxel_is_nnls_at_any_lambda():
    K, M, _ = small_problem(P=9, Q=6, dims=(1,), seed=5, snr=10.0)
    for lam in (0.0, 0.3, 10.0):           # D^T D = 0 on one voxel
        out = L.ladmm(K, M, (1,), lam, beta=3.0, rank=6, iters=6000, check_every=0)
        np.testing.assert_allclose(out["z"][:, 0],
                                   scipy.optimize.nnls(K, M[:, 0])[0], atol=1e-8)


def test_noise_free_recovery():
    K, M, F = small_problem(P=10, Q=6, dims=(4, 3), seed=7, snr=None)
    out = L.ladmm(K, M, (4, 3), 0.0, beta=2.0, rank=6, iters=8000, check_every=0)
    np.testing.assert_allclose(out["z"], F, atol=1e-8)


def test_single_compartment_interior_solution_is_a_linear_system():
    # Q = 1: (k^T k I + lambda D^T D) z = k^T M when the solution is positive
    dims = (5, 4)
    N = 20
    rng = np.random.default_rng(11)
    k = rng.uniform(0.5, 1.5, (6, 1))
    zt = 2.0 + np.sin(np.arange(N) / 3.0)
    M = k @ zt[None, :] + 0.05 * rng.standard_normal((6, N))
    lam = 0.7
    A = float((k.T @ k)[0, 0]) * np.eye(N) + lam * grid.dtd(dims, 2).toarray()
    z_lin = np.linalg.solve(A, (k.T @ M).ravel())
    assert z_lin.min() > 0
    out = L.ladmm(k, M, dims, lam, beta=float((k.T @ k)[0, 0]), rank=1, iters=3000, check_every=0)
    np.testing.assert_allclose(out["z"].ravel(), z_lin, atol=1e-9)
    # pairs=1 halves the penalty: it must equal pairs=2 with lambda/2
    A1 = float((k.T @ k)[0, 0]) * np.eye(N) + lam * grid.dtd(dims, 1).toarray()
    out1 = L.ladmm(k, M, dims, lam, beta=float((k.T @ k)[0, 0]), rank=1, iters=3000,
                   check_every=0, pairs=1)
    np.testing.assert_allclose(out1["z"].ravel(), np.linalg.solve(A1, (k.T @ M).ravel()),
                               atol=1e-9)


@pytest.mark.parametrize("P,lam,rtol", [(6, 0.05, 1e-9), (12, 1.0, 1e-12), (12, 0.05, 1e-12)])
def test_objective_matches_fista_and_kkt(P, lam, rtol):
    # P = 6 < Q = 9: rank-deficient K (non-unique minimiser, slow tail);
    # P = 12: full column rank (unique minimiser, linear convergence)
    K, M, _ = synth.random_problem(P, 9, (4, 3), seed=21, snr=30.0, full_rank=P >= 9)
    dims = (4, 3)
    out = L.ladmm(K, M, dims, lam, beta=1.0 if P < 9 else 3.0, rank=min(P, 9),
                  iters=20000, check_every=0)
    J_ladmm = L.objective(K, M, out["z"], dims, lam)
    _, J_pg = pg.fista(K, M, dims, lam, iters=400000, tol=1e-17)
    assert J_ladmm == pytest.approx(J_pg, rel=rtol)
    neg, dual, comp = kkt.kkt_residuals(K, M, out["z"], dims, lam)
    assert neg == 0.0 and dual < 1e-9 and comp < 1e-9
    # the LADMM fixed point: z = f and d = g - K^T K f (from the f-step)
    np.testing.assert_allclose(out["z"], out["f"], atol=1e-9)
    np.testing.assert_allclose(out["d"], K.T @ M - K.T @ K @ out["f"], atol=1e-8)
    if P >= 9:     # unique minimiser: the iterates agree too
        Z_pg, _ = pg.fista(K, M, dims, lam, iters=400000, tol=1e-17)
        np.testing.assert_allclose(out["z"], Z_pg, atol=1e-7)


def test_algorithm1_admm_reaches_same_objective():
    K, M, _ = synth.random_problem(6, 8, (3, 3), seed=4, snr=30.0)
    dims, lam = (3, 3), 0.2
    out = L.ladmm(K, M, dims, lam, beta=1.0, rank=6, iters=20000, check_every=0)
    res = admm.admm(K, M, dims, lam, beta=1.0, iters=20000)
    J_l = L.objective(K, M, out["z"], dims, lam)
    J_a = L.objective(K, M, res["y"], dims, lam)
    assert J_a == pytest.approx(J_l, rel=1e-7)


def test_dense_and_lowrank_full_rank_give_same_iterates():
    K = synth.dictionary_for("dr2d_tiny")[:, ::9]      # 30 x 25, full column rank
    _, M, _ = synth.make_problem("dr2d_tiny", dims=(6, 5))
    M = M.astype(np.float64)
    for beta in (0.03, 3.0):
        a = L.ladmm(K, M, (6, 5), 1e-2, beta, rank=K.shape[1], iters=50, check_every=0)
        b = L.ladmm(K, M, (6, 5), 1e-2, beta, dense=True, iters=50, check_every=0)
        np.testing.assert_allclose(a["z"], b["z"], rtol=0, atol=1e-8 * np.abs(b["z"]).max())


def test_zero_iterations_and_zero_data():
    K, M, _ = small_problem()
    out = L.ladmm(K, M, (3, 2), 0.1, 1.0, iters=0)
    assert out["iters"] == 0 and not out["z"].any()
    out = L.ladmm(K, np.zeros_like(M), (3, 2), 0.1, 1.0, iters=20)
    assert not out["z"].any() and not out["d"].any()


def test_stopping_rule_stops_on_check_boundary():
    K, M, _ = small_problem(seed=3, snr=10.0)
    out = L.ladmm(K, M, (3, 2), 0.1, 1.0, iters=1000, check_every=7, tol_primal=1e-3,
                  tol_change=1e-3, return_history=True)
    assert out["iters"] % 7 == 0 and out["iters"] < 1000
    k, rp, rc = out["history"][-1]
    assert rp <= 1e-3 and rc <= 1e-3
    # every earlier check failed the test
    assert all(max(a, b) > 1e-3 for _, a, b in out["history"][:-1])
    # with no tolerance the budget is spent
    out = L.ladmm(K, M, (3, 2), 0.1, 1.0, iters=33, check_every=7)
    assert out["iters"] == 33


@pytest.mark.parametrize("dense", [False, True])
def test_continuing_from_a_state_repeats_the_longer_run(dense):
    """Algorithm 2's state is (z, d): k1 iterations, then k2 more from (z, d), are the
    k1 + k2 iterations of one run, bit for bit."""
    K, M, _ = synth.random_problem(9, 14, (6, 5), seed=4, snr=30.0)
    kw = dict(rank=5, dense=dense, check_every=0)
    full = L.ladmm(K, M, (6, 5), 0.2, 0.7, iters=25, **kw)
    first = L.ladmm(K, M, (6, 5), 0.2, 0.7, iters=10, **kw)
    rest = L.ladmm(K, M, (6, 5), 0.2, 0.7, iters=15, z0=first["z"], d0=first["d"], **kw)
    assert np.array_equal(rest["z"], full["z"]) and np.array_equal(rest["d"], full["d"])
