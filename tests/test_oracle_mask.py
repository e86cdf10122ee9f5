"""Pins of the oracle's voxel masks (no GPU).

With a mask the problem lives on the voxels inside the object, coupled only through
the pairs of the grid graph they induce (no smoothing across the object boundary, the
paper's maskless form). Pins that do not use the mask code's own construction:
  - an all-inside mask is the unmasked problem;
  - two disconnected blocks of voxels are two independent problems: solving the masked
    grid equals solving each block as its own box grid (with the same xi_p) and
    placing the results, in 2D and 3D;
  - data outside the mask does not matter, and z is 0 there;
  - the masked objective is the sum of the blocks' objectives.
A planted mistake that keeps the pairs crossing the boundary fails the block pin.
"""
import os

import numpy as np

from oracle import grid, ladmm as L
from paper_2401_12890_gb300 import synth

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle")


def blocks_2d():
    """A 12 x 9 grid with two rectangles inside (x 1..4 and x 7..10, y 2..6)."""
    dims = (12, 9)
    mask = np.zeros((9, 12), bool)             # [y][x]
    mask[2:7, 1:5] = True
    mask[2:7, 7:11] = True
    parts = [((4, 5), (slice(2, 7), slice(1, 5))), ((4, 5), (slice(2, 7), slice(7, 11)))]
    return dims, mask.ravel(), parts


def blocks_3d():
    dims = (6, 5, 4)
    mask = np.zeros((4, 5, 6), bool)           # [z][y][x]
    mask[0:2, 1:4, 0:6] = True                 # z 0..1
    mask[3:4, 0:5, 1:5] = True                 # z 3 (z = 2 empty: no contact)
    parts = [((6, 3, 2), (slice(0, 2), slice(1, 4), slice(0, 6))),
             ((4, 5, 1), (slice(3, 4), slice(0, 5), slice(1, 5)))]
    return dims, mask.ravel(), parts


def solve_by_blocks(K, M, dims, lam, beta, xi, parts, ladmm=L.ladmm, **kw):
    Q = K.shape[1]
    full = np.zeros((Q,) + tuple(reversed(dims)))
    Mg = M.reshape((M.shape[0],) + tuple(reversed(dims)))
    for pdims, sl in parts:
        Mb = Mg[(slice(None),) + sl].reshape(M.shape[0], -1)
        res = ladmm(K, Mb, pdims, lam, beta, xi_p=xi, **kw)
        full[(slice(None),) + sl] = res["z"].reshape((Q,) + Mg[(0,) + sl].shape)
    return full.reshape(Q, -1)


def test_all_inside_mask_is_the_unmasked_problem():
    K, M, _ = synth.random_problem(10, 12, (7, 5), seed=3, snr=40.0)
    a = L.ladmm(K, M, (7, 5), 0.1, 1.0, iters=60, check_every=0)
    b = L.ladmm(K, M, (7, 5), 0.1, 1.0, iters=60, check_every=0, mask=np.ones(35, bool))
    np.testing.assert_allclose(b["z"], a["z"], rtol=0, atol=1e-13)


def test_disconnected_blocks_are_independent_problems():
    for make, seed in ((blocks_2d, 5), (blocks_3d, 6)):
        dims, mask, parts = make()
        K, M, _ = synth.random_problem(9, 14, dims, seed=seed, snr=40.0)
        xi = grid.xi_p_rule(0.2, dims)
        for dense in (False, True):
            kw = dict(iters=80, check_every=0, dense=dense)
            z = L.ladmm(K, M, dims, 0.2, 1.5, mask=mask, **kw)["z"]
            ref = solve_by_blocks(K, M, dims, 0.2, 1.5, xi, parts, **kw)
            np.testing.assert_allclose(z, ref, rtol=0, atol=1e-12)


def test_outside_data_is_ignored_and_z_is_zero_there():
    dims, mask, _ = blocks_2d()
    K, M, _ = synth.random_problem(9, 14, dims, seed=7, snr=40.0)
    M2 = M.copy()
    M2[:, ~mask] = np.random.default_rng(1).normal(size=(M.shape[0], int((~mask).sum())))
    a = L.ladmm(K, M, dims, 0.2, 1.5, iters=50, check_every=0, mask=mask)["z"]
    b = L.ladmm(K, M2, dims, 0.2, 1.5, iters=50, check_every=0, mask=mask)["z"]
    np.testing.assert_array_equal(a, b)
    assert np.all(a[:, ~mask] == 0.0)


def test_masked_objective_is_the_sum_over_blocks():
    dims, mask, parts = blocks_2d()
    K, M, _ = synth.random_problem(9, 14, dims, seed=8, snr=40.0)
    Z = np.abs(np.random.default_rng(2).normal(size=(14, int(np.prod(dims)))))
    Z[:, ~mask] = 0.0
    J = L.objective(K, M, Z, dims, 0.3, mask=mask)
    Zg = Z.reshape((14,) + tuple(reversed(dims)))
    Mg = M.reshape((M.shape[0],) + tuple(reversed(dims)))
    Jb = 0.0
    for pdims, sl in parts:
        Jb += L.objective(K, Mg[(slice(None),) + sl].reshape(M.shape[0], -1),
                          Zg[(slice(None),) + sl].reshape(14, -1), pdims, 0.3)
    assert abs(J - Jb) <= 1e-12 * abs(Jb)


def test_planted_boundary_coupling_is_caught():
    """A mask that keeps every pair touching an inside voxel (instead of both ends
    inside) couples the blocks to the zero voxels around them."""
    import types
    src = open(os.path.join(ORACLE_DIR, "grid.py")).read()
    old = "keep = inside[n] & inside[m]"
    assert old in src
    mut = types.ModuleType("grid_mut")
    exec(compile(src.replace(old, "keep = inside[n] | inside[m]"), "<mutant>", "exec"),
         mut.__dict__)
    dims, mask, parts = blocks_2d()
    K, M, _ = synth.random_problem(9, 14, dims, seed=5, snr=40.0)
    xi = grid.xi_p_rule(0.2, dims)
    inside = np.flatnonzero(mask)
    sub = mut.dtd(dims, 2, mask)[inside][:, inside]
    res = L._ladmm_core(K, M[:, inside], sub, 0.2, 1.5, rank=None, dense=False, xi_p=xi,
                        iters=80, tol_primal=0.0, tol_change=0.0, check_every=0,
                        rank_tol=5e-5)
    z = np.zeros((14, int(np.prod(dims))))
    z[:, inside] = res["z"]
    ref = solve_by_blocks(K, M, dims, 0.2, 1.5, xi, parts, iters=80, check_every=0)
    assert np.abs(z - ref).max() > 1e-6
