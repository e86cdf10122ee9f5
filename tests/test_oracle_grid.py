"""Pins for the oracle's finite-difference operator (Eq. 8) and xi_p (Eq. 32).

The spectrum of D^T D on a free-boundary box grid is known in closed form: the
path-graph Laplacian on n points has eigenvalues 2 - 2 cos(pi k / n), k = 0..n-1,
and the grid Laplacian's eigenvalues are all sums of one per axis. With the literal
reading of Eq. 8 (each neighbour pair visited from both ends), D^T D = 2 L.
"""
import itertools

import numpy as np
import pytest

from oracle import grid


def closed_form_spectrum(dims, s):
    per_axis = [2.0 - 2.0 * np.cos(np.pi * np.arange(n) / n) for n in dims]
    vals = [sum(c) for c in itertools.product(*per_axis)]
    return s * np.sort(np.array(vals))


@pytest.mark.parametrize("dims", [(7,), (5, 4), (3, 4, 2), (1, 6), (2, 2, 2), (6, 1, 3)])
@pytest.mark.parametrize("pairs", [1, 2])
def test_dtd_spectrum_matches_closed_form(dims, pairs):
    A = grid.dtd(dims, pairs).toarray()
    ev = np.sort(np.linalg.eigvalsh(A))
    np.testing.assert_allclose(ev, closed_form_spectrum(dims, 2.0 if pairs == 2 else 1.0),
                               atol=1e-12)


@pytest.mark.parametrize("dims", [(7,), (5, 4), (3, 4, 2), (8, 8), (1, 1), (9, 2, 3)])
def test_dtd_norm_closed_form_vs_eigensolve(dims):
    for pairs in (1, 2):
        A = grid.dtd(dims, pairs).toarray()
        lam_max = np.linalg.eigvalsh(A).max() if A.size else 0.0
        assert grid.dtd_norm(dims, pairs) == pytest.approx(lam_max, abs=1e-12)


def test_dtd_norm_large_grids_power_iteration():
    # power iteration on a 2D and a 3D grid of the benchmark shapes' kind
    for dims in [(32, 32), (12, 10, 6)]:
        A = grid.dtd(dims, 2)
        x = np.random.default_rng(1).standard_normal(A.shape[0])
        lam = 0.0
        for _ in range(20000):
            y = A @ x
            lam = float(x @ y) / float(x @ x)
            x = y / np.linalg.norm(y)
        assert lam == pytest.approx(grid.dtd_norm(dims, 2), rel=1e-4)


def test_dtd_structure():
    dims = (6, 5, 3)
    A = grid.dtd(dims, 2)
    N = 6 * 5 * 3
    assert abs(A - A.T).max() == 0
    np.testing.assert_allclose(A @ np.ones(N), 0.0, atol=1e-13)
    # diagonal = 2 * degree; interior voxel has 6 neighbours
    deg = np.asarray(A.diagonal()) / 2.0
    n_interior = 2 + 6 * (2 + 5 * 1)
    assert deg[n_interior] == 6
    assert deg[0] == 3                     # corner
    # number of ordered pairs = 2 * edges
    edges = (6 - 1) * 5 * 3 + 6 * (5 - 1) * 3 + 6 * 5 * (3 - 1)
    assert grid.difference_operator(dims, 2).shape[0] == 2 * edges
    assert grid.difference_operator(dims, 1).shape[0] == edges


def test_roughness_of_ramps():
    # f_n = x: every x-edge differs by 1; literal Eq. 8 counts each edge twice with 1/2
    nx, ny = 7, 4
    x = np.tile(np.arange(nx, dtype=float), ny)[None, :]
    assert grid.roughness(x, (nx, ny), 2) == pytest.approx((nx - 1) * ny)
    assert grid.roughness(x, (nx, ny), 1) == pytest.approx(0.5 * (nx - 1) * ny)
    y = np.repeat(np.arange(ny, dtype=float), nx)[None, :] * 3.0
    assert grid.roughness(y, (nx, ny), 2) == pytest.approx(9.0 * nx * (ny - 1))
    # a constant map has no roughness; maps add independently
    c = np.full((1, nx * ny), 2.5)
    assert grid.roughness(c, (nx, ny), 2) == pytest.approx(0.0)
    assert grid.roughness(np.vstack([x, y]), (nx, ny), 2) == pytest.approx(
        (nx - 1) * ny + 9.0 * nx * (ny - 1))


def test_neighbor_index_layout_x_fastest():
    n, m = grid.neighbor_pairs((4, 3))
    pairs = set(zip(n.tolist(), m.tolist()))
    assert (0, 1) in pairs and (1, 0) in pairs      # x neighbours
    assert (0, 4) in pairs and (4, 0) in pairs      # y neighbours (stride nx)
    assert (3, 4) not in pairs                      # no wrap across rows


def test_xi_p_rule():
    assert grid.xi_p_rule(1e-2, (32, 32)) == pytest.approx(
        0.75 * 1e-2 * 2 * 2 * (2 + 2 * np.cos(np.pi / 32)) + 1e-10, rel=1e-14)
    assert grid.xi_p_rule(0.0, (5, 5)) == pytest.approx(1e-10)
