"""Pins of the oracle's beta heuristic (Sec. III-E: beta tuned on a 3x3 image patch).

centre_patch is checked against flat voxel indices listed by hand (x fastest,
n = x + nx*(y + ny*z)) on odd and even 1D, 2D and 3D grids. tune_beta is checked on
problems whose iterates follow a linear recurrence written out here from Eq. 28 and
Eq. 31 (one compartment, positive data, so the projection never clamps):

  * one voxel, lambda = 0: the error contracts by beta/(beta + sigma^2) per iteration,
    so J(z^k) = J* + sigma^2 z*^2 rho^(2k) / 2 in closed form and the smallest
    candidate beta wins;
  * a chain of 3 voxels, lambda > 0: xi_p > 0 slows small betas, the f-step slows
    large ones, and the best candidate lies strictly inside the grid.

Planted mistakes in oracle/tune.py (axes swapped, an off-by-one start, argmax for
argmin, sigma_1 for sigma_1^2, one iteration too many) each fail one of these pins.
"""
import os
import sys
import types

import numpy as np
import pytest

from oracle import tune

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle")


def _cols(tune_mod, dims):
    N = int(np.prod(dims))
    M = np.arange(N, dtype=np.float64)[None, :]     # column n holds the value n
    Mp, pdims = tune_mod.centre_patch(M, dims)
    return [int(v) for v in Mp[0]], pdims


CENTRE_CASES = [
    # (dims, hand-listed flat indices, patch dims)
    ((7, 5), [9, 10, 11, 16, 17, 18, 23, 24, 25], (3, 3)),
    ((8, 6), [19, 20, 21, 27, 28, 29, 35, 36, 37], (3, 3)),
    ((5,), [1, 2, 3], (3,)),
    ((3, 2), [0, 1, 2, 3, 4, 5], (3, 2)),
    ((8, 6, 4), [67, 68, 69, 75, 76, 77, 83, 84, 85,
                 115, 116, 117, 123, 124, 125, 131, 132, 133,
                 163, 164, 165, 171, 172, 173, 179, 180, 181], (3, 3, 3)),
    ((5, 3, 3), [1, 2, 3, 6, 7, 8, 11, 12, 13,
                 16, 17, 18, 21, 22, 23, 26, 27, 28,
                 31, 32, 33, 36, 37, 38, 41, 42, 43], (3, 3, 3)),
]


@pytest.mark.parametrize("dims,expected,pdims", CENTRE_CASES)
def test_centre_patch_indices(dims, expected, pdims):
    cols, got_dims = _cols(tune, dims)
    assert cols == expected
    assert tuple(got_dims) == pdims


# ------------------------------------------------------------------ closed-form problems

def _one_voxel_problem():
    k = np.array([[1.0], [0.7], [0.4]])              # P = 3, Q = 1
    z_true = 2.0
    m = k[:, 0] * z_true + np.array([0.05, -0.02, 0.03])
    return k, m[:, None]


def _one_voxel_table(k, m, iters, betas):
    """J(z^iters) per beta from the scalar recurrence (lambda = 0, one voxel).

    One compartment, rank 1: Eq. 28 gives f = c/(beta + sigma^2). With xi_p = 1e-10
    (Eq. 32 with ||D^T D|| = 0) the dual returns to its fixed point 0 after the first
    step and z - z* contracts by rho = beta/(beta + sigma^2) per iteration (xi_p is
    kept exactly below; the recurrence is iterated, not approximated).
    """
    s2 = float(k[:, 0] @ k[:, 0])
    g = float(k[:, 0] @ m[:, 0])
    xi = 1e-10
    out = {}
    for beta in betas:
        z = d = 0.0
        for _ in range(iters):
            f = (g + beta * z - d) / (beta + s2)
            z_new = (xi * z + beta * f + d) / (xi + beta)
            assert z_new > 0.0
            d = d - beta * (z_new - f)
            z = z_new
        out[beta] = 0.5 * float(np.sum((m[:, 0] - k[:, 0] * z) ** 2))
    return out


def test_one_voxel_closed_form_contraction():
    """The recurrence above is the contraction rho^k (checks it against the closed form)."""
    k, m = _one_voxel_problem()
    s2 = float(k[:, 0] @ k[:, 0])
    zs = float(k[:, 0] @ m[:, 0]) / s2
    Jstar = 0.5 * float(np.sum((m[:, 0] - k[:, 0] * zs) ** 2))
    for beta in (0.1, 1.0, 7.0):
        rho = beta / (beta + s2)
        J = _one_voxel_table(k, m, 25, [beta])[beta]
        assert J == pytest.approx(Jstar + 0.5 * s2 * (zs * rho ** 25) ** 2, rel=1e-9, abs=1e-14)


def _chain_problem():
    """Q = 1 on a 5-voxel line; the centre patch is voxels 1..3 (a 3-voxel chain)."""
    k = np.array([[1.2], [0.9], [0.5], [0.3]])       # P = 4
    z_true = np.array([1.5, 1.0, 1.4, 0.9, 1.2])
    noise = np.array([[0.03, -0.02, 0.01, 0.02, -0.01]]) * np.array([[1.0], [0.5], [-0.7], [0.2]])
    return k, k @ z_true[None, :] + noise


def _chain_table(k, m_patch, lam, iters, betas):
    """J(z^iters) per beta from the 3-voxel affine recurrence (Eq. 28 and Eq. 31).

    L2 = D^T D of the literal Eq. 8 on a 3-chain (each pair counted from both ends):
    twice the path Laplacian [[1,-1,0],[-1,2,-1],[0,-1,1]], whose norm is 2*3 = 6,
    so xi_p = 0.75*lambda*6 + 1e-10 (Eq. 32).
    """
    L2 = 2.0 * np.array([[1.0, -1.0, 0.0], [-1.0, 2.0, -1.0], [0.0, -1.0, 1.0]])
    xi = 0.75 * lam * 6.0 + 1e-10
    s2 = float(k[:, 0] @ k[:, 0])
    g = k[:, 0] @ m_patch                            # K^T m_n per voxel
    out = {}
    for beta in betas:
        z = np.zeros(3)
        d = np.zeros(3)
        for _ in range(iters):
            f = (g + beta * z - d) / (beta + s2)
            z_new = (xi * z - lam * (L2 @ z) + beta * f + d) / (xi + beta)
            assert np.all(z_new > 0.0)
            d = d - beta * (z_new - f)
            z = z_new
        data = 0.5 * float(np.sum((m_patch - k @ z[None, :]) ** 2))
        out[beta] = data + lam * 0.5 * float(z @ L2 @ z)
    return out


def _betas(k, n_grid, lo, hi):
    s = float(np.linalg.norm(k))
    return [float(b) for b in s ** 2 * np.logspace(lo, hi, n_grid)]


def test_tune_beta_one_voxel_lambda0(tune_mod=tune):
    k, m = _one_voxel_problem()
    # few iterations, so that J(z^k) - J* stays far above FP64 rounding of J*
    best, table = tune_mod.tune_beta(k, m, (1,), 0.0, iters=3, n_grid=9, grid_lo=-1.0,
                                     grid_hi=1.0)
    ref = _one_voxel_table(k, m, 3, _betas(k, 9, -1.0, 1.0))
    assert len(table) == len(ref)
    for (b, J), (rb, rJ) in zip(sorted(table.items()), sorted(ref.items())):
        assert b == pytest.approx(rb, rel=1e-12)
        assert J == pytest.approx(rJ, rel=1e-9, abs=1e-14)
    # the contraction beta/(beta + sigma^2) grows with beta: the smallest candidate wins
    assert best == pytest.approx(min(ref), rel=1e-12)


def test_tune_beta_chain_interior_optimum(tune_mod=tune):
    k, m = _chain_problem()
    lam, iters = 0.4, 15
    best, table = tune_mod.tune_beta(k, m, (5,), lam, iters=iters, n_grid=13, grid_lo=-3.0,
                                     grid_hi=2.0)
    ref = _chain_table(k, m[:, 1:4], lam, iters, _betas(k, 13, -3.0, 2.0))
    for (b, J), (rb, rJ) in zip(sorted(table.items()), sorted(ref.items())):
        assert b == pytest.approx(rb, rel=1e-12)
        assert J == pytest.approx(rJ, rel=1e-9)
    ref_best = min(ref, key=lambda b: (ref[b], b))
    betas = sorted(ref)
    assert betas[0] < ref_best < betas[-1]           # the optimum is not at an end
    assert best == pytest.approx(ref_best, rel=1e-12)


# ------------------------------------------------------------------ planted mistakes

def load_tune_mutant(old, new):
    src = open(os.path.join(ORACLE_DIR, "tune.py")).read()
    assert old in src, f"mutation anchor not found: {old!r}"
    at = src.rindex(old)
    src = src[:at] + new + src[at + len(old):]
    import oracle.ladmm
    pkg = types.ModuleType("oracle_tune_mut")
    pkg.__path__ = []
    pkg.ladmm = oracle.ladmm
    sys.modules["oracle_tune_mut"] = pkg
    sys.modules["oracle_tune_mut.ladmm"] = oracle.ladmm
    m = types.ModuleType("oracle_tune_mut.tune")
    m.__package__ = "oracle_tune_mut"
    exec(compile(src, "<mutant tune>", "exec"), m.__dict__)
    return m


TUNE_MUTATIONS = [
    ("coord = list(reversed(n))", "coord = list(n)"),
    ("starts = [max(0, d // 2 - size // 2) for d in dims]",
     "starts = [max(0, d // 2 - size // 2 + 1) for d in dims]"),
    ("best = min(table, key=lambda b: (table[b], b))",
     "best = max(table, key=lambda b: (table[b], b))"),
    ("for b in s[0] ** 2 * np.logspace", "for b in s[0] * np.logspace"),
    ("rank=r, iters=iters, check_every=0", "rank=r, iters=iters + 1, check_every=0"),
]


def _tune_pins_pass(mod):
    try:
        for dims, expected, pdims in CENTRE_CASES:
            cols, got = _cols(mod, dims)
            if cols != expected or tuple(got) != pdims:
                return False
        test_tune_beta_one_voxel_lambda0(mod)
        test_tune_beta_chain_interior_optimum(mod)
        return True
    except AssertionError:
        return False


def test_unmutated_tune_passes():
    assert _tune_pins_pass(load_tune_mutant("import numpy as np", "import numpy as np"))


@pytest.mark.parametrize("old,new", TUNE_MUTATIONS)
def test_tune_mutation_is_caught(old, new):
    assert not _tune_pins_pass(load_tune_mutant(old, new))
