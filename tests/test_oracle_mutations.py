"""Planted mistakes in the oracle must be caught by its pins.

Each case copies an oracle module's source, plants one plausible mistake (a sign,
a dropped factor, a wrong index), loads the copy in place of the original, and runs
the pins that do not depend on the oracle's own formulas: per-voxel NNLS at
lambda = 0, an independent FISTA solver at lambda > 0, and the closed-form single-
compartment linear system. At least one must fail for every mutation.
"""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest
import scipy.optimize

from oracle import grid as grid_ok, pg
from paper_2401_12890_gb300 import synth

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle")


def load_mutant(module, old, new):
    src = open(os.path.join(ORACLE_DIR, module + ".py")).read()
    assert old in src, f"mutation anchor not found: {old!r}"
    at = src.rindex(old)            # the code, not the module docstring
    src = src[:at] + new + src[at + len(old):]
    pkg = types.ModuleType("oracle_mut")
    pkg.__path__ = []
    sys.modules["oracle_mut"] = pkg
    mods = {}
    for name in ("grid", "ladmm"):
        text = src if name == module else open(os.path.join(ORACLE_DIR, name + ".py")).read()
        m = types.ModuleType("oracle_mut." + name)
        m.__package__ = "oracle_mut"
        sys.modules["oracle_mut." + name] = m
        setattr(pkg, name, m)
        exec(compile(text, f"<mutant {name}>", "exec"), m.__dict__)
        mods[name] = m
    return mods["ladmm"], mods["grid"]


def pins_pass(L, G):
    try:
        # lambda = 0: per-voxel NNLS
        K, M, _ = synth.random_problem(8, 5, (3, 2), 0, snr=20.0, full_rank=True)
        out = L.ladmm(K, M, (3, 2), 0.0, beta=2.0, rank=5, iters=3000, check_every=0)
        F = np.stack([scipy.optimize.nnls(K, M[:, n])[0] for n in range(M.shape[1])], 1)
        if not np.allclose(out["z"], F, atol=1e-7):
            return False
        # lambda > 0, full column rank: FISTA's minimiser
        K, M, _ = synth.random_problem(12, 9, (4, 3), 21, snr=30.0, full_rank=True)
        out = L.ladmm(K, M, (4, 3), 0.5, beta=3.0, rank=9, iters=4000, check_every=0)
        Z, _ = pg.fista(K, M, (4, 3), 0.5, iters=100000, tol=1e-16)
        if not np.allclose(out["z"], Z, atol=1e-6):
            return False
        # Q = 1 interior solution of a linear system, on a 3D grid
        dims = (3, 4, 2)
        N = 24
        rng = np.random.default_rng(11)
        k = rng.uniform(0.5, 1.5, (6, 1))
        M = k @ (2.0 + np.sin(np.arange(N) / 3.0))[None, :]
        kk = float((k.T @ k)[0, 0])
        A = kk * np.eye(N) + 0.7 * grid_ok.dtd(dims, 2).toarray()
        z_lin = np.linalg.solve(A, (k.T @ M).ravel())
        out = L.ladmm(k, M, dims, 0.7, beta=kk, rank=1, iters=3000, check_every=0)
        if not np.allclose(out["z"].ravel(), z_lin, atol=1e-8):
            return False
        # the dense (Eq. 26) variant on the same lambda > 0 problem
        K, M, _ = synth.random_problem(12, 9, (4, 3), 21, snr=30.0, full_rank=True)
        out = L.ladmm(K, M, (4, 3), 0.5, beta=3.0, dense=True, iters=4000, check_every=0)
        if not np.allclose(out["z"], Z, atol=1e-6):
            return False
        return True
    except Exception:
        return False


def test_unmutated_oracle_passes():
    L, G = load_mutant("ladmm", "import numpy as np", "import numpy as np")
    assert pins_pass(L, G)


MUTATIONS = [
    ("ladmm", "d = d - beta * (z_new - f)", "d = d + beta * (z_new - f)"),
    ("ladmm", "lam * grid.apply_dtd(z, DtD)", "0.5 * lam * grid.apply_dtd(z, DtD)"),
    ("ladmm", "return s2 / (beta * beta + beta * s2)", "return s2 / (beta * beta + s2)"),
    ("ladmm", "c = G + beta * z - d", "c = G + beta * z + d"),
    ("ladmm", "G = Vr @ (sr[:, None] * (Ur.T @ M))", "G = Vr @ (Ur.T @ M)"),
    ("ladmm", "(xi_p * z - lam", "(- lam"),
    ("ladmm", "/ (xi_p + beta))", "/ (xi_p + 2 * beta))"),
    ("ladmm", "f = c / beta - Vr", "f = c - Vr"),
    ("ladmm", "np.maximum(0.0, (xi_p", "np.abs((xi_p"),
    ("ladmm", "A = K.T @ K + beta * np.eye(K.shape[1])", "A = K.T @ K + np.eye(K.shape[1])"),
    ("ladmm", "G = K.T @ M", "G = K.T @ M * 0.5"),
    ("grid", "for ax in range(nd):", "for ax in range(nd - 1):"),
    ("grid", "b = np.take(idx, np.arange(1, dims[ax]), axis=arr_ax).ravel()",
     "b = np.take(idx, np.arange(0, dims[ax] - 1), axis=arr_ax).ravel()"),
    ("grid", "s = 2.0 if pairs == 2 else 1.0", "s = 1.0 if pairs == 2 else 2.0"),
]


@pytest.mark.parametrize("module,old,new", MUTATIONS)
def test_mutation_is_caught(module, old, new):
    L, G = load_mutant(module, old, new)
    if module == "grid" and "s = " in old:
        # the norm mutation only moves xi_p; the pin is its closed form
        assert G.dtd_norm((5, 4), 2) != pytest.approx(grid_ok.dtd_norm((5, 4), 2))
        return
    assert not pins_pass(L, G)
