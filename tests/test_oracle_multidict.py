"""Pins of the spatially varying dictionary oracle (oracle/multidict.py), no GPU.

Each pin checks against something other than the module's own formulas: the single-
dictionary oracle (itself pinned in test_oracle_ladmm.py) when every voxel has the same
dictionary, per-voxel NNLS with each voxel's own dictionary at lambda = 0, an
independent projected-gradient solver (and the KKT conditions) at lambda > 0, and
invariance under relabelling the dictionaries. Planted mistakes in a copy of the
module (the wrong voxel's dictionary, a dropped group, a wrong weight) must fail them.
"""
import functools
import os
import sys
import types

import numpy as np
import pytest
import scipy.optimize

from oracle import grid, ladmm as L, multidict as MD
from paper_2401_12890_gb300 import synth


def dictionaries(C, P, Q, seed):
    """C full-column-rank random dictionaries sharing P >= Q."""
    return [synth.random_problem(P, Q, (1, 1), seed + 17 * c, full_rank=True)[0]
            for c in range(C)]


def labelled_data(Ks, dims, seed, snr=40.0):
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    labels = rng.integers(0, len(Ks), N)
    Q = Ks[0].shape[1]
    F = rng.uniform(0.0, 1.0, (Q, N)) * (rng.uniform(0.0, 1.0, (Q, N)) < 0.5)
    M = np.empty((Ks[0].shape[0], N))
    for c, K in enumerate(Ks):
        sel = labels == c
        M[:, sel] = K @ F[:, sel]
    M += rng.standard_normal(M.shape) * (np.abs(M).max() / snr)
    return labels, M


@functools.lru_cache(maxsize=None)
def pin_cases():
    """The two pin problems and their independent solutions (computed once)."""
    Ks0 = dictionaries(3, 8, 5, 0)
    lab0, M0 = labelled_data(Ks0, (3, 4), 0)
    F0 = np.stack([scipy.optimize.nnls(Ks0[lab0[n]], M0[:, n])[0] for n in range(M0.shape[1])],
                  1)
    Ks1 = dictionaries(3, 12, 9, 5)
    lab1, M1 = labelled_data(Ks1, (4, 3), 5, snr=30.0)
    Z1, _ = MD.fista_multi(Ks1, lab1, M1, (4, 3), 0.5, iters=100000, tol=1e-16)
    return (Ks0, lab0, M0, F0), (Ks1, lab1, M1, Z1)



@pytest.mark.parametrize("dense,rank", [(False, None), (False, 3), (True, None)])
def test_one_dictionary_is_the_single_dictionary_oracle(dense, rank):
    K, M, _ = synth.random_problem(10, 7, (5, 4), seed=2, snr=30.0)
    labels = np.zeros(20, np.int64)
    a = MD.ladmm_multi([K], labels, M, (5, 4), 0.3, 1.5, dense=dense, rank=rank, iters=60,
                       check_every=0)
    b = L.ladmm(K, M, (5, 4), 0.3, 1.5, dense=dense, rank=rank, iters=60, check_every=0)
    assert np.allclose(a["z"], b["z"], rtol=0, atol=1e-12 * np.abs(b["z"]).max())
    assert np.allclose(a["d"], b["d"], rtol=0, atol=1e-12 * max(np.abs(b["d"]).max(), 1.0))


@pytest.mark.parametrize("seed", [0, 1])
def test_lambda_zero_is_voxelwise_nnls_with_own_dictionary(seed):
    Ks = dictionaries(3, 8, 5, seed)
    dims = (3, 4)
    labels, M = labelled_data(Ks, dims, seed)
    out = MD.ladmm_multi(Ks, labels, M, dims, 0.0, 2.0, rank=5, iters=3000, check_every=0)
    F = np.stack([scipy.optimize.nnls(Ks[labels[n]], M[:, n])[0] for n in range(M.shape[1])],
                 1)
    assert np.allclose(out["z"], F, atol=1e-7)


@pytest.mark.parametrize("dense", [False, True])
def test_positive_lambda_matches_projected_gradient_and_kkt(dense):
    _, (Ks, labels, M, Z) = pin_cases()         # FISTA's minimiser, computed once
    dims = (4, 3)
    lam = 0.5
    out = MD.ladmm_multi(Ks, labels, M, dims, lam, 3.0, dense=dense, rank=9, iters=4000,
                         check_every=0)
    J = MD.objective_multi(Ks, labels, M, Z, dims, lam)
    assert np.allclose(out["z"], Z, atol=1e-6)
    J_ladmm = MD.objective_multi(Ks, labels, M, out["z"], dims, lam)
    assert J_ladmm == pytest.approx(J, rel=1e-10)
    # KKT of the nonnegative problem at the LADMM point: gradient >= 0, complementary
    DtD = grid.dtd(dims)
    G = lam * grid.apply_dtd(out["z"], DtD)
    for c, K in enumerate(Ks):
        sel = labels == c
        G[:, sel] += K.T @ (K @ out["z"][:, sel] - M[:, sel])
    scale = np.abs(G).max()
    assert G.min() >= -1e-6 * scale
    assert np.abs(G[out["z"] > 1e-8]).max() <= 1e-6 * scale


def test_relabelling_the_dictionaries_changes_nothing():
    Ks = dictionaries(4, 9, 6, 9)
    dims = (5, 3)
    labels, M = labelled_data(Ks, dims, 9)
    perm = np.array([2, 0, 3, 1])               # new index of old dictionary c
    Ks2 = [None] * 4
    for c in range(4):
        Ks2[perm[c]] = Ks[c]
    a = MD.ladmm_multi(Ks, labels, M, dims, 0.2, 1.0, iters=50, check_every=0)
    b = MD.ladmm_multi(Ks2, perm[labels], M, dims, 0.2, 1.0, iters=50, check_every=0)
    assert np.array_equal(a["z"], b["z"]) and a["ranks"] == [b["ranks"][perm[c]] for c in range(4)]


def test_lowrank_at_full_rank_equals_dense():
    Ks = dictionaries(2, 10, 6, 13)
    dims = (4, 4)
    labels, M = labelled_data(Ks, dims, 13)
    a = MD.ladmm_multi(Ks, labels, M, dims, 0.4, 2.0, rank=6, iters=80, check_every=0)
    b = MD.ladmm_multi(Ks, labels, M, dims, 0.4, 2.0, dense=True, iters=80, check_every=0)
    assert np.allclose(a["z"], b["z"], rtol=0, atol=1e-10 * np.abs(b["z"]).max())


def test_b1_varying_stand_in_reaches_the_projected_gradient_objective():
    """The fingerprinting stand-in (4 B1 levels of the SPGR dictionary, 60 time points,
    Q = 30): LADMM's objective approaches FISTA's from above. The SPGR columns are
    strongly correlated, and convergence along the flat directions is slow whatever beta
    (3e-3 .. 3e-2 give the same gap): 5.7e-5 after 3000 iterations, 2.3e-6 after 30000,
    hence the 1e-5 bar at 30000."""
    Ks, labels, M, _ = synth.b1_varying_problem((8, 6), 4, seed=3)
    lam = 1e-2
    out = MD.ladmm_multi(Ks, labels, M, (8, 6), lam, 1e-2, dense=True, iters=30000,
                         check_every=0)
    _, J = MD.fista_multi(Ks, labels, M, (8, 6), lam, iters=200000, tol=1e-16)
    J_ladmm = MD.objective_multi(Ks, labels, M, out["z"], (8, 6), lam)
    assert J <= J_ladmm * (1 + 1e-12)
    assert J_ladmm == pytest.approx(J, rel=1e-5)


# --------------------------------------------------------------------------------------
# planted mistakes
# --------------------------------------------------------------------------------------
ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def load_mutant(old, new):
    src = open(os.path.join(ORACLE_DIR, "multidict.py")).read()
    assert old in src, old
    at = src.rindex(old)
    src = src[:at] + new + src[at + len(old):]
    pkg = types.ModuleType("oracle_md_mut")
    pkg.__path__ = []
    sys.modules["oracle_md_mut"] = pkg
    for name in ("grid", "ladmm"):
        m = types.ModuleType("oracle_md_mut." + name)
        m.__package__ = "oracle_md_mut"
        sys.modules["oracle_md_mut." + name] = m
        setattr(pkg, name, m)
        exec(compile(open(os.path.join(ORACLE_DIR, name + ".py")).read(), name, "exec"),
             m.__dict__)
    m = types.ModuleType("oracle_md_mut.multidict")
    m.__package__ = "oracle_md_mut"
    exec(compile(src, "<mutant multidict>", "exec"), m.__dict__)
    return m


def pins_pass(mod):
    (Ks, labels, M, F), (Ks1, lab1, M1, Z1) = pin_cases()
    out = mod.ladmm_multi(Ks, labels, M, (3, 4), 0.0, 2.0, rank=5, iters=3000, check_every=0)
    if not np.allclose(out["z"], F, atol=1e-7):
        return False
    out = mod.ladmm_multi(Ks1, lab1, M1, (4, 3), 0.5, 3.0, rank=9, iters=4000, check_every=0)
    return bool(np.allclose(out["z"], Z1, atol=1e-6))


MUTATIONS = [
    ("groups = [np.flatnonzero(labels == c) for c in range(len(Ks))]\n\n    # steps",
     "groups = [np.flatnonzero(labels == (c + 1) % len(Ks)) for c in range(len(Ks))]\n\n"
     "    # steps"),                                             # another voxel's dictionary
    ("                f[:, idx] = c / beta - Vr @ (W[:, None] * (Vr.T @ c))",
     "                f[:, idx] = c / beta - Vr @ (W[:, None] * (Vr.T @ c)) * (idx[0] != 0)"),
    ("G[:, idx] = Vr @ (sr[:, None] * (Ur.T @ M[:, idx]))",
     "G[:, idx] = Vr @ (Ur.T @ M[:, idx])"),                   # g without sigma
    ("for step, idx in zip(fstep, groups):\n            if not idx.size:",
     "for step, idx in zip(fstep[:1], groups[:1]):\n            if not idx.size:"),  # groups dropped
]


def test_unmutated_module_passes_the_pins():
    assert pins_pass(MD)


@pytest.mark.parametrize("old,new", MUTATIONS, ids=["wrong_dictionary", "missing_weight_term",
                                                    "g_without_sigma", "groups_dropped"])
def test_planted_mistake_fails_a_pin(old, new):
    assert not pins_pass(load_mutant(old, new))
