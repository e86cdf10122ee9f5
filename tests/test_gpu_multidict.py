"""Spatially varying dictionaries on the GPU (ssm_plan_multi) against the FP64 oracle
(oracle/multidict.py, pinned in test_oracle_multidict.py). Needs a GB300.

Bar: after a fixed iteration count from the zero start, ||z_gpu - z_oracle||_F <=
1e-5 ||z_oracle||_F -- the FP32 bar of the single-dictionary low-rank form, whose
arithmetic this path shares. Cases: random labels (every 32-voxel tile mixes
dictionaries), the smooth quantised-B1 labels of the fingerprinting stand-in, 1D, 2D and
3D grids with ragged last tiles, each dictionary's rank by the rank rule and a fixed
rank on both sides of the Gram eigenproblem (P < Q and P > Q). At the bench size the
sampled voxels are checked against the oracle on the patch of half-width k around them.
"""
import numpy as np
import pytest
import torch

from oracle import grid, multidict as MD
from paper_2401_12890_gb300 import ssm, synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    yield


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(M):
    return torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()


def b1_case(dims, levels, seed, random_labels=False, n_tp=60):
    Ks, labels, M, _ = synth.b1_varying_problem(dims, levels, n_tp=n_tp, seed=seed)
    if random_labels:
        labels = np.random.default_rng(seed + 1).integers(0, levels, labels.size)
    return Ks, labels, M


def random_case(ndict, P, Q, dims, seed):
    Ks = [synth.random_problem(P, Q, (1, 1), seed + 13 * c)[0] for c in range(ndict)]
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    labels = rng.integers(0, ndict, N)
    M = rng.uniform(0.0, 1.0, (P, N)) * 5.0
    return Ks, labels, M


def run_gpu(Ks, labels, M, dims, lam, beta, **kw):
    plan = ssm.MultiPlan(Ks, labels, dims, lam, beta, **kw)
    F, info = plan.solve(dev(M))
    out = F.cpu().numpy().astype(np.float64)
    plan.close()
    return out, info


CASES = [
    # (id, problem builder, dims, lam, beta, iters, rank)
    ("b1_random_labels_2d", lambda d: b1_case(d, 4, 1, random_labels=True), (37, 29), 0.02,
     0.05, 200, 0),
    ("b1_smooth_labels_2d", lambda d: b1_case(d, 6, 2), (48, 40), 0.01, 0.03, 150, 0),
    ("b1_3d", lambda d: b1_case(d, 3, 3, random_labels=True), (9, 7, 5), 0.02, 0.05, 120, 0),
    ("b1_1d", lambda d: b1_case(d, 5, 4, random_labels=True), (301,), 0.02, 0.05, 150, 0),
    ("random_kkt_side_rank12", lambda d: random_case(3, 20, 50, d, 5), (23, 17), 0.05, 0.8, 100,
     12),
    ("random_ktk_side_rank8", lambda d: random_case(4, 50, 20, d, 6), (19, 21), 0.05, 0.8, 100,
     8),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_matches_the_oracle(case):
    _, build, dims, lam, beta, iters, rank = case
    Ks, labels, M = build(dims)
    F, info = run_gpu(Ks, labels, M, dims, lam, beta, rank=rank, max_iter=iters,
                      check_every=0)
    ref = MD.ladmm_multi(Ks, labels, M.astype(np.float32).astype(np.float64), dims, lam,
                         beta, rank=rank or None, iters=iters, check_every=0)
    assert info["iterations"] == iters
    assert info["rank"] == max(ref["ranks"])
    assert info["xi_p"] == pytest.approx(ref["xi_p"], rel=1e-12)
    assert F.min() >= 0.0
    err = rel(F, ref["z"])
    print(f"{case[0]}: ranks {ref['ranks']} rel err {err:.3e}")
    assert err <= RTOL


def test_stopping_rule_matches_the_oracle():
    dims = (40, 33)
    Ks, labels, M = b1_case(dims, 4, 7, random_labels=True)
    kw = dict(tol_primal=3e-3, tol_change=3e-3, check_every=10)
    F, info = run_gpu(Ks, labels, M, dims, 0.02, 0.05, max_iter=5000, **kw)
    ref = MD.ladmm_multi(Ks, labels, M.astype(np.float32).astype(np.float64), dims, 0.02, 0.05,
                         iters=5000, **kw)
    assert info["status"] == ssm.SSM_OK
    assert info["iterations"] == ref["iters"]
    k, rp, rc = ref["history"][-1]
    assert info["res_primal"] == pytest.approx(rp, rel=1e-3)
    assert info["res_change"] == pytest.approx(rc, rel=1e-3)
    assert rel(F, ref["z"]) <= RTOL


def test_one_dictionary_is_the_single_dictionary_plan():
    dims = (45, 31)
    Ks, _, M = b1_case(dims, 1, 8)
    labels = np.zeros(int(np.prod(dims)), np.int64)
    F, info = run_gpu(Ks, labels, M, dims, 0.02, 0.05, max_iter=150, check_every=0)
    plan = ssm.Plan(Ks[0], dims, 0.02, 0.05, form="lowrank", max_iter=150, check_every=0)
    F1, info1 = plan.solve(dev(M))
    plan.close()
    assert info["rank"] == info1["rank"]
    # the same iteration; the kernels sum the rank-r products in another order
    assert rel(F, F1.cpu().numpy().astype(np.float64)) <= 1e-6


def test_relabelling_the_dictionaries_is_bitwise():
    dims = (33, 18)
    Ks, labels, M = b1_case(dims, 5, 9, random_labels=True)
    F, _ = run_gpu(Ks, labels, M, dims, 0.02, 0.05, max_iter=60, check_every=0)
    perm = np.array([3, 0, 4, 1, 2])          # dictionary c moves to slot perm[c]
    Kp = [None] * len(Ks)
    for c, K in enumerate(Ks):
        Kp[perm[c]] = K
    Fp, _ = run_gpu(Kp, perm[labels], M, dims, 0.02, 0.05, max_iter=60, check_every=0)
    assert np.array_equal(F, Fp)


def test_resume_repeats_the_longer_solve():
    dims = (29, 26)
    Ks, labels, M = b1_case(dims, 3, 10, random_labels=True)
    Md = dev(M)
    full = ssm.MultiPlan(Ks, labels, dims, 0.02, 0.05, max_iter=50, check_every=7)
    F_full, _ = full.solve(Md)
    full.close()
    part = ssm.MultiPlan(Ks, labels, dims, 0.02, 0.05, max_iter=20, check_every=7)
    part.solve(Md)
    part.set_max_iter(30)
    F_res, info = part.resume(Md)
    part.close()
    assert info["iterations"] == 30
    assert torch.equal(F_res, F_full)


def test_graphs_give_the_same_iterates():
    dims = (31, 27)
    Ks, labels, M = b1_case(dims, 4, 11, random_labels=True)
    Md = dev(M)
    a = ssm.MultiPlan(Ks, labels, dims, 0.02, 0.05, max_iter=90, check_every=10,
                      tol_primal=1e-9)
    Fa, ia = a.solve(Md)
    a.close()
    b = ssm.MultiPlan(Ks, labels, dims, 0.02, 0.05, max_iter=90, check_every=10,
                      tol_primal=1e-9)
    b.set_graphs(True)
    Fb, ib = b.solve(Md)
    Fb2, _ = b.solve(Md)                     # replayed graphs
    b.close()
    assert torch.equal(Fa, Fb) and torch.equal(Fa, Fb2)
    assert ia["res_primal"] == ib["res_primal"]


def test_invalid_and_unsupported_calls():
    dims = (6, 5)
    Ks, labels, M = b1_case(dims, 3, 12, random_labels=True)
    bad = labels.copy()
    bad[7] = 3
    with pytest.raises(ssm.SsmError) as e:
        ssm.MultiPlan(Ks, bad, dims, 0.02, 0.05)
    assert e.value.status == ssm.SSM_EINVAL
    bad[7] = -1
    with pytest.raises(ssm.SsmError) as e:
        ssm.MultiPlan(Ks, bad, dims, 0.02, 0.05)
    assert e.value.status == ssm.SSM_EINVAL
    # a dictionary of rank 40 is past the path's rank limit (32)
    Kbig = [synth.random_problem(60, 40, (1, 1), 3, full_rank=True)[0]] * 2
    with pytest.raises(ssm.SsmError) as e:
        ssm.MultiPlan(Kbig, np.zeros(30, np.int64), dims, 0.02, 0.05)
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    plan = ssm.MultiPlan(Ks, labels, dims, 0.02, 0.05, max_iter=5)
    Md = dev(M)
    F, _ = plan.solve(Md)
    with pytest.raises(ssm.SsmError) as e:
        plan.objective(Md, F)
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    with pytest.raises(ssm.SsmError) as e:
        plan.set_beta(0.1)
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    with pytest.raises(ssm.SsmError) as e:
        plan.set_mask(np.ones(30))
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    info = plan.info()
    assert info["rank"] >= 1 and info["kk_norm"] > 0
    plan.close()


def patch_reference_multi(Ks, labels, M, dims, lam, beta, xi, n_iter, centre):
    """The oracle on the box of half-width n_iter around `centre`, clipped to the grid."""
    lo = [max(0, c - n_iter) for c in centre]
    hi = [min(d, c + n_iter + 1) for c, d in zip(centre, dims)]
    pd = tuple(h - l for l, h in zip(lo, hi))
    cols = []
    for idx in np.ndindex(*reversed(pd)):
        coord = list(reversed(idx))
        flat, stride = 0, 1
        for ax in range(len(dims)):
            flat += (lo[ax] + coord[ax]) * stride
            stride *= dims[ax]
        cols.append(flat)
    # only the patch's dictionaries (relabelling them changes nothing: an oracle pin)
    present, local = np.unique(labels[cols], return_inverse=True)
    res = MD.ladmm_multi([Ks[c] for c in present], local, M[:, cols], pd, lam, beta, xi_p=xi,
                         iters=n_iter, check_every=0)
    loc, stride = 0, 1
    for ax in range(len(dims)):
        loc += (centre[ax] - lo[ax]) * stride
        stride *= pd[ax]
    flat, stride = 0, 1
    for ax in range(len(dims)):
        flat += centre[ax] * stride
        stride *= dims[ax]
    return res["z"][:, loc], flat


def test_bench_size_sampled_voxels():
    """The fingerprinting stand-in at the bench's size (156 x 156, 61 B1 levels)."""
    w = synth.B1_WORKLOAD
    Ks, labels, M, _ = synth.make_b1_problem()
    n_iter = 6
    plan = ssm.MultiPlan(Ks, labels, w.dims, w.lam, w.beta, max_iter=n_iter, check_every=0)
    F, info = plan.solve(dev(M))
    plan.close()
    assert info["iterations"] == n_iter
    rng = np.random.default_rng(21)
    centres = [(0, 0), (155, 155), (78, 0), (0, 90)] + [tuple(int(v) for v in
                                                           rng.integers(0, 156, 2))
                                                     for _ in range(4)]
    xi = grid.xi_p_rule(w.lam, w.dims)
    M64 = M.astype(np.float64)
    worst = 0.0
    for c in centres:
        zref, flat = patch_reference_multi(Ks, labels, M64, w.dims, w.lam, w.beta, xi, n_iter, c)
        err = rel(F[:, flat].cpu().numpy().astype(np.float64), zref)
        worst = max(worst, err)
        assert err <= RTOL, (c, err)
    print(f"b1 bench size: rank {info['rank']}, worst sampled rel err {worst:.3e}")
