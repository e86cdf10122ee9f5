"""The TF32x3 low-rank form (SSM_TF32X3: Algorithm 2 with both rank-r products of Eq. 28
on the tcgen05 tensor cores) against the FP64 oracle, through the C ABI. Needs a GB300.

Tolerance. Each rank-r product is formed from TF32 hi/lo splits of both operands as
hi.hi + hi.lo + lo.hi; a split leaves at most 2^-11 of its operand in lo and the dropped
lo.lo term is at most 2^-22 of the product, the same order as FP32's own rounding
(2^-24) times the few terms it is summed over. So the form is held to the FP32 forms'
bar: ||z_gpu - z_oracle||_F <= 1e-5 ||z_oracle||_F after a fixed iteration count from
the zero start, on the 300-iteration 32x32 workload and on the edge cases (ragged tiles,
1D/3D grids, one voxel, P > Q, ranks padded to 32 and to 64, lambda = 0, both stencil
conventions, masks, batched slices, shares that split tiles into segments). Full-size
workloads are checked voxel by voxel against patch oracles, as for the FP32 forms.
"""
import numpy as np
import pytest
import torch

from oracle import grid, ladmm as L
from paper_2401_12890_gb300 import ssm, synth
from test_gpu_mask import random_mask
from test_gpu_parity import patch_reference, rel

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    yield


def tc_solve(K, M, dims, lam, beta, mask=None, **kw):
    plan = ssm.Plan(K, dims, lam, beta, form="lowrank", precision="tf32x3", **kw)
    if mask is not None:
        plan.set_mask(mask)
    F, info = plan.solve(torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda())
    out = F.cpu().numpy()
    plan.close()
    return out, info


def test_tiny_workload_300_iterations():
    w = synth.WORKLOADS["dr2d_tiny"]
    K, M, _ = synth.make_problem("dr2d_tiny")
    F, info = tc_solve(K, M, w.dims, w.lam, w.beta, max_iter=300, check_every=0)
    ref = L.ladmm(K, M, w.dims, w.lam, w.beta, iters=300, check_every=0)
    assert info["iterations"] == 300 and info["rank"] == ref["r"]
    assert F.min() >= 0.0
    err = rel(F, ref["z"])
    print(f"tf32x3 32x32, 300 iterations: rel err {err:.3e}")
    assert err <= RTOL


CASES = [
    # (P, Q, dims, lam, beta, rank, pairs)
    (8, 7, (13, 7), 0.05, 0.5, 3, 2),
    (6, 10, (37,), 0.2, 1.0, 0, 2),            # 1D
    (6, 10, (5, 4, 3), 0.2, 1.0, 5, 2),        # 3D
    (12, 5, (9, 9), 0.1, 2.0, 5, 2),           # P > Q: K^T K side
    (5, 9, (1, 1), 0.3, 1.0, 0, 2),            # single voxel
    (5, 9, (33, 1), 0.0, 1.0, 0, 2),           # lambda = 0
    (10, 33, (40, 3, 2), 0.02, 0.3, 1, 1),     # rank 1, one edge per pair
    (30, 70, (65, 65), 0.01, 0.1, 0, 2),       # several tiles + ragged tail
    (48, 100, (20, 9), 0.05, 1.0, 40, 2),      # rank padded to 64
    (40, 48, (6, 5, 4), 0.05, 1.0, 32, 2),     # rank 32 on a 3D grid
]


@pytest.mark.parametrize("P,Q,dims,lam,beta,rank,pairs", CASES)
def test_edge_cases_match_oracle(P, Q, dims, lam, beta, rank, pairs):
    K, M, _ = synth.random_problem(P, Q, dims, seed=P * 100 + Q, snr=50.0)
    iters = 40
    F, info = tc_solve(K, M, dims, lam, beta, rank=rank, stencil_pairs=pairs, max_iter=iters,
                       check_every=0)
    ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), dims, lam, beta,
                  rank=(rank or None), iters=iters, check_every=0, pairs=pairs)
    err = rel(F, ref["z"])
    print(f"tf32x3 {dims} r={info['rank']}: rel err {err:.3e}")
    assert info["rank"] == ref["r"]
    assert err <= RTOL


def test_rank_above_32_on_3d_grids_is_refused():
    K, _, _ = synth.random_problem(40, 48, (6, 5, 4), seed=3)
    with pytest.raises(ssm.SsmError) as e:
        ssm.Plan(K, (6, 5, 4), 0.05, 1.0, form="lowrank", precision="tf32x3", rank=40)
    assert e.value.status == ssm.SSM_EUNSUPPORTED


def test_dense_form_refuses_tf32x3():
    K, _, _ = synth.random_problem(8, 12, (5, 5), seed=3)
    with pytest.raises(ssm.SsmError) as e:
        ssm.Plan(K, (5, 5), 0.05, 1.0, form="dense", precision="tf32x3")
    assert e.value.status == ssm.SSM_EUNSUPPORTED


# shares of the (tile, chunk) units that split tiles into several segments, few CTAs
# with many tiles each, and the stopping rule (the residual-test variant)
@pytest.mark.parametrize("grid,P,Q,dims,tol,stop", [
    (7, 14, 100, (20, 16, 12), 0.0, 40),    # 30 tiles over 7 CTAs
    (5, 10, 70, (40, 36), 0.0, 40),         # 12 tiles over 5 CTAs
    (3, 12, 64, (30, 30, 9), 1e-3, 400),    # 64 tiles over 3 CTAs, with the stopping rule
    (150, 14, 130, (20, 16, 12), 0.0, 40),  # more CTAs than tiles: several segments per tile
])
def test_share_layouts_match_oracle(monkeypatch, grid, P, Q, dims, tol, stop):
    monkeypatch.setenv("SSM_LRTC_GRID", str(grid))
    K, M, _ = synth.random_problem(P, Q, dims, seed=grid * 7 + Q, snr=50.0)
    F, info = tc_solve(K, M, dims, 0.05, 1.0, max_iter=stop, check_every=10 if tol else 0,
                       tol_primal=tol, tol_change=tol)
    ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), dims, 0.05, 1.0, iters=stop,
                  check_every=10 if tol else 0, tol_primal=tol, tol_change=tol)
    if tol:
        # residuals agree to ~1e-5 relative: the stop is the same test unless the
        # oracle's last one was within that margin of the tolerance
        assert abs(info["iterations"] - ref["iters"]) <= 10
    else:
        assert info["iterations"] == ref["iters"]
    err = rel(F, ref["z"]) if info["iterations"] == ref["iters"] else 0.0
    print(f"grid {grid} dims {dims}: {info['iterations']} iterations, rel err {err:.3e}")
    assert err <= RTOL


@pytest.mark.parametrize("waves", [2, 8])
def test_launch_waves_match_oracle(waves):
    K, M, _ = synth.random_problem(20, 90, (48, 40), seed=waves, snr=50.0)
    F, info = tc_solve(K, M, (48, 40), 0.05, 1.0, max_iter=30, check_every=0,
                       launch_waves=waves)
    ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), (48, 40), 0.05, 1.0, iters=30,
                  check_every=0)
    assert rel(F, ref["z"]) <= RTOL


@pytest.mark.parametrize("dims,seed", [((30, 26), 1), ((12, 10, 8), 2), ((200, 3), 3)])
def test_masked_solve_matches_oracle(dims, seed):
    K, M, _ = synth.random_problem(16, 40, dims, seed=seed, snr=50.0)
    mask = random_mask(dims, seed)
    F, info = tc_solve(K, M, dims, 0.05, 1.0, mask=mask, max_iter=40, check_every=0)
    ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), dims, 0.05, 1.0, iters=40,
                  check_every=0, rank=info["rank"], mask=mask)
    assert not F[:, ~mask].any()
    assert rel(F, ref["z"]) <= RTOL


def test_batched_slices_match_oracle_per_slice():
    dims, B = (21, 17), 3
    K, _, _ = synth.random_problem(14, 36, dims, seed=4)
    rng = np.random.default_rng(4)
    N = int(np.prod(dims))
    Ms = []
    for b in range(B):
        Ft = rng.uniform(0, 1, (36, N)) * (rng.uniform(0, 1, (36, N)) < 0.4)
        Mb = K @ Ft
        Ms.append(Mb + rng.standard_normal(Mb.shape) * (np.abs(Mb).max() / 50.0))
    M = np.concatenate(Ms, axis=1)
    F, info = tc_solve(K, M, dims, 0.05, 1.0, max_iter=40, check_every=0, batch=B)
    for b in range(B):
        ref = L.ladmm(K, Ms[b].astype(np.float32).astype(np.float64), dims, 0.05, 1.0,
                      iters=40, check_every=0)
        assert rel(F[:, b * N:(b + 1) * N], ref["z"]) <= RTOL


def test_repeat_solves_are_bitwise_identical():
    w = synth.WORKLOADS["dr2d_tiny"]
    K, M, _ = synth.make_problem("dr2d_tiny")
    plan = ssm.Plan(K, w.dims, w.lam, w.beta, form="lowrank", precision="tf32x3", max_iter=50,
                    check_every=0)
    Md = torch.from_numpy(M).cuda()
    a, _ = plan.solve(Md)
    b, _ = plan.solve(Md)
    plan.close()
    assert torch.equal(a, b)


@pytest.mark.parametrize("name,n_iter", [("dr2d_slice", 12), ("mrf2d", 10), ("rr3d_t1t2", 6)])
def test_full_size_sampled_voxels(name, n_iter):
    w = synth.WORKLOADS[name]
    K, M, _ = synth.make_problem(name)
    F, info = tc_solve(K, M, w.dims, w.lam, w.beta, max_iter=n_iter, check_every=0)
    rng = np.random.default_rng(5)
    dims = w.dims
    centres = [tuple(0 for _ in dims), tuple(d - 1 for d in dims), tuple(d // 2 for d in dims)]
    centres += [tuple(int(v) for v in rng.integers(0, dims)) for _ in range(3)]
    xi = grid.xi_p_rule(w.lam, dims)
    M64 = M.astype(np.float64)
    for c in centres:
        zref, flat = patch_reference(K, M64, dims, w.lam, w.beta, xi, n_iter, c, "lowrank",
                                     info["rank"])
        err = rel(F[:, flat], zref)
        print(f"{name} {c}: rel err {err:.3e}")
        assert err <= RTOL, (c, err)
    assert F.min() >= 0.0


@pytest.mark.parametrize("precision", ["tf32x3", "fp32"])
@pytest.mark.parametrize("name,dims", [("dr2d_tiny", None), ("rr3d_t1t2", (20, 18, 12))])
def test_residual_tests_leave_the_iterate_unchanged(precision, name, dims):
    """The iteration kernels with a residual test (which also read d^k, and in the TF32x3
    form run twice the epilogue warps) and those that store d for the next test must
    produce the same z as the plain ones: a test at every iteration and a test at none
    give the same iterate, bit for bit."""
    w = synth.WORKLOADS[name]
    dims = dims or w.dims
    K, M, _ = synth.make_problem(name, dims=dims)
    Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
    out = []
    for ce, tol in ((0, 0.0), (1, 1e-30), (3, 1e-30)):
        plan = ssm.Plan(K, dims, w.lam, w.beta, form="lowrank", precision=precision,
                        max_iter=24, check_every=ce, tol_primal=tol)
        F, info = plan.solve(Md)
        assert info["iterations"] == 24
        out.append(F.clone())
        plan.close()
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])
