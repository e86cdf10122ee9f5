"""Batched plans (ssm_plan_batched): B independent slices sharing K solved by one plan,
against the FP64 oracle run on each slice alone. Needs a GB300.

The slices sit one after another in M and F; each slice's problem is Eq. 7 on its own
grid (no smoothness across the batch axis, the slice's own xi_p), so the oracle solves
them one by one. Slice sizes are not multiples of the 128-voxel tiles, so tiles straddle
slices. Bars: FP32 forms 1e-5 relative per slice after a fixed iteration count, BF16x3
1e-4 after 20 iterations.
"""
import numpy as np
import pytest
import torch

from oracle import admm as A
from oracle import ladmm as L
from paper_2401_12890_gb300 import ssm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    yield


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def batch_problem(dims, B, P=14, Q=36, seed=0):
    K, _, _ = synth.random_problem(P, Q, dims, seed=seed)
    # one K for every slice; each slice its own ground truth and noise
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    Ms = []
    for b in range(B):
        F = rng.uniform(0, 1, (Q, N)) * (rng.uniform(0, 1, (Q, N)) < 0.4)
        M = K @ F
        Ms.append(M + rng.standard_normal(M.shape) * (np.abs(M).max() / 50.0))
    return K, Ms


CASES = [("lowrank", "fp32", 40, 1e-5), ("dense", "fp32", 40, 1e-5),
         ("dense", "bf16x3", 20, 1e-4), ("admm", "fp32", 40, 1e-5)]


@pytest.mark.parametrize("form,prec,iters,tol", CASES, ids=[c[0] + "_" + c[1] for c in CASES])
@pytest.mark.parametrize("dims,B", [((20, 17), 5), ((37,), 3)])
def test_batched_slices_match_oracle_per_slice(form, prec, iters, tol, dims, B):
    K, Ms = batch_problem(dims, B)
    N = int(np.prod(dims))
    Mall = np.ascontiguousarray(np.concatenate(Ms, axis=1), np.float32)
    plan = ssm.Plan(K, dims, 0.1, 1.0, form=form, precision=prec, max_iter=iters,
                    check_every=0, batch=B)
    F, info = plan.solve(torch.from_numpy(Mall).cuda())
    F = F.cpu().numpy()
    plan.close()
    assert info["iterations"] == iters
    worst = 0.0
    for b in range(B):
        Mb = Mall[:, b * N:(b + 1) * N].astype(np.float64)
        if form == "admm":
            ref = A.admm(K, Mb, dims, 0.1, 1.0, iters=iters)["y"]
        else:
            ref = L.ladmm(K, Mb, dims, 0.1, 1.0, iters=iters, check_every=0,
                          dense=form == "dense",
                          rank=info["rank"] if form == "lowrank" else None)["z"]
        err = rel(F[:, b * N:(b + 1) * N], ref)
        worst = max(worst, err)
        assert err <= tol, (b, err)
    print(f"{form}_{prec} {dims} x {B}: worst slice rel err {worst:.3e}")


def test_batched_slices_with_a_mask():
    dims, B = (18, 15), 4
    K, Ms = batch_problem(dims, B, seed=9)
    N = int(np.prod(dims))
    Mall = np.ascontiguousarray(np.concatenate(Ms, axis=1), np.float32)
    mask = np.random.default_rng(3).random(N * B) > 0.3
    plan = ssm.Plan(K, dims, 0.1, 1.0, max_iter=40, check_every=0, batch=B)
    plan.set_mask(mask)
    F = plan.solve(torch.from_numpy(Mall).cuda())[0].cpu().numpy()
    plan.close()
    for b in range(B):
        sl = slice(b * N, (b + 1) * N)
        ref = L.ladmm(K, Mall[:, sl].astype(np.float64), dims, 0.1, 1.0, iters=40,
                      check_every=0, mask=mask[sl])["z"]
        assert rel(F[:, sl], ref) <= 1e-5
    assert np.all(F[:, ~mask] == 0.0)


def test_batched_plan_rejects_3d_slices():
    K, _ = batch_problem((4, 4), 1)
    with pytest.raises(ssm.SsmError) as e:
        ssm.Plan(K, (4, 4, 4), 0.1, 1.0, batch=2)
    assert e.value.status == ssm.SSM_EINVAL
