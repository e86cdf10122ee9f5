"""Voxel masks on the GPU (ssm_plan_set_mask) vs the FP64 oracle with the same mask.
Needs a GB300.

The problem lives on the voxels inside the object, coupled by the pairs of the grid
graph the mask induces (the paper's maskless form); F is exactly 0 outside. Bars as for
the unmasked forms: FP32 forms ||F - z_oracle||_F <= 1e-5 ||z_oracle||_F after a fixed
iteration count, BF16x3 1e-4 after 20 iterations.
"""
import numpy as np
import pytest
import torch

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


def random_mask(dims, seed, holes=0.15):
    """An ellipsoid with random holes: boundaries in every direction, isolated voxels."""
    rng = np.random.default_rng(seed)
    axes = [(np.arange(n) + 0.5) / n - 0.5 for n in dims]
    grids = np.meshgrid(*reversed(axes), indexing="ij")       # [z][y][x] order
    r2 = sum((g / 0.45) ** 2 for g in grids)
    m = (r2 <= 1.0) & (rng.random(r2.shape) > holes)
    return m.ravel()


def solve(K, M, dims, lam, beta, mask, iters, **kw):
    plan = ssm.Plan(K, dims, lam, beta, max_iter=iters, check_every=0, **kw)
    plan.set_mask(mask)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
    F, info = plan.solve(Md)
    J = plan.objective(Md, F)
    out = F.cpu().numpy()
    plan.close()
    return out, info, J


FORMS = [("lowrank", "fp32", 40, 1e-5), ("dense", "fp32", 40, 1e-5),
         ("dense", "bf16x3", 20, 1e-4)]


@pytest.mark.parametrize("form,prec,iters,tol", FORMS, ids=[f[0] + "_" + f[1] for f in FORMS])
@pytest.mark.parametrize("dims,seed", [((30, 26), 1), ((12, 10, 8), 2), ((200, 3), 3)])
def test_masked_solve_matches_oracle(form, prec, iters, tol, dims, seed):
    K, M, _ = synth.random_problem(16, 40, dims, seed=seed, snr=50.0)
    mask = random_mask(dims, seed)
    F, info, J = solve(K, M, dims, 0.1, 1.0, mask, iters, form=form, precision=prec)
    M64 = M.astype(np.float32).astype(np.float64)
    ref = L.ladmm(K, M64, dims, 0.1, 1.0, iters=iters, check_every=0, dense=form == "dense",
                  rank=info["rank"] if form == "lowrank" else None, mask=mask)
    assert np.all(F[:, ~mask] == 0.0)
    err = rel(F, ref["z"])
    print(f"{form}_{prec} {dims}: {int(mask.sum())}/{mask.size} inside, rel err {err:.3e}")
    assert err <= tol
    Kf = K if form == "dense" else L.truncated_dictionary(K, info["rank"])
    J_ref = L.objective(Kf, M64, F.astype(np.float64), dims, 0.1, mask=mask)
    assert J == pytest.approx(J_ref, rel=2e-6)


@pytest.mark.parametrize("form", ["lowrank", "dense"])
def test_masked_1d_spectrum_workload(form):
    """The multi-echo T2 workload: a 1D spectrum of 300 T2 values per voxel, 32 echoes,
    an elliptical object of 4472 voxels in an 84 x 72 grid."""
    w = synth.WORKLOADS["mse_t2"]
    K, M, _ = synth.make_problem("mse_t2")
    mask = synth.mask_for("mse_t2")
    F, info, _ = solve(K, M, w.dims, w.lam, w.beta, mask, 60, form=form)
    ref = L.ladmm(K, M.astype(np.float64), w.dims, w.lam, w.beta, iters=60, check_every=0,
                  dense=form == "dense", mask=mask)
    err = rel(F, ref["z"])
    print(f"mse_t2 {form}: rank {info['rank']}, rel err {err:.3e}")
    assert err <= 1e-5
    assert np.all(F[:, ~mask] == 0.0)


def test_mask_removed_gives_the_unmasked_solve_and_stopping_rule():
    K, M, _ = synth.random_problem(12, 30, (24, 20), seed=4, snr=50.0)
    mask = random_mask((24, 20), 4)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
    plan = ssm.Plan(K, (24, 20), 0.1, 1.0, max_iter=2000, check_every=10, tol_primal=1e-3,
                    tol_change=1e-3)
    F0, i0 = plan.solve(Md)
    plan.set_mask(mask)
    Fm, im = plan.solve(Md)
    plan.set_mask(None)
    F1, i1 = plan.solve(Md)
    plan.close()
    assert torch.equal(F0, F1) and i0["iterations"] == i1["iterations"]
    ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), (24, 20), 0.1, 1.0,
                  iters=2000, check_every=10, tol_primal=1e-3, tol_change=1e-3, mask=mask)
    assert im["iterations"] == ref["iters"]
    assert rel(Fm.cpu().numpy(), ref["z"]) <= 1e-5


def test_admm_rejects_a_mask():
    K, M, _ = synth.random_problem(8, 10, (12, 10), seed=1)
    plan = ssm.Plan(K, (12, 10), 0.1, 1.0, form="admm")
    with pytest.raises(ssm.SsmError) as e:
        plan.set_mask(np.ones(120, bool))
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    plan.close()
