"""Algorithm 1 (the three-split ADMM of Sec. II-C) on the GPU vs the FP64 oracle
(`oracle/admm.py`, whose z-step is a sparse LU solve: a different route from the
GPU's DCT diagonalisation). Needs a GB300.

Bar: the returned y (the nonnegative split) matches the oracle's y after a fixed
iteration count from the zero start with ||y_gpu - y_oracle||_F <= 1e-5 ||y_oracle||_F,
the FP32 parity bar of the other FP32 forms.
"""
import numpy as np
import pytest
import torch

from oracle import admm as A
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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gpu_admm(K, M, dims, lam, beta, iters, **kw):
    plan = ssm.Plan(K, dims, lam, beta, form="admm", max_iter=iters, check_every=0, **kw)
    F, info = plan.solve(torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda())
    out = F.cpu().numpy()
    plan.close()
    return out, info


CASES = [
    # (dims, P, Q, lambda, beta, stencil_pairs)
    ((16, 12), 30, 20, 0.05, 1.0, 2),
    ((7, 6, 5), 12, 9, 0.1, 2.0, 2),          # 3D, P > Q
    ((37,), 8, 15, 0.2, 0.5, 2),              # 1D
    ((1, 1), 5, 9, 0.3, 1.0, 2),              # one voxel: D^T D = 0
    ((33, 1), 5, 9, 0.0, 1.0, 2),             # lambda = 0
    ((128, 3), 10, 30, 0.02, 0.7, 2),         # an axis of 128: two k blocks
    ((200, 2), 6, 10, 0.05, 1.0, 2),          # an axis of 200: four k blocks
    ((9, 11), 10, 14, 0.1, 1.0, 1),           # one term per neighbour pair
]


@pytest.mark.parametrize("dims,P,Q,lam,beta,pairs", CASES)
def test_admm_matches_oracle(dims, P, Q, lam, beta, pairs):
    K, M, _ = synth.random_problem(P, Q, dims, seed=P * 31 + Q, snr=50.0)
    iters = 60
    F, info = gpu_admm(K, M, dims, lam, beta, iters, stencil_pairs=pairs)
    ref = A.admm(K, M.astype(np.float32).astype(np.float64), dims, lam, beta, iters=iters,
                 pairs=pairs)
    assert info["iterations"] == iters
    assert F.min() >= 0.0
    err = rel(F, ref["y"])
    print(f"{dims}: rel err {err:.3e}")
    assert err <= RTOL


def test_admm_moderate_grid_and_objective():
    """A 64 x 48 grid with the diffusion-relaxation dictionary: y after 40 iterations;
    then both algorithms (Algorithm 1 and the full-rank Algorithm 2, which solve the same
    Eq. 7) approach the same objective."""
    w = synth.WORKLOADS["dr2d_tiny"]
    K, M, _ = synth.make_problem("dr2d_tiny", dims=(64, 48))
    F, _ = gpu_admm(K, M, (64, 48), w.lam, w.beta, 40)
    ref = A.admm(K, M.astype(np.float64), (64, 48), w.lam, w.beta, iters=40)
    assert rel(F, ref["y"]) <= RTOL
    Md = torch.from_numpy(M).cuda()
    J = {}
    for form in ("admm", "dense"):
        for it in (4000, 20000):
            p = ssm.Plan(K, (64, 48), w.lam, w.beta, form=form, max_iter=it, check_every=0)
            Fx, _ = p.solve(Md)
            J[form, it] = p.objective(Md, Fx)
            p.close()
    print({k: f"{v:.8g}" for k, v in J.items()})
    gap4 = abs(J["admm", 4000] - J["dense", 4000])
    gap20 = abs(J["admm", 20000] - J["dense", 20000])
    assert gap20 < gap4
    assert J["admm", 20000] == pytest.approx(J["dense", 20000], rel=1e-4)


def test_admm_stopping_rule_and_graphs():
    K, M, _ = synth.random_problem(20, 16, (24, 20), seed=3, snr=50.0)
    kw = dict(form="admm", max_iter=3000, check_every=10, tol_primal=1e-4, tol_change=1e-4)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
    p0 = ssm.Plan(K, (24, 20), 0.05, 1.0, **kw)
    F0, i0 = p0.solve(Md)
    p1 = ssm.Plan(K, (24, 20), 0.05, 1.0, **kw)
    p1.set_graphs(True)
    p1.solve(Md)
    F1, i1 = p1.solve(Md)
    p0.close()
    p1.close()
    assert 0 < i0["iterations"] < 3000 and i0["iterations"] % 10 == 0
    assert i0["res_primal"] <= 1e-4 and i0["res_change"] <= 1e-4
    assert i1["iterations"] == i0["iterations"]
    assert torch.equal(F0, F1)


def test_admm_set_beta_equals_a_fresh_plan():
    K, M, _ = synth.random_problem(12, 20, (18, 14), seed=9, snr=50.0)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
    fresh = ssm.Plan(K, (18, 14), 0.05, 2.5, form="admm", max_iter=50, check_every=0)
    F0 = fresh.solve(Md)[0]
    fresh.close()
    plan = ssm.Plan(K, (18, 14), 0.05, 1.0, form="admm", max_iter=50, check_every=0)
    plan.solve(Md)
    plan.set_beta(2.5)
    F1 = plan.solve(Md)[0]
    plan.close()
    assert torch.equal(F0, F1)


def test_admm_rejects_bf16_and_long_axes():
    K, M, _ = synth.random_problem(6, 8, (300, 2), seed=1)
    with pytest.raises(ssm.SsmError) as e:
        ssm.Plan(K, (300, 2), 0.1, 1.0, form="admm")
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    with pytest.raises(ssm.SsmError) as e:
        ssm.Plan(K, (30, 2), 0.1, 1.0, form="admm", precision="bf16x3")
    assert e.value.status == ssm.SSM_EUNSUPPORTED
