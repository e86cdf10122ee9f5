"""Groups of independent problems in one launch per iteration (ssm_group_*), against the
FP64 oracle. Needs a GB300.

Each problem of a group runs Algorithm 2's low-rank iteration on its own grid with its
own dictionary, lambda, beta and stopping rule. Bars: the FP32 one, ||z_gpu - z_oracle||
<= 1e-5 ||z_oracle|| after a fixed count from the zero start, per problem; the stopping
rule stops each problem at the oracle's iteration; a problem's result is bitwise the same
in any group (alone, with others, with others of higher rank); and within 1e-6 of
ssm_solve on the same plan (another kernel, another summation order).
"""
import numpy as np
import pytest
import torch

from oracle import ladmm as L
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


# (dims, P, Q, lambda, beta, seed): 2D, 1D, 3D, ragged tiles, both Gram sides
SHAPES = [((32, 32), 30, 225, 0.01, 0.05, 1), ((19, 23), 12, 40, 0.05, 0.8, 2),
          ((301,), 9, 30, 0.02, 0.5, 3), ((9, 7, 5), 20, 16, 0.05, 0.6, 4),
          ((45, 13), 40, 25, 0.03, 0.4, 5), ((7, 6), 6, 50, 0.1, 1.2, 6)]


def make(shape, rank=0, **kw):
    dims, P, Q, lam, beta, seed = shape
    if shape[0] == (32, 32):
        K, M, _ = synth.make_problem("dr2d_tiny")
    else:
        K, M, _ = synth.random_problem(P, Q, dims, seed=seed, snr=60.0)
    plan = ssm.Plan(K, dims, lam, beta, form="lowrank", precision="fp32", rank=rank, **kw)
    return plan, K, np.asarray(M, np.float64)


def test_each_problem_matches_the_oracle():
    made = [make(sh, rank=(8 if i == 3 else 0), max_iter=60 + 20 * i, check_every=0)
            for i, sh in enumerate(SHAPES)]
    plans = [m[0] for m in made]
    grp = ssm.Group(plans)
    Fs, infos, st = grp.solve([dev(m[2]) for m in made])
    assert st == ssm.SSM_OK
    for (plan, K, M), sh, F, info in zip(made, SHAPES, Fs, infos):
        dims, _, _, lam, beta, _ = sh
        ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), dims, lam, beta,
                      rank=plan.info()["rank"], iters=plan.params.max_iter, check_every=0)
        assert info["iterations"] == plan.params.max_iter
        assert info["rank"] == ref["r"]
        err = rel(F.cpu().numpy().astype(np.float64), ref["z"])
        print(f"{dims}: r {ref['r']} iters {info['iterations']} rel err {err:.3e}")
        assert err <= RTOL
    grp.close()
    for p in plans:
        p.close()


def test_stopping_rule_per_problem():
    tols = [3e-3, 1e-3, 5e-3, 2e-3]
    made = [make(sh, max_iter=3000, check_every=ce, tol_primal=t, tol_change=t)
            for sh, t, ce in zip(SHAPES[:4], tols, [10, 7, 10, 5])]
    grp = ssm.Group([m[0] for m in made])
    Fs, infos, st = grp.solve([dev(m[2]) for m in made])
    assert st == ssm.SSM_OK
    for (plan, K, M), sh, F, info, t in zip(made, SHAPES, Fs, infos, tols):
        dims, _, _, lam, beta, _ = sh
        ref = L.ladmm(K, M.astype(np.float32).astype(np.float64), dims, lam, beta,
                      iters=3000, check_every=plan.params.check_every, tol_primal=t,
                      tol_change=t, return_history=True)
        assert info["status"] == ssm.SSM_OK
        assert info["iterations"] == ref["iters"], (dims, info["iterations"], ref["iters"])
        k, rp, rc = ref["history"][-1]
        assert info["res_primal"] == pytest.approx(rp, rel=1e-3)
        assert rel(F.cpu().numpy().astype(np.float64), ref["z"]) <= RTOL
    # different stopping points: the group ran them to different counts
    assert len({i["iterations"] for i in infos}) > 1
    grp.close()


def test_budget_runs_out():
    plan, K, M = make(SHAPES[1], max_iter=15, check_every=5, tol_primal=1e-12)
    grp = ssm.Group([plan])
    _, infos, st = grp.solve([dev(M)])
    assert st == ssm.SSM_ENOTCONVERGED
    assert infos[0]["status"] == ssm.SSM_ENOTCONVERGED and infos[0]["iterations"] == 15
    grp.close()


def test_a_problem_gives_the_same_bits_in_any_group():
    a = make(SHAPES[1], max_iter=80, check_every=10, tol_primal=1e-9)
    b = make(SHAPES[0], max_iter=50, check_every=0)
    c = make(SHAPES[4], max_iter=120, check_every=0)   # a higher rank: R grows
    alone = ssm.Group([a[0]])
    Fa, ia, _ = alone.solve([dev(a[2])])
    alone.close()
    mixed = ssm.Group([b[0], a[0], c[0]])
    Fm, im, _ = mixed.solve([dev(b[2]), dev(a[2]), dev(c[2])])
    mixed.close()
    assert torch.equal(Fa[0], Fm[1])
    assert ia[0]["res_primal"] == im[1]["res_primal"]
    # and within rounding of the plan's own solve
    F1, _ = a[0].solve(dev(a[2]))
    assert rel(F1.cpu().numpy(), Fa[0].cpu().numpy()) <= 1e-6


def test_one_launch_per_iteration():
    made = [make(sh, max_iter=40, check_every=0) for sh in SHAPES[:5]]
    grp = ssm.Group([m[0] for m in made])
    Ms = [dev(m[2]) for m in made]
    grp.solve(Ms)
    n0 = ssm.launch_count()
    grp.solve(Ms)
    launches = ssm.launch_count() - n0
    # 5 projections + 40 iterations + 1 residual finish (every problem's last iteration)
    assert launches == 5 + 40 + 1, launches
    grp.close()


def test_unsupported_plans_are_refused():
    K, M, _ = synth.random_problem(12, 40, (8, 8), seed=1)
    lr = ssm.Plan(K, (8, 8), 0.05, 0.8, form="lowrank")
    for kw in (dict(form="dense"), dict(form="lowrank", precision="tf32x3")):
        other = ssm.Plan(K, (8, 8), 0.05, 0.8, **kw)
        with pytest.raises(ssm.SsmError) as e:
            ssm.Group([lr, other])
        assert e.value.status == ssm.SSM_EUNSUPPORTED
        other.close()
    masked = ssm.Plan(K, (8, 8), 0.05, 0.8, form="lowrank")
    masked.set_mask(np.ones(64))
    with pytest.raises(ssm.SsmError) as e:
        ssm.Group([masked])
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    Kb = synth.random_problem(60, 40, (1, 1), 3, full_rank=True)[0]   # rank 40 > 32
    big = ssm.Plan(Kb, (8, 8), 0.05, 0.8, form="lowrank")
    with pytest.raises(ssm.SsmError) as e:
        ssm.Group([big])
    assert e.value.status == ssm.SSM_EUNSUPPORTED
    with pytest.raises(ssm.SsmError) as e:
        ssm.Group([])
    assert e.value.status == ssm.SSM_EINVAL
