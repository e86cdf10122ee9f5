"""Continuing a solve (ssm_solve_resume) repeats the longer solve exactly. Needs a GB300.

Algorithm 2's state is (z, d) (and the forms' internal operands: the low-rank forms'
partial u, the tensor-core form's split w), all resident on the device between calls. A
solve of k1 iterations followed by a resumed solve of k2 more must give the iterate of one
solve of k1 + k2 iterations, bit for bit, for every form; the residual tests in between
do not change the iterates. The oracle's own continuation is pinned on the CPU
(tests/test_oracle_ladmm.py).
"""
import numpy as np
import pytest
import torch

from paper_2401_12890_gb300 import ssm, synth

pytestmark = pytest.mark.gpu

FORMS = [("lowrank", "fp32"), ("lowrank", "tf32x3"), ("dense", "fp32"), ("dense", "bf16x3"),
         ("admm", "fp32")]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    yield


@pytest.mark.parametrize("form,prec", FORMS, ids=[f"{a}_{b}" for a, b in FORMS])
@pytest.mark.parametrize("check_every", [0, 7])
def test_resume_repeats_the_longer_solve(form, prec, check_every):
    dims = (37, 29)
    K, M, _ = synth.random_problem(20, 70, dims, seed=11, snr=50.0)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
    k1, k2 = 23, 31
    kw = dict(form=form, precision=prec, check_every=check_every)
    full = ssm.Plan(K, dims, 0.05, 0.8, max_iter=k1 + k2, **kw)
    F_full, info_full = full.solve(Md)
    full.close()
    part = ssm.Plan(K, dims, 0.05, 0.8, max_iter=k1, **kw)
    part.solve(Md)
    part.set_max_iter(k2)
    F_res, info_res = part.resume(Md)
    # a second continuation from there is the longer solve again
    part.set_max_iter(5)
    F_more, _ = part.resume(Md)
    part.close()
    longer = ssm.Plan(K, dims, 0.05, 0.8, max_iter=k1 + k2 + 5, **kw)
    F_longer, _ = longer.solve(Md)
    longer.close()
    assert info_res["iterations"] == k2
    assert torch.equal(F_res, F_full)
    assert torch.equal(F_more, F_longer)


def test_resume_needs_a_state():
    dims = (9, 8)
    K, M, _ = synth.random_problem(6, 10, dims, seed=2)
    Md = torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda()
    plan = ssm.Plan(K, dims, 0.05, 1.0, max_iter=5)
    with pytest.raises(ssm.SsmError) as e:
        plan.resume(Md)
    assert e.value.status == ssm.SSM_EINVAL
    plan.solve(Md)
    plan.resume(Md)                          # fine after a solve
    plan.set_beta(0.5)                       # another iteration: the state is dropped
    with pytest.raises(ssm.SsmError) as e:
        plan.resume(Md)
    assert e.value.status == ssm.SSM_EINVAL
    plan.close()
