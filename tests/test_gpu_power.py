"""The FP64 device iterations for lambda_max of the Hessian of Eq. 7 (ssm_plan): power
iteration on the Gram factor, inverse iteration on the grid axes.

H = I_N (x) K^T K + lambda D^T D (x) I_Q bounds the step of a gradient method on Eq. 7;
xi_p of Eq. 32 is to exceed 0.75 lambda ||D^T D|| (the convergence condition cited in
Sec. III-C). Checked through the C ABI (ssm_plan_info) against
  * the oracle's power iteration on the whole Q x N operator (oracle.pg.hessian_norm) on
    small problems, and
  * the closed form sigma_1^2 + lambda ||D^T D|| (exact: H is a Kronecker sum), with
    sigma_1 from numpy's SVD and ||D^T D|| from the path-Laplacian spectrum,
on 1D, 2D and 3D grids, both Gram sides (P < Q and P > Q), both stencil conventions, a
batched plan (independent slices) and the full-size workloads' plans.
"""
import numpy as np
import pytest

from oracle import grid, pg
from paper_2401_12890_gb300 import ssm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return ssm.load_library()


def closed_form(K, dims, lam, pairs):
    s1 = float(np.linalg.svd(np.asarray(K, np.float64), compute_uv=False)[0])
    return s1 * s1, grid.dtd_norm(dims, pairs), s1 * s1 + lam * grid.dtd_norm(dims, pairs)


SMALL = [((7, 5), 6, 9, 0.3, 2, "lowrank"), ((11,), 9, 4, 1.2, 2, "dense"),
         ((4, 3, 5), 5, 8, 0.05, 1, "lowrank"), ((6, 6), 12, 7, 2.0, 2, "dense")]


@pytest.mark.parametrize("dims,P,Q,lam,pairs,form", SMALL)
def test_power_iteration_matches_oracle_and_closed_form(dims, P, Q, lam, pairs, form):
    K, _, _ = synth.random_problem(P, Q, dims, seed=P + 3 * Q)
    plan = ssm.Plan(K, dims, lam, 1.0, form=form, stencil_pairs=pairs, max_iter=1)
    info = plan.info()
    plan.close()
    kk, dtd, hess = closed_form(K, dims, lam, pairs)
    assert info["power_converged"] == 1
    assert info["kk_norm"] == pytest.approx(kk, rel=1e-10)
    assert info["dtd_norm_power"] == pytest.approx(dtd, rel=1e-10)
    assert info["hess_norm"] == pytest.approx(hess, rel=1e-10)
    ref = pg.hessian_norm(K, dims, lam, pairs, iters=20000)
    assert info["hess_norm"] == pytest.approx(ref, rel=1e-10)
    # the step-size condition of the linearised z-step holds for the rule of Eq. 32
    assert info["xi_p"] > 0.75 * lam * info["dtd_norm_power"]


def test_batched_slices_have_the_slice_operator():
    K, _, _ = synth.random_problem(5, 7, (6, 4), seed=3)
    plan = ssm.Plan(K, (6, 4), 0.4, 1.0, form="lowrank", max_iter=1, batch=3)
    info = plan.info()
    plan.close()
    _, _, hess = closed_form(K, (6, 4), 0.4, 2)
    assert info["power_converged"] == 1
    assert info["hess_norm"] == pytest.approx(hess, rel=1e-10)


@pytest.mark.parametrize("name", ["dr2d_slice", "mrf2d", "rr3d_t1t2"])
def test_full_size_plans(name):
    w = synth.WORKLOADS[name]
    K = synth.dictionary_for(name)
    plan = ssm.Plan(K, w.dims, w.lam, w.beta, form="lowrank", max_iter=1)
    info = plan.info()
    plan.close()
    kk, dtd, hess = closed_form(K, w.dims, w.lam, 2)
    assert info["power_converged"] == 1, info
    assert info["kk_norm"] == pytest.approx(kk, rel=1e-10)
    # the axes run inverse iteration (about a factor 4 per step): the stopping rule
    # leaves well under 1e-10 relative
    assert info["dtd_norm_power"] == pytest.approx(dtd, rel=1e-10)
    assert info["power_iters"] <= 4096


@pytest.mark.parametrize("dims", [(6000,), (3000, 3), (2, 2), (2,)])
def test_long_and_short_axes(dims):
    """Inverse iteration on axes far longer than a power iteration could resolve in its
    budget (plain power iteration contracts like 1 - (pi/n)^2 per step), and the
    shortest ones."""
    K, _, _ = synth.random_problem(6, 9, (1, 1), seed=4)
    plan = ssm.Plan(K, dims, 0.3, 1.0, form="lowrank", max_iter=1)
    info = plan.info()
    plan.close()
    kk, dtd, hess = closed_form(K, dims, 0.3, 2)
    assert info["power_converged"] == 1, info
    assert info["dtd_norm_power"] == pytest.approx(dtd, rel=1e-10)
    assert info["hess_norm"] == pytest.approx(hess, rel=1e-10)
    assert info["hess_norm"] == pytest.approx(hess, rel=1e-10)
