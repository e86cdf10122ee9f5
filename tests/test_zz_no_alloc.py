"""ssm_objective_noalloc: the objective for callers that cannot allocate device memory.

Such callers (a pipeline that forbids allocation once running, a process whose device
memory is held by another allocator, work on a busy device where cudaMalloc would
synchronise it) get the same number as the planned ssm_objective, computed with the
library's fixed scratch only. This file runs last so that a failure here does not hide
the rest of the suite; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ladmm as oracle_ladmm
from paper_2401_12890_gb300 import ssm, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return ssm.load_library()


def noalloc_objective(lib, K32, Md, Fd, dims, lam, pairs=2):
    d = (ctypes.c_int64 * 3)(*(list(dims) + [1] * (3 - len(dims))))
    J = ctypes.c_double()
    st = lib.ssm_objective_noalloc(
        ctypes.c_void_p(K32.data_ptr()), K32.shape[0], K32.shape[1],
        ctypes.c_void_p(Md.data_ptr()), Md.stride(0), ctypes.c_void_p(Fd.data_ptr()),
        Fd.stride(0), len(dims), d, lam, pairs, ctypes.byref(J),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, J.value


def test_matches_planned_objective_on_two_calls(lib):
    w = synth.WORKLOADS["dr2d_tiny"]
    K, M, _ = synth.make_problem("dr2d_tiny")
    plan = ssm.Plan(K, w.dims, w.lam, w.beta, form="lowrank", max_iter=40, check_every=0)
    Md = torch.from_numpy(M).cuda()
    Fd, _ = plan.solve(Md)
    J_plan = plan.objective(Md, Fd, use_full_k=True)
    plan.close()
    K32 = torch.from_numpy(K.astype(np.float32)).cuda()
    for _ in range(2):                      # the shared scratch keeps the last call's data
        st, J = noalloc_objective(lib, K32, Md, Fd, w.dims, w.lam)
        assert st == ssm.SSM_OK
        assert J == pytest.approx(J_plan, rel=2e-6)
    # a different grid shape and stencil convention on the same scratch
    F2 = torch.rand((K.shape[1], 7 * 9), device="cuda")
    M2 = torch.rand((K.shape[0], 7 * 9), device="cuda")
    plan2 = ssm.Plan(K, (7, 9), 0.3, 1.0, form="dense", stencil_pairs=1, max_iter=1)
    J2_plan = plan2.objective(M2, F2)
    plan2.close()
    st, J2 = noalloc_objective(lib, K32, M2, F2, (7, 9), 0.3, pairs=1)
    assert st == ssm.SSM_OK and J2 == pytest.approx(J2_plan, rel=2e-6)


def _oracle_objective(K32, Md, Fd, dims, lam, pairs):
    """Eq. 7 / Eq. 8 in FP64 on the host from the same FP32 buffers (the oracle)."""
    K = K32.cpu().double().numpy()
    M = Md.cpu().double().numpy()
    F = Fd.cpu().double().numpy()
    return oracle_ladmm.objective(K, M, F, dims, lam, pairs)


@pytest.mark.parametrize("dims,pairs", [((5, 4, 3), 2), ((5, 4, 3), 1), ((6, 7), 2),
                                        ((11,), 2)])
def test_matches_the_oracle_on_1d_2d_3d_grids(lib, dims, pairs):
    rng = np.random.default_rng(7 + len(dims) + pairs)
    P, Q = 9, 13
    N = int(np.prod(dims))
    K32 = torch.from_numpy(rng.uniform(0.0, 1.0, (P, Q)).astype(np.float32)).cuda()
    Md = torch.from_numpy(rng.uniform(0.0, 2.0, (P, N)).astype(np.float32)).cuda()
    Fd = torch.from_numpy(rng.uniform(0.0, 1.0, (Q, N)).astype(np.float32)).cuda()
    J_ref = _oracle_objective(K32, Md, Fd, dims, 0.37, pairs)
    for _ in range(2):                      # a second call on the same shared scratch
        st, J = noalloc_objective(lib, K32, Md, Fd, dims, 0.37, pairs)
        assert st == ssm.SSM_OK
        # FP32 product K F with FP32 accumulation over Q = 13 terms, FP64 sums
        assert J == pytest.approx(J_ref, rel=1e-6)


def test_rejects_dimensions_that_do_not_fit_an_int(lib):
    K32 = torch.ones((2, 2), device="cuda")
    for dims in ((2 ** 32 + 5,), (2 ** 32 + 5, 1), (1, 2 ** 33 + 1), (4096, 4096, 4096)):
        st, _ = noalloc_objective(lib, K32, K32, K32, dims, 0.1)
        assert st == ssm.SSM_EINVAL


def test_rejects_grids_beyond_the_fixed_scratch(lib):
    K32 = torch.ones((2, 2), device="cuda")
    big = (2049, 2048)                       # 4,196,352 voxels > 4,194,304
    st, _ = noalloc_objective(lib, K32, K32, K32, big, 0.1)
    assert st == ssm.SSM_EINVAL
    assert b"4194304" in lib.ssm_last_error()
