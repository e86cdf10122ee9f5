"""Failure detection without a GPU fault (needs a GB300).

Every mbarrier wait in the solver's kernels is bounded and reports SSM_ETIMEOUT through
the device error word. ssm_selftest_wait_timeout runs a kernel whose wait can never
succeed (nothing arrives at its barrier) with a short poll limit: the status must come
back as SSM_ETIMEOUT, and the device must stay usable (a solve right after matches the
oracle).
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


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    lib = ssm.load_library()
    stream = torch.cuda.Stream()
    for polls in (1, 1000):
        st = lib.ssm_selftest_wait_timeout(polls, ssm._stream_handle(stream))
        assert st == ssm.SSM_ETIMEOUT
        assert b"timed out" in lib.ssm_last_error()
    w = synth.WORKLOADS["dr2d_tiny"]
    K, M, _ = synth.make_problem("dr2d_tiny", dims=(16, 12))
    plan = ssm.Plan(K, (16, 12), w.lam, w.beta, max_iter=30, check_every=10, tol_primal=1e-12)
    F, info = plan.solve(torch.from_numpy(M).cuda())
    plan.close()
    assert info["status"] == ssm.SSM_ENOTCONVERGED and info["iterations"] == 30
    ref = L.ladmm(K, M.astype(np.float64), (16, 12), w.lam, w.beta, iters=30, check_every=0)
    err = np.linalg.norm(F.cpu().numpy() - ref["z"]) / np.linalg.norm(ref["z"])
    assert err <= 1e-5
