"""The C-ABI library builds, loads and exports what include/ssm.h declares (no GPU).

Only calls that never reach the GPU are made here: parameter defaults, argument
validation (rejected before any CUDA call), status strings and NULL handling.
"""
import ctypes
import os
import subprocess

import pytest

import __graft_entry__
from paper_2401_12890_gb300 import ssm


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ssm.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = ssm.declared_symbols()
    assert {"ssm_plan", "ssm_solve", "ssm_destroy", "ssm_solve_host", "ssm_objective"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", ssm.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in names:
        assert name in exported, f"{name} not exported with C linkage"


def test_struct_layout_matches_header(lib, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ssm.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   ' sizeof(ssm_params), sizeof(ssm_info), offsetof(ssm_params, tol_change),'
                   ' offsetof(ssm_info, plan_ms), sizeof(ssm_server_config),'
                   ' offsetof(ssm_server_config, reserved_small), sizeof(ssm_request_info),'
                   ' offsetof(ssm_request_info, plan_reused), sizeof(ssm_server_stats),'
                   ' offsetof(ssm_server_stats, pending), sizeof(ssm_launch_info),'
                   ' offsetof(ssm_launch_info, tc_fused), offsetof(ssm_info, power_converged),'
                   ' offsetof(ssm_server_config, group_small), offsetof(ssm_request_info, group_size));'
                   ' return 0;}\n')
    exe = tmp_path / "sz"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(ssm.SsmParams), ctypes.sizeof(ssm.SsmInfo),
                    ssm.SsmParams.tol_change.offset, ssm.SsmInfo.plan_ms.offset,
                    ctypes.sizeof(ssm.SsmServerConfig), ssm.SsmServerConfig.reserved_small.offset,
                    ctypes.sizeof(ssm.SsmRequestInfo), ssm.SsmRequestInfo.plan_reused.offset,
                    ctypes.sizeof(ssm.SsmServerStats), ssm.SsmServerStats.pending.offset,
                    ctypes.sizeof(ssm.SsmLaunchInfo), ssm.SsmLaunchInfo.tc_fused.offset,
                    ssm.SsmInfo.power_converged.offset, ssm.SsmServerConfig.group_small.offset,
                    ssm.SsmRequestInfo.group_size.offset]


def test_defaults_and_status_strings(lib):
    p = ssm.SsmParams()
    assert lib.ssm_default_params(ctypes.byref(p)) == ssm.SSM_OK
    assert p.ndim == 2 and p.beta == 1.0 and p.stencil_pairs == 2 and p.max_iter == 300
    assert p.rank_tol == pytest.approx(5e-5)
    for code in range(9):
        assert lib.ssm_status_string(code)
    assert lib.ssm_status_string(99) == b"unknown status"
    assert lib.ssm_destroy(None) == ssm.SSM_OK


@pytest.mark.parametrize("field,value", [
    ("beta", 0.0), ("beta", -1.0), ("lam", -1.0), ("ndim", 0), ("ndim", 4), ("P", 0),
    ("Q", 0), ("form", 5), ("precision", 9), ("stencil_pairs", 3), ("max_iter", -1),
    ("rank", -2),
])
def test_invalid_params_rejected_before_any_gpu_call(lib, field, value):
    p = ssm.SsmParams()
    lib.ssm_default_params(ctypes.byref(p))
    p.P, p.Q = 4, 5
    p.dims[0], p.dims[1] = 3, 3
    setattr(p, field, value)
    K = (ctypes.c_double * 20)()
    h = ctypes.c_void_p()
    st = lib.ssm_plan(ctypes.byref(h), ctypes.byref(p), ctypes.cast(K, ctypes.c_void_p), 0, None)
    assert st == ssm.SSM_EINVAL
    assert h.value is None
    assert lib.ssm_last_error()


def test_null_arguments_rejected(lib):
    p = ssm.SsmParams()
    lib.ssm_default_params(ctypes.byref(p))
    p.P, p.Q = 2, 2
    h = ctypes.c_void_p()
    assert lib.ssm_plan(ctypes.byref(h), ctypes.byref(p), None, 0, None) == ssm.SSM_EINVAL
    assert lib.ssm_plan(None, ctypes.byref(p), None, 0, None) == ssm.SSM_EINVAL
    assert lib.ssm_solve(None, None, 0, None, 0, None, None) == ssm.SSM_EINVAL
    J = ctypes.c_double()
    assert lib.ssm_objective(None, None, 0, None, 0, 0, ctypes.byref(J), None) == ssm.SSM_EINVAL


def test_selftest_rejects_bad_poll_counts_before_any_gpu_call(lib):
    assert lib.ssm_selftest_wait_timeout(0, None) == ssm.SSM_EINVAL
    assert lib.ssm_selftest_wait_timeout((1 << 20) + 1, None) == ssm.SSM_EINVAL
