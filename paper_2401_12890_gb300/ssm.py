"""Thin ctypes binding of the C ABI in include/ssm.h (argument marshalling only).

Every step of the solve runs in the CUDA library (libssm.so, built by
paper_2401_12890_gb300.build). Importing this module does not need a GPU; creating a
Plan does, and raises if the library is missing -- there is no CPU fallback.

    plan = Plan(K, dims=(128, 128), lam=1e-2, beta=0.99, form="dense", precision="bf16x3")
    F, info = plan.solve(M_gpu)          # M: torch.cuda float32 tensor P x N
    plan.close()
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SSM_LIBRARY selects another build of the library (e.g. an instrumented one)
LIB_PATH = os.environ.get("SSM_LIBRARY", os.path.join(HERE, "libssm.so"))
HEADER = os.path.join(os.path.dirname(HERE), "include", "ssm.h")

SSM_OK, SSM_EINVAL, SSM_ENOMEM, SSM_ECUDA, SSM_ENAN, SSM_ETIMEOUT, SSM_EUNSUPPORTED, \
    SSM_ENOTCONVERGED, SSM_EPENDING = range(9)
FORMS = {"lowrank": 0, "dense": 1, "admm": 2}
PRECISIONS = {"fp32": 0, "bf16x3": 1, "tf32x3": 2}


class SsmParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("dims", ctypes.c_int64 * 3), ("P", ctypes.c_int),
        ("Q", ctypes.c_int), ("lam", ctypes.c_double), ("beta", ctypes.c_double),
        ("xi_p", ctypes.c_double), ("form", ctypes.c_int), ("rank", ctypes.c_int),
        ("rank_tol", ctypes.c_double), ("precision", ctypes.c_int),
        ("stencil_pairs", ctypes.c_int), ("max_iter", ctypes.c_int),
        ("check_every", ctypes.c_int), ("tol_primal", ctypes.c_double),
        ("tol_change", ctypes.c_double),
    ]


class SsmInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int), ("rank", ctypes.c_int),
        ("gram_side", ctypes.c_int), ("xi_p", ctypes.c_double), ("dtd_norm", ctypes.c_double),
        ("sigma1", ctypes.c_double), ("res_primal", ctypes.c_double),
        ("res_change", ctypes.c_double), ("plan_ms", ctypes.c_double),
        ("hess_norm", ctypes.c_double), ("kk_norm", ctypes.c_double),
        ("dtd_norm_power", ctypes.c_double), ("power_iters", ctypes.c_int),
        ("power_converged", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SsmServerConfig(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int), ("max_active", ctypes.c_int), ("hbm_budget", ctypes.c_int64),
        ("use_graphs", ctypes.c_int), ("cache_plans", ctypes.c_int),
        ("max_bypass", ctypes.c_int), ("simulate_us", ctypes.c_int64),
        ("small_bytes", ctypes.c_int64), ("large_waves", ctypes.c_int),
        ("reserved_small", ctypes.c_int), ("group_small", ctypes.c_int),
    ]


class SsmRequestInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int),
        ("res_primal", ctypes.c_double), ("res_change", ctypes.c_double),
        ("queue_ms", ctypes.c_double), ("plan_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
        ("footprint", ctypes.c_int64), ("order", ctypes.c_int64), ("slot", ctypes.c_int),
        ("plan_reused", ctypes.c_int), ("group_size", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SsmServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
        ("rejected", ctypes.c_int64), ("plans_created", ctypes.c_int64),
        ("plans_reused", ctypes.c_int64), ("plans_evicted", ctypes.c_int64),
        ("bytes_held", ctypes.c_int64), ("peak_bytes_held", ctypes.c_int64),
        ("budget", ctypes.c_int64), ("active", ctypes.c_int), ("pending", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SsmLaunchInfo(ctypes.Structure):
    _fields_ = [
        ("launch_waves", ctypes.c_int), ("gemm_tile_n", ctypes.c_int), ("gemm_grid", ctypes.c_int),
        ("update_grid", ctypes.c_int), ("lowrank_grid", ctypes.c_int), ("sm_count", ctypes.c_int),
        ("tc_fused", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


class SsmError(RuntimeError):
    def __init__(self, status, where):
        lib = load_library()
        msg = lib.ssm_status_string(status).decode()
        detail = lib.ssm_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def declared_symbols(header: str = HEADER):
    """Names of the functions include/ssm.h declares."""
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\*?(ssm_\w+)\s*\(", text, re.M)))


def load_library(path: str = LIB_PATH):
    """Load libssm.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i64, dp, fp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    lib.ssm_default_params.argtypes = [ctypes.POINTER(SsmParams)]
    lib.ssm_plan.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SsmParams), vp, ctypes.c_int, vp]
    lib.ssm_solve.argtypes = [vp, fp, i64, fp, i64, ctypes.POINTER(SsmInfo), vp]
    lib.ssm_solve_host.argtypes = [vp, fp, i64, fp, i64, ctypes.POINTER(SsmInfo), vp]
    lib.ssm_solve_resume.argtypes = [vp, fp, i64, fp, i64, ctypes.POINTER(SsmInfo), vp]
    lib.ssm_plan_set_stopping.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double]
    lib.ssm_objective.argtypes = [vp, fp, i64, fp, i64, ctypes.c_int, dp, vp]
    lib.ssm_plan_factors.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
    lib.ssm_plan_info.argtypes = [vp, ctypes.POINTER(SsmInfo)]
    lib.ssm_destroy.argtypes = [vp]
    lib.ssm_objective_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, i64, vp, i64,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.c_double, ctypes.c_int, dp, vp]
    lib.ssm_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.ssm_profile_read.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.ssm_plan_ex.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SsmParams), vp, ctypes.c_int, vp,
                                ctypes.c_int]
    lib.ssm_plan_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SsmParams), i64, vp,
                                     ctypes.c_int, vp, ctypes.c_int]
    lib.ssm_plan_multi.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SsmParams), ctypes.c_int,
                                   vp, vp, ctypes.c_int, vp]
    lib.ssm_group_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, vp]
    lib.ssm_group_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(SsmInfo), vp]
    lib.ssm_group_device_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.ssm_group_destroy.argtypes = [vp]
    lib.ssm_server_submit_device.argtypes = [vp, ctypes.POINTER(SsmParams), vp, vp, i64, vp, i64,
                                             ctypes.POINTER(ctypes.c_int64)]
    lib.ssm_plan_set_graphs.argtypes = [vp, ctypes.c_int]
    lib.ssm_plan_launch_info.argtypes = [vp, ctypes.POINTER(SsmLaunchInfo)]
    lib.ssm_plan_set_beta.argtypes = [vp, ctypes.c_double, vp]
    lib.ssm_plan_set_mask.argtypes = [vp, vp, vp]
    lib.ssm_selftest_wait_timeout.argtypes = [ctypes.c_uint, vp]
    lib.ssm_tune_beta.argtypes = [ctypes.POINTER(SsmParams), vp, vp, i64, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  vp, dp, vp, vp]
    lib.ssm_plan_footprint.argtypes = [ctypes.POINTER(SsmParams), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.ssm_plan_device_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.ssm_server_default_config.argtypes = [ctypes.POINTER(SsmServerConfig)]
    lib.ssm_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(SsmServerConfig)]
    lib.ssm_server_submit.argtypes = [vp, ctypes.POINTER(SsmParams), vp, vp, i64, vp, i64,
                                      ctypes.POINTER(ctypes.c_int64)]
    lib.ssm_server_poll.argtypes = [vp, i64, ctypes.POINTER(SsmRequestInfo)]
    lib.ssm_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(SsmRequestInfo)]
    lib.ssm_server_stats_read.argtypes = [vp, ctypes.POINTER(SsmServerStats)]
    lib.ssm_server_destroy.argtypes = [vp]
    lib.ssm_status_string.argtypes = [ctypes.c_int]
    lib.ssm_status_string.restype = ctypes.c_char_p
    lib.ssm_last_error.restype = ctypes.c_char_p
    lib.ssm_launch_count.restype = ctypes.c_int64
    for name in ("ssm_default_params", "ssm_plan", "ssm_solve", "ssm_solve_host",
                 "ssm_solve_resume", "ssm_plan_set_stopping",
                 "ssm_objective", "ssm_plan_factors", "ssm_plan_info", "ssm_destroy",
                 "ssm_profile_enable",
                 "ssm_profile_read", "ssm_objective_noalloc", "ssm_plan_set_graphs",
                 "ssm_plan_ex", "ssm_server_submit_device", "ssm_plan_set_beta",
                 "ssm_tune_beta", "ssm_plan_launch_info", "ssm_plan_set_mask",
                 "ssm_selftest_wait_timeout", "ssm_plan_batched", "ssm_plan_multi",
                 "ssm_group_create", "ssm_group_solve", "ssm_group_device_bytes",
                 "ssm_group_destroy",
                 "ssm_plan_footprint", "ssm_plan_device_bytes", "ssm_server_default_config",
                 "ssm_server_create", "ssm_server_submit", "ssm_server_poll", "ssm_server_wait",
                 "ssm_server_stats_read", "ssm_server_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def launch_count() -> int:
    return int(load_library().ssm_launch_count())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_params(P, Q, dims, lam, beta, *, form="lowrank", precision="fp32", rank=0,
                rank_tol=5e-5, xi_p=0.0, stencil_pairs=2, max_iter=300, check_every=10,
                tol_primal=0.0, tol_change=0.0) -> SsmParams:
    """ssm_params for a P x Q dictionary on the grid `dims`."""
    lib = load_library()
    p = SsmParams()
    lib.ssm_default_params(ctypes.byref(p))
    dims = tuple(int(d) for d in dims)
    p.ndim = len(dims)
    for i, d in enumerate(dims):
        p.dims[i] = d
    p.P, p.Q = int(P), int(Q)
    p.lam, p.beta, p.xi_p = float(lam), float(beta), float(xi_p)
    p.form = FORMS[form]
    p.precision = PRECISIONS[precision]
    p.rank, p.rank_tol = int(rank), float(rank_tol)
    p.stencil_pairs = int(stencil_pairs)
    p.max_iter, p.check_every = int(max_iter), int(check_every)
    p.tol_primal, p.tol_change = float(tol_primal), float(tol_change)
    return p


def footprint(P, Q, dims, *, device=0, **kw):
    """(persistent, peak) device bytes of a plan (ssm_plan_footprint)."""
    p = make_params(P, Q, dims, kw.pop("lam", 0.0), kw.pop("beta", 1.0), **kw)
    a, b = ctypes.c_int64(), ctypes.c_int64()
    st = load_library().ssm_plan_footprint(ctypes.byref(p), int(device), ctypes.byref(a),
                                           ctypes.byref(b))
    if st != SSM_OK:
        raise SsmError(st, "ssm_plan_footprint")
    return a.value, b.value


def tune_beta(K, M, dims, lam, *, iters=300, n_grid=15, grid_lo=-6.0, grid_hi=1.0, rank=0,
              stencil_pairs=2, device=0, stream=None):
    """The beta heuristic of Sec. III-E on the centre patch (ssm_tune_beta).
    M: P x N host array. Returns (best beta, betas, objectives)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float32)
    P, Q = K.shape
    p = make_params(P, Q, dims, lam, 1.0, rank=rank, stencil_pairs=stencil_pairs)
    best = ctypes.c_double()
    betas = np.zeros(n_grid)
    J = np.zeros(n_grid)
    st = load_library().ssm_tune_beta(
        ctypes.byref(p), K.ctypes.data_as(ctypes.c_void_p), M.ctypes.data_as(ctypes.c_void_p),
        M.shape[1], int(iters), int(n_grid), float(grid_lo), float(grid_hi), int(device),
        _stream_handle(stream), ctypes.byref(best), betas.ctypes.data_as(ctypes.c_void_p),
        J.ctypes.data_as(ctypes.c_void_p))
    if st != SSM_OK:
        raise SsmError(st, "ssm_tune_beta")
    return best.value, betas, J


class Plan:
    """A planned solver for one dictionary K (P x Q) and one voxel grid."""

    def __init__(self, K, dims, lam, beta, *, form="lowrank", precision="fp32", rank=0,
                 rank_tol=5e-5, xi_p=0.0, stencil_pairs=2, max_iter=300, check_every=10,
                 tol_primal=0.0, tol_change=0.0, device=0, stream=None, launch_waves=1,
                 batch=None):
        """batch=B: B independent slices of the grid `dims` (1D or 2D) sharing K, solved
        together (ssm_plan_batched); M and F then hold the slices one after another."""
        lib = load_library()
        K = np.ascontiguousarray(K, dtype=np.float64)
        p = make_params(K.shape[0], K.shape[1], dims, lam, beta, form=form,
                        precision=precision, rank=rank, rank_tol=rank_tol, xi_p=xi_p,
                        stencil_pairs=stencil_pairs, max_iter=max_iter,
                        check_every=check_every, tol_primal=tol_primal, tol_change=tol_change)
        dims = tuple(int(d) for d in dims)
        self.params = p
        self.dims = dims
        self.P, self.Q = p.P, p.Q
        self.N = int(np.prod(dims)) * (int(batch) if batch else 1)
        self.device = device
        self._h = ctypes.c_void_p()
        if batch:
            st = lib.ssm_plan_batched(ctypes.byref(self._h), ctypes.byref(p), int(batch),
                                      K.ctypes.data_as(ctypes.c_void_p), int(device),
                                      _stream_handle(stream), int(launch_waves))
        else:
            st = lib.ssm_plan_ex(ctypes.byref(self._h), ctypes.byref(p),
                                 K.ctypes.data_as(ctypes.c_void_p), int(device),
                                 _stream_handle(stream), int(launch_waves))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan")

    def set_mask(self, mask, stream=None):
        """Estimate only the voxels where `mask` (N values, voxel order) is nonzero
        (ssm_plan_set_mask); None removes the mask."""
        if mask is None:
            ptr = None
        else:
            m = np.ascontiguousarray(np.asarray(mask).ravel() != 0, dtype=np.uint8)
            assert m.size == self.N
            ptr = m.ctypes.data_as(ctypes.c_void_p)
        st = load_library().ssm_plan_set_mask(self._h, ptr, _stream_handle(stream))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_set_mask")

    def set_beta(self, beta, stream=None):
        """Change beta without refactorising K (ssm_plan_set_beta)."""
        st = load_library().ssm_plan_set_beta(self._h, float(beta), _stream_handle(stream))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_set_beta")

    def set_graphs(self, enable=True):
        """Replay iteration blocks as CUDA graphs (ssm_plan_set_graphs)."""
        st = load_library().ssm_plan_set_graphs(self._h, int(bool(enable)))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_set_graphs")

    def launch_info(self):
        """Launch configuration (ssm_plan_launch_info): tile width, grids, waves."""
        li = SsmLaunchInfo()
        st = load_library().ssm_plan_launch_info(self._h, ctypes.byref(li))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_launch_info")
        return li.as_dict()

    def device_bytes(self):
        b = ctypes.c_int64()
        st = load_library().ssm_plan_device_bytes(self._h, ctypes.byref(b))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_device_bytes")
        return b.value

    def solve(self, M, out=None, stream=None):
        """M: CUDA float32 tensor P x N (row stride >= N). Returns (F tensor Q x N, info)."""
        import torch
        assert M.is_cuda and M.dtype == torch.float32 and M.dim() == 2 and M.stride(1) == 1
        assert M.shape[0] == self.P and M.shape[1] == self.N
        if out is None:
            out = torch.empty((self.Q, self.N), dtype=torch.float32, device=M.device)
        info = SsmInfo()
        st = load_library().ssm_solve(self._h, ctypes.c_void_p(M.data_ptr()), M.stride(0),
                                      ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                      ctypes.byref(info), _stream_handle(stream))
        if st not in (SSM_OK, SSM_ENOTCONVERGED):
            raise SsmError(st, "ssm_solve")
        return out, info.as_dict()

    def resume(self, M, out=None, stream=None):
        """Continue from the state the last solve left for max_iter more iterations
        (ssm_solve_resume). Returns (F, info) like solve()."""
        import torch
        assert M.is_cuda and M.dtype == torch.float32 and M.dim() == 2 and M.stride(1) == 1
        if out is None:
            out = torch.empty((self.Q, self.N), dtype=torch.float32, device=M.device)
        info = SsmInfo()
        st = load_library().ssm_solve_resume(self._h, ctypes.c_void_p(M.data_ptr()), M.stride(0),
                                             ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                             ctypes.byref(info), _stream_handle(stream))
        if st not in (SSM_OK, SSM_ENOTCONVERGED):
            raise SsmError(st, "ssm_solve_resume")
        return out, info.as_dict()

    def set_max_iter(self, max_iter):
        """The iteration budget of later solves (the plan's other parameters stay)."""
        self.params.max_iter = int(max_iter)
        st = load_library().ssm_plan_set_stopping(self._h, int(max_iter),
                                                  int(self.params.check_every),
                                                  float(self.params.tol_primal),
                                                  float(self.params.tol_change))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_set_stopping")

    def solve_async(self, M, out, stream=None):
        """As solve() without the info read-back (no host synchronisation unless a
        tolerance test needs it). Returns the status."""
        st = load_library().ssm_solve(self._h, ctypes.c_void_p(M.data_ptr()), M.stride(0),
                                      ctypes.c_void_p(out.data_ptr()), out.stride(0), None,
                                      _stream_handle(stream))
        if st not in (SSM_OK, SSM_ENOTCONVERGED):
            raise SsmError(st, "ssm_solve")
        return st

    def solve_host(self, M_host, F_host, stream=None, with_info=False):
        """Host buffers (torch CPU tensors, pinned for async copies). Returns the status,
        or (status, info) with `with_info`."""
        info = SsmInfo()
        st = load_library().ssm_solve_host(self._h, ctypes.c_void_p(M_host.data_ptr()),
                                           M_host.stride(0), ctypes.c_void_p(F_host.data_ptr()),
                                           F_host.stride(0),
                                           ctypes.byref(info) if with_info else None,
                                           _stream_handle(stream))
        if st not in (SSM_OK, SSM_ENOTCONVERGED):
            raise SsmError(st, "ssm_solve_host")
        return (st, info.as_dict()) if with_info else st

    def objective(self, M, F, use_full_k=False, stream=None):
        J = ctypes.c_double()
        st = load_library().ssm_objective(self._h, ctypes.c_void_p(M.data_ptr()), M.stride(0),
                                          ctypes.c_void_p(F.data_ptr()), F.stride(0),
                                          int(bool(use_full_k)), ctypes.byref(J),
                                          _stream_handle(stream))
        if st != SSM_OK:
            raise SsmError(st, "ssm_objective")
        return J.value

    def info(self):
        """Plan-level ssm_info fields (rank, xi_p, sigma1, the power-iteration results)."""
        out = SsmInfo()
        st = load_library().ssm_plan_info(self._h, ctypes.byref(out))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_info")
        return out.as_dict()

    def factors(self, with_vr=True):
        n = min(self.P, self.Q)
        sig = np.zeros(n)
        r = ctypes.c_int()
        load_library().ssm_plan_factors(self._h, sig.ctypes.data_as(ctypes.c_void_p), None,
                                        ctypes.byref(r))
        vr = None
        if with_vr:
            vr = np.zeros((self.Q, r.value))
            st = load_library().ssm_plan_factors(self._h, None,
                                                 vr.ctypes.data_as(ctypes.c_void_p), None)
            if st != SSM_OK:
                raise SsmError(st, "ssm_plan_factors")
        return sig, vr, r.value

    def profile(self, enable=True):
        """Time the dominant kernel of every iteration with CUDA events."""
        st = load_library().ssm_profile_enable(self._h, int(bool(enable)))
        if st != SSM_OK:
            raise SsmError(st, "ssm_profile_enable")

    def profile_read(self):
        """(summed device ms, launches) of the dominant kernel since the last read."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        st = load_library().ssm_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n))
        if st != SSM_OK:
            raise SsmError(st, "ssm_profile_read")
        return ms.value, n.value

    def close(self):
        if self._h:
            load_library().ssm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MultiPlan(Plan):
    """A planned solver with a dictionary per voxel label (ssm_plan_multi): Ks holds the
    ndict dictionaries (each P x Q), labels the dictionary of every voxel (N ints in
    voxel order). The low-rank form in FP32; solve/resume/set_max_iter/set_graphs/
    profile/info as for Plan."""

    def __init__(self, Ks, labels, dims, lam, beta, *, rank=0, rank_tol=5e-5, xi_p=0.0,
                 stencil_pairs=2, max_iter=300, check_every=10, tol_primal=0.0,
                 tol_change=0.0, device=0, stream=None):
        lib = load_library()
        Ks = np.ascontiguousarray(np.stack([np.asarray(K, np.float64) for K in Ks]))
        ndict, P, Q = Ks.shape
        lab = np.ascontiguousarray(np.asarray(labels).ravel(), dtype=np.int32)
        dims = tuple(int(d) for d in dims)
        assert lab.size == int(np.prod(dims)), "one label per voxel"
        p = make_params(P, Q, dims, lam, beta, form="lowrank", precision="fp32", rank=rank,
                        rank_tol=rank_tol, xi_p=xi_p, stencil_pairs=stencil_pairs,
                        max_iter=max_iter, check_every=check_every, tol_primal=tol_primal,
                        tol_change=tol_change)
        self.params = p
        self.dims = dims
        self.P, self.Q = P, Q
        self.N = lab.size
        self.ndict = ndict
        self.device = device
        self._h = ctypes.c_void_p()
        st = lib.ssm_plan_multi(ctypes.byref(self._h), ctypes.byref(p), int(ndict),
                                Ks.ctypes.data_as(ctypes.c_void_p),
                                lab.ctypes.data_as(ctypes.c_void_p), int(device),
                                _stream_handle(stream))
        if st != SSM_OK:
            raise SsmError(st, "ssm_plan_multi")


class Group:
    """Independent low-rank FP32 plans solved together, one launch per iteration for all
    (ssm_group_*). The plans must stay open while the group is used."""

    def __init__(self, plans, stream=None):
        self.plans = list(plans)
        n = len(self.plans)
        arr = (ctypes.c_void_p * n)(*[p._h.value for p in self.plans])
        self._h = ctypes.c_void_p()
        st = load_library().ssm_group_create(ctypes.byref(self._h), n, arr,
                                             _stream_handle(stream))
        if st != SSM_OK:
            raise SsmError(st, "ssm_group_create")

    def solve(self, Ms, outs=None, stream=None):
        """Ms: CUDA float32 tensors (P_i x N_i). Returns ([F_i], [info_i], status)."""
        import torch
        n = len(self.plans)
        assert len(Ms) == n
        if outs is None:
            outs = [torch.empty((p.Q, p.N), dtype=torch.float32, device=M.device)
                    for p, M in zip(self.plans, Ms)]
        for p, M in zip(self.plans, Ms):
            assert M.is_cuda and M.dtype == torch.float32 and M.stride(1) == 1
            assert M.shape[0] == p.P and M.shape[1] == p.N
        mp = (ctypes.c_void_p * n)(*[M.data_ptr() for M in Ms])
        lm = (ctypes.c_int64 * n)(*[M.stride(0) for M in Ms])
        fp = (ctypes.c_void_p * n)(*[F.data_ptr() for F in outs])
        lf = (ctypes.c_int64 * n)(*[F.stride(0) for F in outs])
        infos = (SsmInfo * n)()
        st = load_library().ssm_group_solve(self._h, mp, lm, fp, lf, infos,
                                            _stream_handle(stream))
        if st not in (SSM_OK, SSM_ENOTCONVERGED):
            raise SsmError(st, "ssm_group_solve")
        return outs, [infos[i].as_dict() for i in range(n)], st

    def device_bytes(self):
        b = ctypes.c_int64()
        st = load_library().ssm_group_device_bytes(self._h, ctypes.byref(b))
        if st != SSM_OK:
            raise SsmError(st, "ssm_group_device_bytes")
        return b.value

    def close(self):
        if self._h:
            load_library().ssm_group_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching solve server (ssm_server_* in include/ssm.h).

    submit() queues one solve on host arrays and returns a ticket; wait() returns
    (F, info) when it has finished. The arrays are kept alive here until then.
    """

    def __init__(self, *, device=0, max_active=4, hbm_budget=0, use_graphs=True,
                 cache_plans=True, max_bypass=-1, simulate_us=0, small_bytes=None,
                 large_waves=None, reserved_small=None, group_small=None):
        lib = load_library()
        c = SsmServerConfig()
        lib.ssm_server_default_config(ctypes.byref(c))
        c.device, c.max_active, c.hbm_budget = int(device), int(max_active), int(hbm_budget)
        c.use_graphs, c.cache_plans = int(bool(use_graphs)), int(bool(cache_plans))
        c.max_bypass, c.simulate_us = int(max_bypass), int(simulate_us)
        if small_bytes is not None:
            c.small_bytes = int(small_bytes)
        if large_waves is not None:
            c.large_waves = int(large_waves)
        if reserved_small is not None:
            c.reserved_small = int(reserved_small)
        if group_small is not None:
            c.group_small = int(group_small)
        self._h = ctypes.c_void_p()
        st = lib.ssm_server_create(ctypes.byref(self._h), ctypes.byref(c))
        if st != SSM_OK:
            raise SsmError(st, "ssm_server_create")
        self._keep = {}

    def submit(self, K, M, dims, lam, beta, *, out=None, **kw):
        """K: P x Q (float64); M: P x N float32, a host array (F returned in a numpy
        array) or a CUDA tensor (F returned in a CUDA tensor, nothing copied to the
        host). Returns a ticket."""
        K = np.ascontiguousarray(K, dtype=np.float64)
        P, Q = K.shape
        N = int(np.prod(dims))
        p = make_params(P, Q, dims, lam, beta, **kw)
        t = ctypes.c_int64()
        if hasattr(M, "is_cuda") and M.is_cuda:
            import torch
            assert M.dtype == torch.float32 and M.shape == (P, N) and M.stride(1) == 1
            F = out if out is not None else torch.empty((Q, N), dtype=torch.float32,
                                                        device=M.device)
            assert F.is_cuda and F.stride(1) == 1 and F.shape == (Q, N)
            st = load_library().ssm_server_submit_device(
                self._h, ctypes.byref(p), K.ctypes.data_as(ctypes.c_void_p),
                ctypes.c_void_p(M.data_ptr()), M.stride(0), ctypes.c_void_p(F.data_ptr()),
                F.stride(0), ctypes.byref(t))
        else:
            M = np.ascontiguousarray(M, dtype=np.float32)
            assert M.shape == (P, N)
            F = out if out is not None else np.empty((Q, N), dtype=np.float32)
            assert F.dtype == np.float32 and F.flags.c_contiguous and F.shape == (Q, N)
            st = load_library().ssm_server_submit(
                self._h, ctypes.byref(p), K.ctypes.data_as(ctypes.c_void_p),
                M.ctypes.data_as(ctypes.c_void_p), N, F.ctypes.data_as(ctypes.c_void_p), N,
                ctypes.byref(t))
        if st != SSM_OK:
            raise SsmError(st, "ssm_server_submit")
        self._keep[t.value] = (K, M, F)
        return t.value

    def _finish(self, ticket, st, info):
        if st == SSM_EPENDING:
            return None
        if st != SSM_OK:
            raise SsmError(st, "ssm_server_wait")
        _, _, F = self._keep.pop(ticket)
        return F, info.as_dict()

    def wait(self, ticket, timeout_ms=-1.0):
        """(F, info) of a finished request; None if the timeout ran out first."""
        info = SsmRequestInfo()
        st = load_library().ssm_server_wait(self._h, int(ticket), float(timeout_ms),
                                            ctypes.byref(info))
        return self._finish(ticket, st, info)

    def poll(self, ticket):
        info = SsmRequestInfo()
        st = load_library().ssm_server_poll(self._h, int(ticket), ctypes.byref(info))
        return self._finish(ticket, st, info)

    def stats(self):
        s = SsmServerStats()
        st = load_library().ssm_server_stats_read(self._h, ctypes.byref(s))
        if st != SSM_OK:
            raise SsmError(st, "ssm_server_stats_read")
        return s.as_dict()

    def close(self):
        if self._h:
            load_library().ssm_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
