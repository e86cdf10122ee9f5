"""Seeded synthetic inputs shaped like the paper's four experiments (Sec. IV).

This module only builds inputs: dictionaries K (P x Q) from the signal models the
experiments use, nonnegative ground-truth spectroscopic images F (Q x N), and noisy
data M = K F + noise (the linear mixture model of Eq. 1 / its matrix form). It holds
none of the estimation method's arithmetic, so the CUDA path and the FP64 oracle can
both take their inputs from here without sharing any solver code.

Layouts (all row-major, float64 on return):
  K : P x Q, row p = one contrast encoding, column q = one spectral position.
  F : Q x N, row q = the spatial map of compartment q ("map-major").
  M : P x N, row p = the p-th measured image.
  voxel index n = x + nx*(y + ny*z) (x fastest).

The paper's datasets (DR-CSI mouse cord, IR-MSE brain, MSE-T2 brain, MRF brain) are
not available; these workloads stand in for them with the same kind of dictionary
and the (P, Q, N) of the benchmark configurations.
"""
from __future__ import annotations

import dataclasses

import numpy as np


# --------------------------------------------------------------------------------------
# dictionaries (the physics kernel b(theta_p, gamma_q) of Eq. 1; quadrature weights = 1)
# --------------------------------------------------------------------------------------

def diffusion_relaxation_dictionary(b_values, te_ms, diff_mm2s, t2_ms):
    """K[p, q] = exp(-b D) exp(-TE/T2); p = (b index, TE index), q = (D index, T2 index)."""
    b = np.asarray(b_values, np.float64)
    te = np.asarray(te_ms, np.float64)
    dd = np.asarray(diff_mm2s, np.float64)
    t2 = np.asarray(t2_ms, np.float64)
    k_b = np.exp(-b[:, None] * dd[None, :])            # (nb, nD)
    k_t = np.exp(-te[:, None] / t2[None, :])           # (nte, nT2)
    K = k_b[:, None, :, None] * k_t[None, :, None, :]  # (nb, nte, nD, nT2)
    return K.reshape(b.size * te.size, dd.size * t2.size)


def inversion_recovery_dictionary(ti_ms, te_ms, t1_ms, t2_ms):
    """K[p, q] = (1 - 2 exp(-TI/T1)) exp(-TE/T2); p = (TI, TE), q = (T1, T2)."""
    ti = np.asarray(ti_ms, np.float64)
    te = np.asarray(te_ms, np.float64)
    t1 = np.asarray(t1_ms, np.float64)
    t2 = np.asarray(t2_ms, np.float64)
    k1 = 1.0 - 2.0 * np.exp(-ti[:, None] / t1[None, :])
    k2 = np.exp(-te[:, None] / t2[None, :])
    K = k1[:, None, :, None] * k2[None, :, None, :]
    return K.reshape(ti.size * te.size, t1.size * t2.size)


def spgr_fingerprint_dictionary(n_tp, t1_ms, t2_ms, seed, b1=1.0):
    """Spoiled-gradient-echo fingerprinting dictionary, columns L2-normalised.

    Flip angles alpha_p ~ U(5, 70) degrees and TR_p ~ U(10, 15) ms are drawn from the
    seed; TE_p = TR_p / 2. Longitudinal magnetisation starts at 1; each time point
    reads Mz sin(alpha) exp(-TE/T2) and then relaxes Mz <- 1 - (1 - Mz cos a) exp(-TR/T1).
    b1 scales the whole flip-angle train (the transmit field's relative amplitude).
    """
    rng = np.random.default_rng(seed)
    alpha = np.deg2rad(rng.uniform(5.0, 70.0, n_tp)) * float(b1)
    tr = rng.uniform(10.0, 15.0, n_tp)
    te = 0.5 * tr
    t1 = np.asarray(t1_ms, np.float64)
    t2 = np.asarray(t2_ms, np.float64)
    T1, T2 = np.meshgrid(t1, t2, indexing="ij")
    T1 = T1.ravel()
    T2 = T2.ravel()
    mz = np.ones_like(T1)
    K = np.empty((n_tp, T1.size))
    for p in range(n_tp):
        K[p] = mz * np.sin(alpha[p]) * np.exp(-te[p] / T2)
        mz = 1.0 - (1.0 - mz * np.cos(alpha[p])) * np.exp(-tr[p] / T1)
    K /= np.linalg.norm(K, axis=0, keepdims=True)
    return K


# --------------------------------------------------------------------------------------
# ground truth and data
# --------------------------------------------------------------------------------------

def _smooth_field(rng, dims, n_waves=4):
    """A smooth nonnegative field on the grid: a few low-frequency cosines, offset."""
    axes = [np.arange(d, dtype=np.float64) / max(d, 1) for d in dims]
    mesh = np.meshgrid(*axes, indexing="ij")  # dims order (nx, ny[, nz])
    field = np.zeros(dims)
    for _ in range(n_waves):
        k = rng.uniform(0.3, 2.0, len(dims)) * 2.0 * np.pi
        ph = rng.uniform(0.0, 2.0 * np.pi)
        arg = sum(kk * m for kk, m in zip(k, mesh))
        field += np.cos(arg + ph)
    field /= n_waves
    # voxel index x fastest: transpose (x, y, z) -> (z, y, x) before ravel
    return np.ascontiguousarray(field.transpose(tuple(reversed(range(len(dims)))))).ravel()


def multi_echo_t2_dictionary(te_ms, t2_ms):
    """Multi-echo spin-echo T2 relaxometry (a 1D spectrum): K[p, q] = exp(-TE_p / T2_q)."""
    te = np.asarray(te_ms, np.float64)[:, None]
    t2 = np.asarray(t2_ms, np.float64)[None, :]
    return np.exp(-te / t2)


def ellipse_mask(dims, fill):
    """A 2D object mask, voxel order: the ellipse inscribed in `fill` of the grid."""
    nx, ny = dims
    x = (np.arange(nx) + 0.5) / nx - 0.5
    y = (np.arange(ny) + 0.5) / ny - 0.5
    X, Y = np.meshgrid(x, y, indexing="xy")          # [y][x]
    return ((X / (0.5 * fill)) ** 2 + (Y / (0.5 * fill)) ** 2 <= 1.0).ravel()


def spectral_peaks(shape2d, centers, widths):
    """Unit-sum Gaussian peaks on a 2D spectral grid in normalised log coordinates.

    Returns S with shape (Q, J): column j is peak j over q = i0 * n1 + i1.
    """
    n0, n1 = shape2d
    u0 = (np.arange(n0) + 0.5) / n0
    u1 = (np.arange(n1) + 0.5) / n1
    U0, U1 = np.meshgrid(u0, u1, indexing="ij")
    cols = []
    for (c0, c1), (w0, w1) in zip(centers, widths):
        g = np.exp(-0.5 * (((U0 - c0) / w0) ** 2 + ((U1 - c1) / w1) ** 2))
        cols.append((g / g.sum()).ravel())
    return np.stack(cols, axis=1)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple           # grid (nx, ny[, nz])
    P: int
    Q: int
    lam: float
    beta: float
    iters: int
    snr: float
    seed: int

    @property
    def N(self) -> int:
        return int(np.prod(self.dims))


# beta: the paper tunes it once on a 3x3 patch for fastest convergence (Sec. III-E);
# these are the values that heuristic picks on each workload (the script that derives
# them with the FP64 oracle, and the record it writes, live in tests/golden).
WORKLOADS = {
    "dr2d_tiny": Workload("dr2d_tiny", (32, 32), 30, 225, 1e-2,
                          0.02616762331016125, 300, 100.0, 42),
    "dr2d_slice": Workload("dr2d_slice", (128, 128), 120, 2500, 1e-2,
                           0.9863724793789308, 300, 100.0, 43),
    "rr3d_t1t2": Workload("rr3d_t1t2", (96, 96, 64), 64, 1600, 1e-2,
                          0.47668520453230206, 300, 100.0, 44),
    "mrf2d": Workload("mrf2d", (192, 192), 1000, 900, 1e-2,
                      0.025222210292153446, 300, 50.0, 45),
    "mse_t2": Workload("mse_t2", (84, 72), 32, 300, 1e-2,
                       0.02809082955801525, 300, 100.0, 47),
}


def dictionary_for(name: str) -> np.ndarray:
    """The dictionary K (P x Q, float64) of a named workload."""
    if name == "dr2d_tiny":
        return diffusion_relaxation_dictionary(
            np.linspace(0, 3000, 6), np.linspace(60, 200, 5),
            np.geomspace(1e-4, 3e-3, 15), np.geomspace(10, 300, 15))
    if name == "dr2d_slice":
        return diffusion_relaxation_dictionary(
            np.linspace(0, 3000, 15), np.linspace(60, 200, 8),
            np.geomspace(1e-4, 3e-3, 50), np.geomspace(10, 300, 50))
    if name == "rr3d_t1t2":
        return inversion_recovery_dictionary(
            np.geomspace(50, 3000, 8), np.linspace(10, 300, 8),
            np.geomspace(200, 4000, 40), np.geomspace(10, 300, 40))
    if name == "mrf2d":
        return spgr_fingerprint_dictionary(
            1000, np.geomspace(200, 4000, 30), np.geomspace(10, 300, 30), seed=1045)
    if name == "mse_t2":
        # 32 echoes every 10 ms, 300 log-spaced T2 values (a 1D spectrum per voxel)
        return multi_echo_t2_dictionary(np.arange(1, 33) * 10.0, np.geomspace(10, 2000, 300))
    raise KeyError(name)


def mask_for(name: str, dims=None):
    """The object mask of a named workload (None: every voxel is estimated). The
    1D-spectrum workload's object is an ellipse of 4472 voxels in an 84 x 72 grid, about
    the voxel count of the paper's multicomponent T2 brain data set (Sec. IV-C)."""
    if name == "mse_t2":
        return ellipse_mask(dims or WORKLOADS[name].dims, fill=0.9695)
    return None


def _spectral_shape(name):
    return {"dr2d_tiny": (15, 15), "dr2d_slice": (50, 50),
            "rr3d_t1t2": (40, 40), "mrf2d": (30, 30), "mse_t2": (300, 1)}[name]


def ground_truth_factors(dims, spec_shape, seed, n_peaks=3):
    """F_true = S @ A with S (Q x J) unit-sum spectral peaks, A (J x N) >= 0 maps.

    The third peak's amplitude is clamped to zero over part of the image so voxels
    hold two or three peaks.
    """
    rng = np.random.default_rng(seed)
    centers = [(0.25, 0.30), (0.60, 0.65), (0.80, 0.25)][:n_peaks]
    widths = [(0.07, 0.09), (0.08, 0.06), (0.06, 0.07)][:n_peaks]
    S = spectral_peaks(spec_shape, centers, widths)
    N = int(np.prod(dims))
    A = np.empty((n_peaks, N))
    for j in range(n_peaks):
        fld = _smooth_field(rng, dims)
        if j < 2:
            A[j] = 1.0 + 0.5 * fld
        else:
            A[j] = np.maximum(0.0, fld) * 1.5
    return S, A


def make_problem(name: str, dims=None, seed=None, snr=None, dtype=np.float32):
    """(K float64, M dtype, F_true factors (S, A)) for a named workload.

    `dims` overrides the grid (same dictionary); `seed`/`snr` override the noise.
    M = K (S A) + N(0, sigma^2), sigma = max_n M_clean[0, n] / SNR.
    """
    w = WORKLOADS[name]
    dims = tuple(dims) if dims is not None else w.dims
    seed = w.seed if seed is None else seed
    snr = w.snr if snr is None else snr
    K = dictionary_for(name)
    S, A = ground_truth_factors(dims, _spectral_shape(name), seed)
    mask = mask_for(name, dims)
    if mask is not None:
        A = A * mask[None, :]       # nothing outside the object: its data is noise alone
    KS = K @ S                      # P x J
    rng = np.random.default_rng(seed + 1000)
    M = np.empty((K.shape[0], A.shape[1]), dtype=dtype)
    sigma = None
    row_block = 16
    for p0 in range(0, K.shape[0], row_block):
        clean = KS[p0:p0 + row_block] @ A
        if sigma is None:
            sigma = float(np.max(np.abs(clean[0]))) / snr if snr and snr > 0 else 0.0
        noise = rng.standard_normal(clean.shape) * sigma if sigma else 0.0
        M[p0:p0 + row_block] = (clean + noise).astype(dtype)
    return K, M, (S, A)


def random_problem(P, Q, dims, seed, snr=None, nonneg_k=True, full_rank=False):
    """A small random problem for edge cases: K P x Q, F_true >= 0 sparse-ish, M = K F (+noise).

    Returns (K, M, F_true), all float64.
    """
    rng = np.random.default_rng(seed)
    N = int(np.prod(dims))
    if nonneg_k:
        K = rng.uniform(0.0, 1.0, (P, Q))
    else:
        K = rng.standard_normal((P, Q))
    if full_rank and P >= Q:
        K += np.eye(P, Q) * 2.0
    F = rng.uniform(0.0, 1.0, (Q, N)) * (rng.uniform(0, 1, (Q, N)) < 0.4)
    M = K @ F
    if snr:
        M = M + rng.standard_normal(M.shape) * (np.abs(M).max() / snr)
    return K, M, F


def b1_varying_problem(dims, levels, n_tp=60, t1_ms=None, t2_ms=None, seed=0, snr=100.0,
                       b1_range=(0.8, 1.2)):
    """A fingerprinting problem with a spatially varying dictionary (one per B1 level).

    A smooth B1 field over the grid is quantised to `levels` values spread evenly over
    `b1_range`; voxel n is labelled with its level c(n) and its data is
    m_n = K_{c(n)} f_n + noise, K_c the dictionary at that B1 (the same seeded flip-angle
    and TR train, scaled). The ground truth has two smooth nonnegative spectral peaks.
    Returns (Ks, labels, M, F_true), float64.
    """
    rng = np.random.default_rng(seed)
    t1 = np.geomspace(300.0, 3000.0, 6) if t1_ms is None else np.asarray(t1_ms, np.float64)
    t2 = np.geomspace(20.0, 300.0, 5) if t2_ms is None else np.asarray(t2_ms, np.float64)
    b1_levels = np.linspace(b1_range[0], b1_range[1], int(levels))
    Ks = [spgr_fingerprint_dictionary(n_tp, t1, t2, seed + 1, b1=b) for b in b1_levels]
    field = _smooth_field(rng, dims)
    lo, hi = field.min(), field.max()
    u = (field - lo) / max(hi - lo, 1e-300)
    labels = np.minimum((u * levels).astype(np.int64), levels - 1)
    Q = t1.size * t2.size
    N = int(np.prod(dims))
    a1 = 0.5 + 0.5 * _smooth_field(rng, dims)
    a2 = np.clip(0.5 + 0.5 * _smooth_field(rng, dims), 0.0, None)
    F = np.zeros((Q, N))
    F[rng.integers(0, Q)] = a1
    F[rng.integers(0, Q)] += a2
    M = np.empty((n_tp, N))
    for c, K in enumerate(Ks):
        sel = labels == c
        M[:, sel] = K @ F[:, sel]
    if snr:
        M = M + rng.standard_normal(M.shape) * (np.abs(M).max() / snr)
    return Ks, labels, M, F


# The fingerprinting experiment with a dictionary per B1 level (Sec. IV-D: 61 quantised
# levels, one dictionary each, about 24000 voxels). Stand-in: the SPGR fingerprint
# dictionary of the 2D fingerprinting workload's T1/T2 grid (30 x 30 atoms) at 120 time
# points, at 61 B1 levels over [0.8, 1.2], on a 156 x 156 grid (24336 voxels) labelled
# by a smooth B1 field. beta: the heuristic of Sec. III-E on the centre 3x3 patch with
# the centre voxel's dictionary (tests/golden/make_golden.py records it).
B1_LEVELS = 61
B1_WORKLOAD = Workload("mrf_b1", (156, 156), 120, 900, 1e-2, 0.026549077590512404, 300,
                       50.0, 48)


def make_b1_problem(dims=None, levels=B1_LEVELS, seed=None):
    """(Ks list of P x Q float64, labels int64 N, M float32 P x N, F_true float64) of the
    spatially varying dictionary workload."""
    w = B1_WORKLOAD
    dims = tuple(dims) if dims is not None else w.dims
    Ks, labels, M, F = b1_varying_problem(
        dims, levels, n_tp=w.P, t1_ms=np.geomspace(200, 4000, 30),
        t2_ms=np.geomspace(10, 300, 30), seed=w.seed if seed is None else seed, snr=w.snr)
    return Ks, labels, M.astype(np.float32), F


def grid_dims_for_n(n: int):
    """A 1D grid of n voxels (n x 1)."""
    return (int(n), 1)


def workload_summary(name):
    w = WORKLOADS[name]
    return {"name": name, "grid": "x".join(str(d) for d in w.dims), "N": w.N,
            "P": w.P, "Q": w.Q, "lambda": w.lam, "beta": w.beta}


__all__ = [
    "WORKLOADS", "Workload", "make_problem", "B1_WORKLOAD", "B1_LEVELS", "make_b1_problem",
    "dictionary_for", "random_problem",
    "diffusion_relaxation_dictionary", "inversion_recovery_dictionary",
    "spgr_fingerprint_dictionary", "spectral_peaks", "ground_truth_factors",
    "workload_summary", "grid_dims_for_n",
]
