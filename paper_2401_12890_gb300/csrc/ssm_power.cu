// FP64 power iteration for the largest eigenvalue of the Hessian of Eq. 7,
//
//     H = I_N (x) K^T K + lambda D^T D (x) I_Q      (acting on the Q x N compartment maps),
//
// the curvature that bounds the step of a gradient method on Eq. 7. The z-step weight of
// Eq. 32 is checked against the D^T D part of it: the convergence condition the paper
// cites for the linearised step (Sec. III-C) asks for xi_p > 0.75 lambda ||D^T D||.
//
// H is a Kronecker sum, so its eigenvalues are mu_i + lambda nu_j (mu_i those of K^T K,
// nu_j those of D^T D) and lambda_max(H) = lambda_max(K^T K) + lambda lambda_max(D^T D).
// On the free-boundary box grid, D^T D = s (L_x (+) L_y (+) L_z) is again a Kronecker sum,
// of path-graph Laplacians, one per axis. Each factor gets its own FP64 power iteration on
// the device, all in one launch:
//   block 0           K^T K through the plan's FP64 Gram matrix of the smaller side
//                     (K K^T has the same nonzero spectrum); one warp per matrix row
//   blocks 1 .. naxes s L_path of one grid axis with >= 2 voxels; one warp, the two
//                     vectors in shared memory
// The start vectors are fixed pseudo-random values (a counter-based hash of the index).
// The Rayleigh quotient x^T A x of the normalised power iterates of a symmetric positive
// semidefinite A never decreases; an iteration stops once 32 further steps have raised it
// by at most 1e-15 of its value, or at its cap, where it is reported as not converged
// (the value is then a lower bound of the eigenvalue).
#include <algorithm>
#include <cmath>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

constexpr int kThreads = 256;
constexpr int kCheck = 32;                 // steps between stopping tests
constexpr int kMaxAxis = 8192;             // longest axis iterated (shared memory)

// splitmix64 of (i, salt) mapped to [0.5, 1.5): start vectors with no special structure
__device__ __forceinline__ double start_value(int64_t i, int salt) {
  uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)(salt + 1) * 0xD1B54A32D192ED03ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct PowerOut {
  double value[4];     // [0] K^T K, [1..3] s L of axis 0..2
  int iters[4];
  int converged[4];
};

// block-wide sums of two values (kThreads threads)
__device__ __forceinline__ void block_sum2(double& a, double& b, double (*red)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    red[warp][0] = a;
    red[warp][1] = b;
  }
  __syncthreads();
  double ta = 0.0, tb = 0.0;
  for (int w = 0; w < kThreads / 32; ++w) {
    ta += red[w][0];
    tb += red[w][1];
  }
  a = ta;
  b = tb;
  __syncthreads();
}

__device__ void power_gram(const double* __restrict__ A, int n, double* __restrict__ x,
                           double* __restrict__ y, int max_iter, PowerOut* out) {
  __shared__ double red[kThreads / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double xx = 0.0, dummy = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const double v = start_value(i, 0);
    x[i] = v;
    xx += v * v;
  }
  block_sum2(xx, dummy, red);
  const double inv0 = 1.0 / sqrt(xx);
  for (int i = threadIdx.x; i < n; i += kThreads) x[i] *= inv0;
  __syncthreads();
  double rq = 0.0, rq_ref = -1.0;
  int k = 0, conv = 0;
  while (k < max_iter) {
    // y = A x: one warp per row, lanes stride the columns (coalesced rows of A)
    for (int i = warp; i < n; i += kThreads / 32) {
      const double* row = A + (int64_t)i * n;
      double acc = 0.0;
      for (int j = lane; j < n; j += 32) acc = fma(row[j], x[j], acc);
      acc = warp_sum(acc);
      if (lane == 0) y[i] = acc;
    }
    __syncthreads();
    double xy = 0.0, yy = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      xy = fma(x[i], y[i], xy);
      yy = fma(y[i], y[i], yy);
    }
    block_sum2(xy, yy, red);
    rq = xy;                               // x has unit norm
    ++k;
    if (!(yy > 0.0)) break;                // A x = 0: the largest eigenvalue is 0
    const double inv = 1.0 / sqrt(yy);
    for (int i = threadIdx.x; i < n; i += kThreads) x[i] = y[i] * inv;
    __syncthreads();
    if (k % kCheck == 0) {
      if (rq_ref >= 0.0 && rq - rq_ref <= 1e-15 * fabs(rq)) {
        conv = 1;
        break;
      }
      rq_ref = rq;
    }
  }
  if (threadIdx.x == 0) {
    out->value[0] = rq;
    out->iters[0] = k;
    out->converged[0] = conv || !(rq > 0.0);
  }
}

// one warp: s L_path of length n (free boundary), vectors in shared memory. The iterate
// is normalised only every kCheck steps, where the Rayleigh quotient is formed: ||s L||
// <= 4 s <= 8 bounds the growth in between by 8^kCheck = 2^96, far inside FP64's range,
// and the eigenvalue is at least s (so the iterate does not shrink). A step is then one
// stencil pass, without the two warp reductions, the square root and the division of a
// normalised step (32-voxel axes: ~2k steps; 128: ~35k).
__device__ void power_axis(int n, double s, int axis, int max_iter, double* x, double* y,
                           PowerOut* out) {
  const int lane = threadIdx.x;
  double xx = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double v = start_value(i, 1 + axis);
    x[i] = v;
    xx += v * v;
  }
  xx = warp_sum(xx);
  const double inv0 = 1.0 / sqrt(xx);
  for (int i = lane; i < n; i += 32) x[i] *= inv0;
  __syncwarp();
  double rq = 0.0, rq_ref = -1.0;
  int k = 0, conv = 0;
  while (k < max_iter) {
    // kCheck - 1 plain steps: y = s L x, then swap
    for (int t = 1; t < kCheck && k < max_iter; ++t, ++k) {
      for (int i = lane; i < n; i += 32) {
        const double xi = x[i];
        double v = 0.0;
        if (i > 0) v += xi - x[i - 1];
        if (i < n - 1) v += xi - x[i + 1];
        y[i] = v * s;
      }
      __syncwarp();
      double* tmp = x;
      x = y;
      y = tmp;
    }
    if (k >= max_iter) break;
    // the last step of the block forms x^T (s L) x / x^T x and normalises
    double xy = 0.0, yy = 0.0, xn = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double xi = x[i];
      double v = 0.0;
      if (i > 0) v += xi - x[i - 1];
      if (i < n - 1) v += xi - x[i + 1];
      v *= s;
      y[i] = v;
      xy = fma(xi, v, xy);
      yy = fma(v, v, yy);
      xn = fma(xi, xi, xn);
    }
    xy = warp_sum(xy);
    yy = warp_sum(yy);
    xn = warp_sum(xn);
    ++k;
    if (!(yy > 0.0) || !(xn > 0.0)) break;
    rq = xy / xn;
    const double inv = 1.0 / sqrt(yy);
    __syncwarp();
    for (int i = lane; i < n; i += 32) x[i] = y[i] * inv;
    __syncwarp();
    if (rq_ref >= 0.0 && rq - rq_ref <= 1e-15 * fabs(rq)) {
      conv = 1;
      break;
    }
    rq_ref = rq;
  }
  if (lane == 0) {
    out->value[1 + axis] = rq;
    out->iters[1 + axis] = k;
    out->converged[1 + axis] = conv;
  }
}

struct AxisSet {
  int len[3];
  int axis[3];     // which grid axis each iterated block handles
  int cap[3];      // iteration cap of each
  int count;
};

__global__ void __launch_bounds__(kThreads) power_kernel(const double* __restrict__ A, int n,
                                                         double* __restrict__ xg,
                                                         double* __restrict__ yg, AxisSet axes,
                                                         double s, int max_gram,
                                                         PowerOut* out) {
  extern __shared__ double sh[];
  if (blockIdx.x == 0) {
    power_gram(A, n, xg, yg, max_gram, out);
    return;
  }
  const int b = blockIdx.x - 1;
  if (b >= axes.count || threadIdx.x >= 32) return;
  const int len = axes.len[b];
  power_axis(len, s, axes.axis[b], axes.cap[b], sh, sh + len, out);
}

}  // namespace

// lambda_max of K^T K (from the Gram matrix A, n x n, of the smaller side; A is read, not
// modified) and of D^T D on the plan's box grid, each by power iteration; stored in the
// plan (pl->kk_power, pl->dtd_power, pl->hess_power, pl->power_iters, pl->power_conv).
// Synchronises `s`.
ssm_status hessian_power(ssm_plan_s* pl, const double* A, int n, cudaStream_t s) {
  AxisSet axes{};
  const int naxes = pl->g.zlink ? pl->p.ndim : std::min(pl->p.ndim, 2);
  bool skipped_axis = false;
  for (int d = 0; d < naxes; ++d) {
    const int64_t len = pl->p.dims[d];
    if (len < 2) continue;
    if (len > kMaxAxis) {
      // not iterated: the result leaves this axis out and is reported as not converged
      skipped_axis = true;
      continue;
    }
    axes.len[axes.count] = (int)len;
    axes.axis[axes.count] = d;
    // an axis of n voxels contracts by about 1 - (pi/n)^2 per step (~25k steps for 128
    // voxels, ~100k for 256); the cap bounds each axis to 2^25 element updates
    axes.cap[axes.count] = (int)std::min<int64_t>(262144, ((int64_t)1 << 25) / len);
    ++axes.count;
  }
  int maxlen = 0;
  for (int i = 0; i < axes.count; ++i) maxlen = std::max(maxlen, axes.len[i]);
  double* buf = nullptr;
  const size_t nbuf = (size_t)2 * n + (sizeof(PowerOut) + 7) / 8;
  SSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(double) * nbuf, s));
  PowerOut* dout = reinterpret_cast<PowerOut*>(buf + 2 * n);
  SSM_CUDA(cudaMemsetAsync(dout, 0, sizeof(PowerOut), s));
  const size_t shm = sizeof(double) * 2 * (size_t)std::max(maxlen, 1);
  if (shm > 48 * 1024)
    SSM_CUDA(cudaFuncSetAttribute(power_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shm));
  const double sc = pl->p.stencil_pairs == 2 ? 2.0 : 1.0;
  // the Gram iteration contracts by (sigma_2/sigma_1)^2 per step
  power_kernel<<<1 + axes.count, kThreads, shm, s>>>(A, n, buf, buf + n, axes, sc, 4096, dout);
  SSM_LAUNCHED();
  PowerOut h{};
  SSM_CUDA(cudaMemcpyAsync(&h, dout, sizeof(PowerOut), cudaMemcpyDeviceToHost, s));
  SSM_CUDA(cudaFreeAsync(buf, s));
  SSM_CUDA(cudaStreamSynchronize(s));
  pl->kk_power = h.value[0];
  double dtd = 0.0;
  int iters = h.iters[0];
  bool conv = h.converged[0] != 0 && !skipped_axis;
  for (int i = 0; i < axes.count; ++i) {
    dtd += h.value[1 + axes.axis[i]];
    iters = std::max(iters, h.iters[1 + axes.axis[i]]);
    conv = conv && h.converged[1 + axes.axis[i]] != 0;
  }
  pl->dtd_power = dtd;
  pl->hess_power = pl->kk_power + pl->p.lambda * dtd;
  pl->power_iters = iters;
  pl->power_conv = conv ? 1 : 0;
  return SSM_OK;
}

}  // namespace ssm
