// FP64 iterations on the device for the largest eigenvalue of the Hessian of Eq. 7,
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
// of path-graph Laplacians, one per axis. Each factor gets its own FP64 iteration:
//   K^T K    power iteration on the plan's FP64 Gram matrix of the smaller side (K K^T has
//            the same nonzero spectrum). A step is a matrix-vector product spread over
//            the device (a warp per row) and a one-block normalisation; the host tests
//            the stopping rule every 32 steps.
//   s L_path power iteration on (sigma I - s L)^{-1} with sigma = 4 s (inverse iteration;
//            sigma lies above the path Laplacian's spectrum, whose largest eigenvalue is
//            s (2 + 2 cos(pi/n)) < 4 s). Its iterates converge to the same eigenvector as
//            plain power iteration on s L, but contract by about 1/4 per step instead of
//            1 - O(1/n^2): ~15 steps instead of tens of thousands for a 192-voxel axis.
//            A step is one tridiagonal solve (Thomas algorithm, one thread per axis).
// The start vectors are fixed pseudo-random values (a counter-based hash of the index).
// The Rayleigh quotient x^T A x / x^T x of the iterates (with A = K^T K, or s L itself)
// does not decrease; an iteration stops once it rises by at most 1e-15 of its value over
// a test interval (32 steps for the Gram factor, one for the axes), or at its cap, where
// it is reported as not converged (the value is then a lower bound of the eigenvalue).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

constexpr int kThreads = 256;
constexpr int kCheck = 32;                 // Gram steps between stopping tests
constexpr int kGramCap = 4096;             // Gram steps at most
constexpr int kAxisCap = 200;              // inverse-iteration steps at most
constexpr int64_t kMaxAxis = (int64_t)1 << 22;   // longest axis iterated

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

// block-wide sums of two values (kThreads threads), the same order every call
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

struct PowerOut {
  double value[4];     // [0] K^T K, [1..3] s L of axis 0..2
  int iters[4];
  int converged[4];
};

// x = start vector / its norm (one block)
__global__ void __launch_bounds__(kThreads) gram_start_kernel(double* __restrict__ x, int n) {
  __shared__ double red[kThreads / 32][2];
  double xx = 0.0, dummy = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const double v = start_value(i, 0);
    x[i] = v;
    xx += v * v;
  }
  block_sum2(xx, dummy, red);
  const double inv = 1.0 / sqrt(xx);
  for (int i = threadIdx.x; i < n; i += kThreads) x[i] *= inv;
}

// y = A x, a warp per row (rows grid-strided), lanes striding the columns (coalesced)
__global__ void __launch_bounds__(kThreads) gram_matvec_kernel(const double* __restrict__ A,
                                                               int n,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
  for (int64_t i = blockIdx.x * (int64_t)(kThreads / 32) + (threadIdx.x >> 5); i < n; i += warps) {
    const double* row = A + i * n;
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc = fma(row[j], x[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[i] = acc;
  }
}

// rq[step] = x^T y (x has unit norm, y = A x); x = y / ||y|| (one block). A zero y
// (A x = 0: the largest eigenvalue is 0) records rq = 0 and leaves x alone.
__global__ void __launch_bounds__(kThreads) gram_normalise_kernel(double* __restrict__ x,
                                                                  const double* __restrict__ y,
                                                                  int n, double* __restrict__ rq,
                                                                  int step) {
  __shared__ double red[kThreads / 32][2];
  double xy = 0.0, yy = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    xy = fma(x[i], y[i], xy);
    yy = fma(y[i], y[i], yy);
  }
  block_sum2(xy, yy, red);
  if (threadIdx.x == 0) rq[step] = yy > 0.0 ? xy : 0.0;
  if (!(yy > 0.0)) return;
  const double inv = 1.0 / sqrt(yy);
  for (int i = threadIdx.x; i < n; i += kThreads) x[i] = y[i] * inv;
}

struct AxisSet {
  int len[3];
  int axis[3];       // which grid axis each entry is
  int64_t base[3];   // offset of its scratch (4 arrays of len doubles)
  int count;
};

// one thread per axis: inverse iteration x <- (sigma I - s L)^{-1} x, sigma = 4 s, on the
// path of n voxels with the free boundary (diagonal of s L: s deg, off-diagonals -s).
// The tridiagonal system is factored once (Thomas: cp = modified super-diagonal,
// im = reciprocal pivots) and each step is one forward and one backward sweep; the
// Rayleigh quotient is formed with s L itself.
__global__ void axis_inverse_kernel(AxisSet axes, double s, double* __restrict__ scratch,
                                    PowerOut* __restrict__ out) {
  const int b = blockIdx.x;
  if (b >= axes.count || threadIdx.x != 0) return;
  const int n = axes.len[b];
  double* x = scratch + axes.base[b];
  double* y = x + n;
  double* cp = y + n;
  double* im = cp + n;
  const double sigma = 4.0 * s, e = s;   // sigma I - s L: off-diagonals +s
  auto diag = [&](int i) { return sigma - s * (double)((i > 0) + (i < n - 1)); };
  // factor
  double m = diag(0);
  im[0] = 1.0 / m;
  cp[0] = e / m;
  for (int i = 1; i < n; ++i) {
    m = diag(i) - e * cp[i - 1];
    im[i] = 1.0 / m;
    cp[i] = e / m;
  }
  // start vector, unit norm
  double xx = 0.0;
  for (int i = 0; i < n; ++i) {
    x[i] = start_value(i, 1 + axes.axis[b]);
    xx += x[i] * x[i];
  }
  double inv = 1.0 / sqrt(xx);
  for (int i = 0; i < n; ++i) x[i] *= inv;
  double rq = 0.0, rq_prev = -1.0;
  int k = 0, conv = 0;
  while (k < kAxisCap) {
    // solve (sigma I - s L) y = x: forward sweep into y, backward in place
    y[0] = x[0] * im[0];
    for (int i = 1; i < n; ++i) y[i] = (x[i] - e * y[i - 1]) * im[i];
    for (int i = n - 2; i >= 0; --i) y[i] -= cp[i] * y[i + 1];
    ++k;
    // Rayleigh quotient of s L at y, and y / ||y|| as the next iterate
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n; ++i) {
      double ly = 0.0;
      if (i > 0) ly += y[i] - y[i - 1];
      if (i < n - 1) ly += y[i] - y[i + 1];
      num = fma(y[i], s * ly, num);
      den = fma(y[i], y[i], den);
    }
    if (!(den > 0.0)) break;
    rq = num / den;
    inv = 1.0 / sqrt(den);
    for (int i = 0; i < n; ++i) x[i] = y[i] * inv;
    if (rq_prev >= 0.0 && rq - rq_prev <= 1e-15 * fabs(rq)) {
      conv = 1;
      break;
    }
    rq_prev = rq;
  }
  out->value[1 + axes.axis[b]] = rq;
  out->iters[1 + axes.axis[b]] = k;
  out->converged[1 + axes.axis[b]] = conv;
}

}  // namespace

// lambda_max of K^T K (from the Gram matrix A, n x n, of the smaller side; A is read, not
// modified) and of D^T D on the plan's box grid; stored in the plan (pl->kk_power,
// pl->dtd_power, pl->hess_power, pl->power_iters, pl->power_conv). Synchronises `s`.
ssm_status hessian_power(ssm_plan_s* pl, const double* A, int n, cudaStream_t s) {
  AxisSet axes{};
  const int naxes = pl->g.zlink ? pl->p.ndim : std::min(pl->p.ndim, 2);
  bool skipped_axis = false;
  int64_t scratch_len = 0;
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
    axes.base[axes.count] = scratch_len;
    scratch_len += 4 * len;
    ++axes.count;
  }
  double* buf = nullptr;
  // Gram x, y and the Rayleigh quotients; the axes' scratch; the result record
  const size_t nbuf = (size_t)2 * n + kGramCap + (size_t)scratch_len + (sizeof(PowerOut) + 7) / 8;
  SSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(double) * nbuf, s));
  double* gx = buf;
  double* gy = gx + n;
  double* rq = gy + n;
  double* ax = rq + kGramCap;
  PowerOut* dout = reinterpret_cast<PowerOut*>(ax + scratch_len);
  auto fail = [&](ssm_status st) {
    cudaFreeAsync(buf, s);
    return st;
  };
  if (cudaMemsetAsync(dout, 0, sizeof(PowerOut), s) != cudaSuccess) return fail(SSM_ECUDA);
  const double sc = pl->p.stencil_pairs == 2 ? 2.0 : 1.0;
  if (axes.count > 0) {
    axis_inverse_kernel<<<axes.count, 32, 0, s>>>(axes, sc, ax, dout);
    SSM_LAUNCHED();
  }
  // Gram factor: blocks of kCheck steps, the stopping rule tested on the host between
  // blocks (the contraction per step is (sigma_2 / sigma_1)^2)
  gram_start_kernel<<<1, kThreads, 0, s>>>(gx, n);
  SSM_LAUNCHED();
  const unsigned mv_grid = (unsigned)std::max(1, std::min(4 * sm_count(), (n + 7) / 8));
  int k = 0, conv = 0;
  double kk = 0.0, ref = -1.0;
  std::vector<double> hrq(kCheck);
  while (k < kGramCap) {
    const int steps = std::min(kCheck, kGramCap - k);
    for (int t = 0; t < steps; ++t) {
      gram_matvec_kernel<<<mv_grid, kThreads, 0, s>>>(A, n, gx, gy);
      SSM_LAUNCHED();
      gram_normalise_kernel<<<1, kThreads, 0, s>>>(gx, gy, n, rq, k + t);
      SSM_LAUNCHED();
    }
    if (cudaMemcpyAsync(hrq.data(), rq + k, sizeof(double) * steps, cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(SSM_ECUDA);
    k += steps;
    kk = hrq[steps - 1];
    if (!(kk > 0.0)) {            // A x = 0
      kk = 0.0;
      conv = 1;
      break;
    }
    if (ref >= 0.0 && kk - ref <= 1e-15 * std::fabs(kk)) {
      conv = 1;
      break;
    }
    ref = kk;
  }
  PowerOut h{};
  if (cudaMemcpyAsync(&h, dout, sizeof(PowerOut), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(SSM_ECUDA);
  SSM_CUDA(cudaFreeAsync(buf, s));
  pl->kk_power = kk;
  double dtd = 0.0;
  int iters = k;
  bool ok = conv != 0 && !skipped_axis;
  for (int i = 0; i < axes.count; ++i) {
    dtd += h.value[1 + axes.axis[i]];
    iters = std::max(iters, h.iters[1 + axes.axis[i]]);
    ok = ok && h.converged[1 + axes.axis[i]] != 0;
  }
  pl->dtd_power = dtd;
  pl->hess_power = pl->kk_power + pl->p.lambda * dtd;
  pl->power_iters = iters;
  pl->power_conv = ok ? 1 : 0;
  return SSM_OK;
}

}  // namespace ssm
