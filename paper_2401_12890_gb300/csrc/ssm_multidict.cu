// Spatially varying dictionaries (ssm_plan_multi): Algorithm 2 with each voxel's own
// dictionary in the f-step, as in the paper's fingerprinting experiment (Sec. IV-D: one
// dictionary per quantised B1 level, chosen per voxel).
//
// With a label c(n) per voxel the problem of Eq. 7 becomes
//     min_{F >= 0}  sum_n 1/2 ||m_n - K_{c(n)} f_n||^2 + lambda/2 ||D F||^2,
// and the splitting of Algorithm 2 is unchanged: the f-step is per voxel, so it takes the
// factors of the voxel's dictionary (Eq. 27, Eq. 28, each dictionary's rank by the rule of
// Sec. III-E), while the z-step (Eq. 31) and the dual step do not involve K. The
// iteration is the d-free recurrence of ssm_lowrank.cu with V, the weights and the
// projections S taken per voxel:
//     a_i = S_i / (beta + sigma_{c,i}^2) - W_{c,i} u_i,   u = V_c^T (beta z - d)
//     t   = z + V_c a
//     z'  = max(0, e1 z + c2 sum_nbr z + c3 V_c a)           (Eq. 31)
//     d'  = beta (t - z'),   u' = V_c^T beta (2 z' - t)
// Each dictionary is factorised by an ordinary single-dictionary plan (FP64 Gram matrix
// and cyclic Jacobi on the device); the ranks are padded to a common R (a multiple of 8,
// at most 32) with zero basis vectors and weights.
//
// Kernels: the projections S_i(n) = sigma_{c,i} u_{c,i}^T m_n with FP64 accumulation (one
// thread per voxel, the dictionary's factors read through the cache), and the iteration
// (one thread per voxel, one block per 128-voxel tile, every compartment of the voxel in
// turn): z and its neighbours are coalesced loads of the map-major state, the voxel's
// dictionary rows are 16-byte loads that voxels of one label share in L1. The state u is
// one R-vector per voxel (no partial sums: a block owns its tiles' whole spectra).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

constexpr int MT = 128;   // voxels per block

// S[i][n] = sum_p B[c(n)][p][i] m[p][n] (B holds sigma_{c,i} u_{c,i}, zero past r_c)
template <int R>
__global__ void __launch_bounds__(MT) multi_project_kernel(const double* __restrict__ B, int P,
                                                           const int32_t* __restrict__ labels,
                                                           const float* __restrict__ M,
                                                           int64_t ldm, int64_t N,
                                                           float* __restrict__ S, int64_t ld) {
  const int64_t n = blockIdx.x * (int64_t)MT + threadIdx.x;
  if (n >= N) return;
  const double* Bc = B + (int64_t)labels[n] * P * R;
  double acc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) acc[i] = 0.0;
  for (int p = 0; p < P; ++p) {
    const double m = (double)M[(int64_t)p * ldm + n];
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = fma(__ldg(Bc + (int64_t)p * R + i), m, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) S[(int64_t)i * ld + n] = (float)acc[i];
}

struct MultiArgs {
  const float* __restrict__ Zin;
  float* __restrict__ Zout;
  const float* __restrict__ Din;    // d^k (residual-test iterations)
  float* __restrict__ Dout;         // d^{k+1} (iterations before a test)
  const float* __restrict__ S;      // R x ld
  const float* __restrict__ Uin;    // u^k, R x ld
  float* __restrict__ Uout;         // u^{k+1}
  const float* __restrict__ V;      // ndict x Q x R  [c][q][i]
  const float* __restrict__ coefA;  // ndict x R: 1/(beta + sigma^2)
  const float* __restrict__ coefW;  // ndict x R: sigma^2/(beta^2 + beta sigma^2)
  const int32_t* __restrict__ labels;
  double* __restrict__ partial;     // 4 doubles per block (residual-test iterations)
  Grid g;
  int Q;
  float beta, inv_beta, xi, lam_s, inv_xb;
};

constexpr int VT = 32;    // voxels per tile of the iteration kernel (one per lane)
constexpr int WPB = 4;    // warps per block: each takes a quarter of the block's compartments

// tile t, segment g: block (g * ntiles + t) -- segment-major, so the blocks resident
// at one time walk the same compartments of neighbouring tiles (the +-nx, +-nx*ny
// neighbour rows are then L2 hits)
template <int R, bool CHECK>
__global__ void __launch_bounds__(VT * WPB) multi_iter_kernel(const MultiArgs a, int64_t ntiles,
                                                             int nseg) {
  __shared__ float sh_a[R][VT];           // a_i of the tile's voxels
  __shared__ float sh_u[WPB][R][VT];      // the warps' partial u', summed in warp order
  __shared__ double sh_red[WPB][3];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t tile = blockIdx.x % ntiles;
  const int seg = (int)(blockIdx.x / ntiles);
  const int Q = a.Q;
  const int q0 = (int)(((int64_t)Q * seg) / nseg);
  const int q1 = (int)(((int64_t)Q * (seg + 1)) / nseg);
  const int64_t ld = a.g.ld, N = a.g.N;
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const bool zl = nz > 1 && a.g.zlink;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t n = tile * VT + lane;
  const bool in = n < N;
  int c = 0;
  bool hxm = false, hxp = false, hym = false, hyp = false, hzm = false, hzp = false;
  if (in) {
    c = a.labels[n];
    const int x = (int)(n % nx);
    const int64_t t = n / nx;
    const int y = (int)(t % ny);
    const int zc = (int)(t / ny);
    hxm = x > 0;
    hxp = x < nx - 1;
    hym = y > 0;
    hyp = y < ny - 1;
    hzm = zl && zc > 0;
    hzp = zl && zc < nz - 1;
  }
  const float deg = (float)(hxm + hxp + hym + hyp + hzm + hzp);
  const float e1 = (a.xi + a.beta - a.lam_s * deg) * a.inv_xb;   // weight of z
  const float c2 = a.lam_s * a.inv_xb;                             // weight of sum_nbr z
  const float c3 = a.beta * a.inv_xb;                              // weight of V a

  // a_i = S_i/(beta + sigma_{c,i}^2) - W_{c,i} u_i, u summed over the tile's segments of
  // the previous iteration in segment order
  for (int i = warp; i < R; i += WPB) {
    float u = 0.f;
    const float* pt = a.Uin + (tile * nseg) * (int64_t)(R * VT) + i * VT + lane;
    for (int g = 0; g < nseg; ++g) u += pt[(int64_t)g * R * VT];
    sh_a[i][lane] = in ? a.S[(int64_t)i * ld + n] * __ldg(a.coefA + c * R + i) -
                             __ldg(a.coefW + c * R + i) * u
                       : 0.f;
  }
  __syncthreads();
  float2 av[R / 2];
#pragma unroll
  for (int i = 0; i < R / 2; ++i) av[i] = make_float2(sh_a[2 * i][lane], sh_a[2 * i + 1][lane]);
  float2 uacc[R / 2];
#pragma unroll
  for (int i = 0; i < R / 2; ++i) uacc[i] = make_float2(0.f, 0.f);
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;

  // this warp's compartments
  const int span = q1 - q0;
  const int qa = q0 + (span * warp) / WPB;
  const int qb = q0 + (span * (warp + 1)) / WPB;
  const float* Vc = a.V + (int64_t)c * Q * R;
  if (in) {
#pragma unroll 1
    for (int q = qa; q < qb; ++q) {
      const float* zr = a.Zin + (int64_t)q * ld;
      const float z = zr[n];
      float nb = 0.f;
      if (hxm) nb += zr[n - 1];
      if (hxp) nb += zr[n + 1];
      if (hym) nb += zr[n - nx];
      if (hyp) nb += zr[n + nx];
      if (hzm) nb += zr[n - plane];
      if (hzp) nb += zr[n + plane];
      const float4* v4 = reinterpret_cast<const float4*>(Vc + (int64_t)q * R);
      float4 vr[R / 4];
      float2 p0 = make_float2(0.f, 0.f), p1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < R / 4; ++i) {
        vr[i] = __ldg(v4 + i);
        p0 = __ffma2_rn(make_float2(vr[i].x, vr[i].y), av[2 * i], p0);
        p1 = __ffma2_rn(make_float2(vr[i].z, vr[i].w), av[2 * i + 1], p1);
      }
      const float va = (p0.x + p0.y) + (p1.x + p1.y);            // (V_c a)_q
      const float zn = fmaxf(0.f, fmaf(e1, z, fmaf(c2, nb, c3 * va)));
      const float t = z + va;
      const float w = a.beta * (2.f * zn - t);                     // beta z' - d'
      const float2 ww = make_float2(w, w);
#pragma unroll
      for (int i = 0; i < R / 4; ++i) {
        uacc[2 * i] = __ffma2_rn(make_float2(vr[i].x, vr[i].y), ww, uacc[2 * i]);
        uacc[2 * i + 1] = __ffma2_rn(make_float2(vr[i].z, vr[i].w), ww, uacc[2 * i + 1]);
      }
      const int64_t o = (int64_t)q * ld + n;
      a.Zout[o] = zn;
      if (a.Dout) a.Dout[o] = a.beta * (t - zn);
      if (CHECK) {
        const float f = t - a.Din[o] * a.inv_beta;                 // f^{k+1}
        const float e = zn - f, ch = zn - z;
        s1 = fmaf(e, e, s1);
        s2 = fmaf(ch, ch, s2);
        s3 = fmaf(zn, zn, s3);
      }
    }
  }
  // the block's partial u' for this segment: warps' sums added in warp order
#pragma unroll
  for (int i = 0; i < R / 2; ++i) {
    sh_u[warp][2 * i][lane] = uacc[i].x;
    sh_u[warp][2 * i + 1][lane] = uacc[i].y;
  }
  __syncthreads();
  float* po = a.Uout + (tile * nseg + seg) * (int64_t)(R * VT);
  for (int i = warp; i < R; i += WPB) {
    float u = 0.f;
#pragma unroll
    for (int w = 0; w < WPB; ++w) u += sh_u[w][i][lane];
    po[i * VT + lane] = in ? u : 0.f;
  }
  if (CHECK) {
    double d1 = s1, d2 = s2, d3 = s3;
    for (int o = 16; o > 0; o >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      d3 += __shfl_xor_sync(0xffffffffu, d3, o);
    }
    if (lane == 0) {
      sh_red[warp][0] = d1;
      sh_red[warp][1] = d2;
      sh_red[warp][2] = d3;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int w = 0; w < WPB; ++w) t += sh_red[w][threadIdx.x];
      a.partial[(int64_t)blockIdx.x * 4 + threadIdx.x] = t;
    }
  }
}

// Ball[c][p][i] = alpha_i Bp[p][i] for i < r (sigma_i u_i), 0 for r <= i < R
__global__ void multi_gather_b(const double* __restrict__ Bp, const double* __restrict__ alpha,
                               int P, int n, int r, int R, double* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)P * R) return;
  const int p = (int)(k / R), i = (int)(k % R);
  out[k] = i < r ? alpha[i] * Bp[(int64_t)p * n + i] : 0.0;
}

int64_t tiles_of(const ssm_plan_s* pl) { return (pl->g.N + VT - 1) / VT; }

}  // namespace

namespace {

template <int R>
int multi_blocks_per_sm() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_acquire);
  if (v != 0) return v;
  int b1 = 0, b2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, multi_iter_kernel<R, true>, VT * WPB, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, multi_iter_kernel<R, false>, VT * WPB, 0);
  v = std::max(1, std::min(b1, b2));
  cached.store(v, std::memory_order_release);
  return v;
}

#define SSM_MULTI_RANKS(X) X(4) X(8) X(12) X(16) X(20) X(24) X(28) X(32)

int bpsm_multi(int R) {
  switch (R) {
#define SSM_R(RR) \
  case RR:        \
    return multi_blocks_per_sm<RR>();
    SSM_MULTI_RANKS(SSM_R)
#undef SSM_R
    default:
      return 1;
  }
}

}  // namespace

int multi_padded_rank(int r) {
  if (r < 1 || r > kMaxMultiRank) return 0;
  return (r + 3) / 4 * 4;
}

// segments per tile: enough blocks to fill every resident slot twice, at least 8
// compartments per warp
int multi_segments(const ssm_plan_s* pl) {
  const int64_t ntiles = tiles_of(pl);
  const int64_t slots = 2 * (int64_t)sm_count() * bpsm_multi(pl->R);
  int64_t nseg = (slots + ntiles - 1) / ntiles;
  nseg = std::min<int64_t>(nseg, std::max(1, pl->Q / (8 * WPB)));
  if (const char* env = getenv("SSM_MULTI_SEGMENTS")) {   // launch-shape override for sweeps
    const long v = atol(env);
    if (v >= 1 && v <= 4096) nseg = v;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(nseg, pl->Q));
}

int64_t multi_grid(const ssm_plan_s* pl) { return tiles_of(pl) * pl->mseg; }

int64_t multi_state_floats(const ssm_plan_s* pl, int nseg) {
  return tiles_of(pl) * nseg * (int64_t)pl->R * VT;
}

ssm_status multi_gather_factors(const double* Bp, const double* alpha, int P, int n, int r, int R,
                                double* out, cudaStream_t s) {
  const int64_t total = (int64_t)P * R;
  multi_gather_b<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Bp, alpha, P, n, r, R, out);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status multi_project(const ssm_plan_s* pl, const float* M, int64_t ldm, cudaStream_t s) {
  const unsigned grid = (unsigned)((pl->g.N + MT - 1) / MT);
  switch (pl->R) {
#define SSM_R(RR)                                                                         \
  case RR:                                                                                \
    multi_project_kernel<RR><<<grid, MT, 0, s>>>(pl->B_multi, pl->P, pl->labels, M, ldm,  \
                                                 pl->g.N, pl->S, pl->g.ld);               \
    break;
    SSM_MULTI_RANKS(SSM_R)
#undef SSM_R
    default:
      set_error("spatially varying dictionaries: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status multi_iteration(ssm_plan_s* pl, int cur, bool check, bool write_d, double* partial,
                           int* nparts, cudaStream_t s) {
  MultiArgs a;
  a.Zin = pl->Z[cur];
  a.Zout = pl->Z[cur ^ 1];
  a.Din = pl->Dl[cur];
  a.Dout = write_d ? pl->Dl[cur ^ 1] : nullptr;
  a.S = pl->S;
  a.Uin = pl->U[cur];
  a.Uout = pl->U[cur ^ 1];
  a.V = pl->V32;
  a.coefA = pl->coefA;
  a.coefW = pl->coefW;
  a.labels = pl->labels;
  a.partial = partial;
  a.g = pl->g;
  a.Q = pl->Q;
  a.beta = (float)pl->p.beta;
  a.inv_beta = (float)(1.0 / pl->p.beta);
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  const int64_t ntiles = tiles_of(pl);
  const int64_t grid = ntiles * pl->mseg;
  *nparts = (int)grid;
  switch (pl->R) {
#define SSM_R(RR)                                                                      \
  case RR:                                                                             \
    if (check)                                                                         \
      multi_iter_kernel<RR, true><<<(unsigned)grid, VT * WPB, 0, s>>>(a, ntiles, pl->mseg); \
    else                                                                               \
      multi_iter_kernel<RR, false><<<(unsigned)grid, VT * WPB, 0, s>>>(a, ntiles, pl->mseg); \
    break;
    SSM_MULTI_RANKS(SSM_R)
#undef SSM_R
    default:
      set_error("spatially varying dictionaries: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
  SSM_LAUNCHED();
  return SSM_OK;
}

}  // namespace ssm
