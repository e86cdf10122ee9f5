// The work-table iteration: Algorithm 2's low-rank iteration (Eq. 28, Eq. 31, the dual
// step) for one or several problems in one launch. A table lists (problem, voxel tile,
// compartment segment) entries, one per block; each problem has its own grid, Q, basis,
// weights and state (TableProblem). Two uses:
//  - spatially varying dictionaries (ssm_plan_multi; the fingerprinting experiment's
//    dictionary per B1 level, Sec. IV-D): one problem whose voxels carry labels, each
//    voxel's f-step taking its own dictionary's factors (Eq. 27, Eq. 28, each
//    dictionary's rank by the rule of Sec. III-E). With a label c(n) per voxel Eq. 7
//    becomes sum_n 1/2 ||m_n - K_{c(n)} f_n||^2 + lambda/2 ||D F||^2; the z-step and the
//    dual step do not involve K.
//  - groups of independent small problems of differing N, P and Q (ssm_group_*; serving's
//    small requests, no counterpart in the paper): one dictionary per problem.
//
// The iteration is the d-free recurrence of ssm_lowrank.cu with V, the weights and the
// projections S taken per voxel (dictionary c = c(n), or the problem's):
//     a_i = S_i / (beta + sigma_{c,i}^2) - W_{c,i} u_i,   u = V_c^T (beta z - d)
//     t   = z + V_c a
//     z'  = max(0, e1 z + c2 sum_nbr z + c3 V_c a)           (Eq. 31)
//     d'  = beta (t - z'),   u' = V_c^T beta (2 z' - t)
// Ranks are padded to a common R (a multiple of 4, at most 32) with zero basis vectors
// and weights, which adds exact zeros only: a problem's iterates do not depend on R.
//
// Kernels: the projections S_i(n) = sigma_{c,i} u_{c,i}^T m_n with FP64 accumulation (one
// thread per voxel, the factors read through the cache), and the iteration (one thread
// per voxel; a block is a tile of 32 voxels and a segment of the compartments, its four
// warps taking a quarter of the segment each). z and its neighbours are coalesced loads
// of the map-major state, four rows' loads in flight per warp; the voxel's basis rows are
// 16-byte loads through L1 (broadcasts when a warp's voxels share a dictionary). Each
// block writes its partial u' = V_c^T w (warps summed in warp order) to its (tile,
// segment) slot, and the next iteration sums a tile's slots in segment order: the
// iterates are deterministic and do not depend on the schedule or on the other problems
// of the table. Residual partial sums go to row blockIdx.x; a problem's rows are
// contiguous (its entries are), summed in row order.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

constexpr int MT = 128;          // voxels per block of the projection kernel
constexpr int VT = kTableTile;   // voxels per tile of the iteration kernel (one per lane)
constexpr int WPB = 4;           // warps per block: each takes a quarter of the segment

// S[i][n] = sum_p B[c(n)][p][i] m[p][n] (B holds sigma_{c,i} u_{c,i}, zero past r_c)
template <int R>
__global__ void __launch_bounds__(MT) table_project_kernel(const double* __restrict__ B, int P,
                                                           const int32_t* __restrict__ labels,
                                                           const float* __restrict__ M,
                                                           int64_t ldm, int64_t N,
                                                           float* __restrict__ S, int64_t ld) {
  const int64_t n = blockIdx.x * (int64_t)MT + threadIdx.x;
  if (n >= N) return;
  const double* Bc = B + (labels ? (int64_t)labels[n] * P * R : 0);
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

// resident blocks per SM the register budget is sized for. Capping registers lower
// (64 or 80 at R = 8) spilled and measured slower (159 us against 131 us) than four
// blocks of 128-register threads with four rows of loads in flight per warp
template <int R> constexpr int min_blocks() { return R <= 8 ? 4 : (R <= 16 ? 3 : 2); }

template <int R, bool CHECK>
__global__ void __launch_bounds__(VT * WPB, min_blocks<R>())
    table_iter_kernel(const TableProblem* __restrict__ probs, const int4* __restrict__ table,
                      int cur, int write_d, double* __restrict__ partial) {
  __shared__ float sh_a[R][VT];           // a_i of the tile's voxels
  __shared__ float sh_u[WPB][R][VT];      // the warps' partial u', summed in warp order
  __shared__ double sh_red[WPB][3];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int4 e = table[blockIdx.x];
  const TableProblem& P = probs[e.x];
  const int64_t tile = e.y;
  const int seg = e.z;
  const int nseg = P.nseg;
  const int Q = P.Q;
  const int q0 = (int)(((int64_t)Q * seg) / nseg);
  const int q1 = (int)(((int64_t)Q * (seg + 1)) / nseg);
  const Grid g = P.g;
  const int64_t ld = g.ld, N = g.N;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const bool zl = nz > 1 && g.zlink;
  const int64_t plane = (int64_t)nx * ny;
  const float beta = P.beta, inv_beta = P.inv_beta;
  const float* __restrict__ Zin = P.Z[cur];
  float* __restrict__ Zo = P.Z[cur ^ 1];
  const float* __restrict__ Din = P.D[cur];
  float* __restrict__ Do = write_d ? P.D[cur ^ 1] : nullptr;
  const float* __restrict__ Uin = P.U[cur];
  float* __restrict__ Uo = P.U[cur ^ 1];
  const int64_t n = tile * VT + lane;
  const bool in = n < N;
  int c = 0;
  bool hxm = false, hxp = false, hym = false, hyp = false, hzm = false, hzp = false;
  if (in) {
    c = P.labels ? P.labels[n] : 0;
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
  const float e1 = (P.xi + beta - P.lam_s * deg) * P.inv_xb;   // weight of z
  const float c2 = P.lam_s * P.inv_xb;                           // weight of sum_nbr z
  const float c3 = beta * P.inv_xb;                              // weight of V a

  // a_i = S_i/(beta + sigma_{c,i}^2) - W_{c,i} u_i, u summed over the tile's segments of
  // the previous iteration in segment order
  {
    // this warp's ranks i = warp + j WPB; slot by slot, their loads in flight together
    constexpr int RPW = R / WPB;
    static_assert(R % WPB == 0, "ranks are padded to a multiple of the warps per block");
    float us[RPW];
#pragma unroll
    for (int j = 0; j < RPW; ++j) us[j] = 0.f;
    const float* pt = Uin + (tile * nseg) * (int64_t)(R * VT) + warp * VT + lane;
    for (int k = 0; k < nseg; ++k) {
#pragma unroll
      for (int j = 0; j < RPW; ++j) us[j] += pt[((int64_t)k * R + j * WPB) * VT];
    }
#pragma unroll
    for (int j = 0; j < RPW; ++j) {
      const int i = warp + j * WPB;
      sh_a[i][lane] = in ? P.S[(int64_t)i * ld + n] * __ldg(P.coefA + c * R + i) -
                               __ldg(P.coefW + c * R + i) * us[j]
                         : 0.f;
    }
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
  // row pointers advance by ld (state) and R (basis) per compartment
  const int64_t nxl = nx;
  const float* zrow = Zin + (int64_t)qa * ld + n;
  // basis rows: [q][c][i], a compartment's rows of all dictionaries side by side (the
  // labels of a warp's voxels, quantised from a smooth field, are mostly neighbours)
  const int64_t vstep = (int64_t)P.ndict * (R / 4);   // float4s from row q to row q + 1
  const float4* vrow = reinterpret_cast<const float4*>(P.V + ((int64_t)qa * P.ndict + c) * R);
  float* zout = Zo + (int64_t)qa * ld + n;
  float* dout = Do ? Do + (int64_t)qa * ld + n : nullptr;
  const float* din = Din + (int64_t)qa * ld + n;
  // one compartment row: the z-step and dual step with the row's state loads done
  auto row = [&](int u, float z, float nb, float dk) {
    float4 vr[R / 4];
#pragma unroll
    for (int i = 0; i < R / 4; ++i) vr[i] = __ldg(vrow + u * vstep + i);
    float2 p0 = make_float2(0.f, 0.f), p1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < R / 4; ++i) {
      p0 = __ffma2_rn(make_float2(vr[i].x, vr[i].y), av[2 * i], p0);
      p1 = __ffma2_rn(make_float2(vr[i].z, vr[i].w), av[2 * i + 1], p1);
    }
    const float va = (p0.x + p0.y) + (p1.x + p1.y);              // (V_c a)_q
    const float zn = fmaxf(0.f, fmaf(e1, z, fmaf(c2, nb, c3 * va)));
    const float t = z + va;
    const float w = beta * (2.f * zn - t);                         // beta z' - d'
    const float2 ww = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < R / 4; ++i) {
      uacc[2 * i] = __ffma2_rn(make_float2(vr[i].x, vr[i].y), ww, uacc[2 * i]);
      uacc[2 * i + 1] = __ffma2_rn(make_float2(vr[i].z, vr[i].w), ww, uacc[2 * i + 1]);
    }
    const int64_t o = (int64_t)u * ld;
    zout[o] = zn;
    if (dout) dout[o] = beta * (t - zn);
    if (CHECK) {
      const float f = t - dk * inv_beta;                           // f^{k+1}
      const float er = zn - f, ch = zn - z;
      s1 = fmaf(er, er, s1);
      s2 = fmaf(ch, ch, s2);
      s3 = fmaf(zn, zn, s3);
    }
  };
  // the row's state loads (and d^k on residual-test iterations), issued together
  auto load = [&](int u, float& z, float& nb, float& dk) {
    const float* zr = zrow + (int64_t)u * ld;
    z = zr[0];
    dk = CHECK ? din[(int64_t)u * ld] : 0.f;
    nb = 0.f;
    if (hxm) nb += zr[-1];
    if (hxp) nb += zr[1];
    if (hym) nb += zr[-nxl];
    if (hyp) nb += zr[nxl];
    if (hzm) nb += zr[-plane];
    if (hzp) nb += zr[plane];
  };
  auto advance = [&](int k) {
    zrow += (int64_t)k * ld;
    zout += (int64_t)k * ld;
    if (dout) dout += (int64_t)k * ld;
    din += (int64_t)k * ld;
    vrow += k * vstep;
  };
  if (in) {
    // UR rows' state loads issued together (memory-level parallelism of a latency-bound
    // loop; one row at a time measured 184 us, two 145, four 131, eight 136 at R = 8 on
    // the 61-level fingerprinting stand-in)
    constexpr int UR = R <= 16 ? 4 : 2;
    int q = qa;
#pragma unroll 1
    for (; q + UR <= qb; q += UR) {
      float zv[UR], nbv[UR], dv[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) load(u, zv[u], nbv[u], dv[u]);
#pragma unroll
      for (int u = 0; u < UR; ++u) row(u, zv[u], nbv[u], dv[u]);
      advance(UR);
    }
#pragma unroll 1
    for (; q < qb; ++q) {
      float z, nb, dk;
      load(0, z, nb, dk);
      row(0, z, nb, dk);
      advance(1);
    }
  }
  // the block's partial u' for this segment: warps' sums added in warp order
#pragma unroll
  for (int i = 0; i < R / 2; ++i) {
    sh_u[warp][2 * i][lane] = uacc[i].x;
    sh_u[warp][2 * i + 1][lane] = uacc[i].y;
  }
  __syncthreads();
  float* po = Uo + (tile * nseg + seg) * (int64_t)(R * VT);
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
      partial[(int64_t)blockIdx.x * 4 + threadIdx.x] = t;
    }
  }
}

// out[k] = alpha_i Bp[p][i] for i < r (sigma_i u_i), 0 for r <= i < R; k = p R + i
__global__ void gather_b_kernel(const double* __restrict__ Bp, const double* __restrict__ alpha,
                                int P, int n, int r, int R, double* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)P * R) return;
  const int p = (int)(k / R), i = (int)(k % R);
  out[k] = i < r ? alpha[i] * Bp[(int64_t)p * n + i] : 0.0;
}

template <int R>
int blocks_per_sm_r() {
  static std::atomic<int> cached{0};
  int v = cached.load(std::memory_order_acquire);
  if (v != 0) return v;
  int b1 = 0, b2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, table_iter_kernel<R, true>, VT * WPB, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, table_iter_kernel<R, false>, VT * WPB, 0);
  v = std::max(1, std::min(b1, b2));
  cached.store(v, std::memory_order_release);
  return v;
}

#define SSM_TABLE_RANKS(X) X(4) X(8) X(12) X(16) X(20) X(24) X(28) X(32)

}  // namespace

int table_padded_rank(int r) {
  if (r < 1 || r > kMaxTableRank) return 0;
  return (r + 3) / 4 * 4;
}

int table_blocks_per_sm(int R) {
  switch (R) {
#define SSM_R(RR) \
  case RR:        \
    return blocks_per_sm_r<RR>();
    SSM_TABLE_RANKS(SSM_R)
#undef SSM_R
    default:
      return 1;
  }
}

// About four blocks per resident slot of an R-rank kernel (measured on the 61-level
// 156 x 156 stand-in: 1, 2, 3, 4, 6, 8, 12 segments gave 154, 131, 124, 123, 133, 129,
// 151 us: fewer leave slots idle in the last wave, more re-read the partial sums); at
// most 8, at least 8 compartments per warp. Depends on the problem's size and the
// device only, so a problem's iterates do not depend on the problems sharing its table.
int table_segments(int64_t ntiles, int Q, int R) {
  const int64_t slots = (int64_t)sm_count() * table_blocks_per_sm(R);
  int64_t nseg = (4 * slots + ntiles - 1) / ntiles;
  nseg = std::min<int64_t>(nseg, 8);
  nseg = std::min<int64_t>(nseg, std::max(1, Q / (8 * WPB)));
  if (const char* env = getenv("SSM_TABLE_SEGMENTS")) {   // launch-shape override for sweeps
    const long v = atol(env);
    if (v >= 1 && v <= 4096) nseg = v;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(nseg, Q));
}

int64_t table_state_floats(int64_t N, int nseg, int R) {
  return (N + VT - 1) / VT * nseg * (int64_t)R * VT;
}

void table_entries(int problem, int64_t ntiles, int nseg, std::vector<int4>* out) {
  for (int s = 0; s < nseg; ++s)
    for (int64_t t = 0; t < ntiles; ++t) out->push_back(make_int4(problem, (int)t, s, 0));
}

ssm_status table_gather_factors(const double* Bp, const double* alpha, int P, int n, int r, int R,
                                double* out, cudaStream_t s) {
  const int64_t total = (int64_t)P * R;
  gather_b_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Bp, alpha, P, n, r, R, out);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status table_project(const double* B, int P, int R, const int32_t* labels, const float* M,
                         int64_t ldm, int64_t N, float* S, int64_t ld, cudaStream_t s) {
  const unsigned grid = (unsigned)((N + MT - 1) / MT);
  switch (R) {
#define SSM_R(RR)                                                                          \
  case RR:                                                                                 \
    table_project_kernel<RR><<<grid, MT, 0, s>>>(B, P, labels, M, ldm, N, S, ld);          \
    break;
    SSM_TABLE_RANKS(SSM_R)
#undef SSM_R
    default:
      set_error("work-table iteration: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status table_iteration(const TableProblem* probs, const int4* table, int64_t nblocks, int R,
                           int cur, bool check, bool write_d, double* partial, cudaStream_t s) {
  if (nblocks < 1 || nblocks > INT32_MAX) {
    set_error("work-table iteration: bad table size");
    return SSM_EINVAL;
  }
  const unsigned grid = (unsigned)nblocks;
  const int wd = write_d ? 1 : 0;
  switch (R) {
#define SSM_R(RR)                                                                           \
  case RR:                                                                                  \
    if (check)                                                                              \
      table_iter_kernel<RR, true><<<grid, VT * WPB, 0, s>>>(probs, table, cur, wd, partial); \
    else                                                                                    \
      table_iter_kernel<RR, false><<<grid, VT * WPB, 0, s>>>(probs, table, cur, wd, partial); \
    break;
    SSM_TABLE_RANKS(SSM_R)
#undef SSM_R
    default:
      set_error("work-table iteration: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
  SSM_LAUNCHED();
  return SSM_OK;
}

}  // namespace ssm
