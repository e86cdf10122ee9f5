// Algorithm 1: the three-split ADMM the paper compares Algorithm 2 against (Sec. II-C),
// FP32, on the GPU. Per iteration, from x = y = z = d_x = d_y = d_z = 0:
//     f    = (beta x + d_x + beta y + d_y + beta z + d_z) / (3 beta)
//     x    = M (g + beta f - d_x),      M = (K^T K + beta I)^{-1}
//     y    = max(0, f - d_y / beta)
//     z    = (lambda D^T D + beta I)^{-1} (beta f - d_z)
//     d_x -= beta (f - x);  d_y -= beta (f - y);  d_z -= beta (f - z)
// The estimate returned is y (nonnegative; at convergence f = x = y = z).
//
// x-step: as in the full-rank LADMM form, M g is large against M (beta f - d_x) in
// FP32, so h = M g is formed once per solve and x = h + M w with w = beta f - d_x (the
// FP32 SIMT GEMM sgemm_kernel).
// z-step: on the free-boundary box grid D^T D = s L, L the Kronecker sum of path-graph
// Laplacians, which the orthonormal DCT-II along each axis diagonalises: the path
// Laplacian of n nodes has eigenvectors c_k(j) = a_k cos(pi (j + 1/2) k / n) (a_0 =
// sqrt(1/n), a_k = sqrt(2/n)) and eigenvalues mu(k) = 2 - 2 cos(pi k / n). So
//     z = C^T diag(1 / (lambda s sum_d mu_d(k_d) + beta)) C r,   C = C_z (x) C_y (x) C_x,
// done map by map as one dense n_d x n_d transform per axis (axis_transform_kernel), a
// spectral scaling (scale_kernel) and the transposed transforms.
// Kernels per iteration: admm_pre (f, w, r, y, d_y), the GEMM, 2 x (axes longer than 1)
// transforms and the scaling, admm_post (x, d_x, d_z); the residual sums are formed by
// admm_pre and admm_post on test iterations.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

constexpr int EW = 256;      // threads of the elementwise kernels
constexpr int TL = 64;       // lines per CTA of the axis transform
constexpr int TK = 8;        // outputs per thread and k block
constexpr int TT = 256;      // threads of the axis transform (8 groups of 8 outputs)

// f, w = beta f - d_x, r = beta f - d_z, y' = max(0, f - d_y/beta), d_y' = d_y - beta (f - y')
// and, on test iterations, ||f - y'||^2, ||y' - y||^2, ||y'||^2 per block (partial row
// blockIdx.y * gridDim.x + blockIdx.x, 4 doubles per row)
template <bool CHECK>
__global__ void __launch_bounds__(EW) admm_pre_kernel(AdmmState st, int Q, Grid g, float beta,
                                                      double* __restrict__ partial) {
  const int64_t n = (int64_t)blockIdx.x * EW + threadIdx.x;
  const float inv3b = 1.f / (3.f * beta), inv_b = 1.f / beta;
  float s_fy = 0.f, s_dy = 0.f, s_y = 0.f;
  if (n < g.N) {
    for (int q = blockIdx.y; q < Q; q += gridDim.y) {
      const int64_t o = (int64_t)q * g.ld + n;
      const float x = st.x[o], y = st.y[o], z = st.z[o];
      const float dx = st.dx[o], dy = st.dy[o], dz = st.dz[o];
      const float f = (beta * x + dx + beta * y + dy + beta * z + dz) * inv3b;
      const float yn = fmaxf(0.f, f - dy * inv_b);
      st.f[o] = f;
      st.w[o] = beta * f - dx;
      st.r[o] = beta * f - dz;
      st.y[o] = yn;
      st.dy[o] = dy - beta * (f - yn);
      if (CHECK) {
        const float a = f - yn, b = yn - y;
        s_fy = fmaf(a, a, s_fy);
        s_dy = fmaf(b, b, s_dy);
        s_y = fmaf(yn, yn, s_y);
      }
    }
  }
  if (CHECK) {
    double v[3] = {s_fy, s_dy, s_y};
    __shared__ double red[EW / 32][3];
    for (int k = 0; k < 3; ++k)
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if ((threadIdx.x & 31) == 0)
      for (int k = 0; k < 3; ++k) red[threadIdx.x >> 5][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int w = 0; w < EW / 32; ++w) t += red[w][threadIdx.x];
      partial[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = t;
    }
  }
}

// x = h + acc, d_x' = d_x - beta (f - x), d_z' = d_z - beta (f - z) and, on test
// iterations, ||f - x||^2 and ||f - z||^2 per block
template <bool CHECK>
__global__ void __launch_bounds__(EW) admm_post_kernel(AdmmState st, const float* __restrict__ H,
                                                       const float* __restrict__ acc, int Q,
                                                       Grid g, float beta,
                                                       double* __restrict__ partial) {
  const int64_t n = (int64_t)blockIdx.x * EW + threadIdx.x;
  float s_fx = 0.f, s_fz = 0.f;
  if (n < g.N) {
    for (int q = blockIdx.y; q < Q; q += gridDim.y) {
      const int64_t o = (int64_t)q * g.ld + n;
      const float f = st.f[o], z = st.z[o];
      const float x = H[o] + acc[o];
      st.x[o] = x;
      st.dx[o] = st.dx[o] - beta * (f - x);
      st.dz[o] = st.dz[o] - beta * (f - z);
      if (CHECK) {
        const float a = f - x, b = f - z;
        s_fx = fmaf(a, a, s_fx);
        s_fz = fmaf(b, b, s_fz);
      }
    }
  }
  if (CHECK) {
    double v[2] = {s_fx, s_fz};
    __shared__ double red[EW / 32][2];
    for (int k = 0; k < 2; ++k)
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if ((threadIdx.x & 31) == 0)
      for (int k = 0; k < 2; ++k) red[threadIdx.x >> 5][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 2) {
      double t = 0.0;
      for (int w = 0; w < EW / 32; ++w) t += red[w][threadIdx.x];
      partial[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = t;
    }
  }
}

// in place: r(q, n) *= D(n), D = 1 / (lambda s sum_d mu_d(k_d) + beta) in the DCT basis
__global__ void __launch_bounds__(EW) scale_kernel(float* __restrict__ r,
                                                   const float* __restrict__ D, int Q, Grid g) {
  const int64_t n = (int64_t)blockIdx.x * EW + threadIdx.x;
  if (n >= g.N) return;
  const float dn = D[n];
  for (int q = blockIdx.y; q < Q; q += gridDim.y) r[(int64_t)q * g.ld + n] *= dn;
}

// Dense transform along one grid axis of every map: out(a, k, i) = sum_j T[k][j] in(a, j, i)
// for the element at q*ld + (a*n + j)*I + i (I = voxels below the axis). A CTA takes TL
// lines (a, i) of a map: it stages them (n values each) in shared memory with loads in
// memory order, each thread forms TK outputs k for two lines per k block (the transposed
// matrix Tt[j][k] is padded with zeros to 64 NKB columns, so a thread's TK coefficients
// of one j are two 16-byte broadcast loads), and the results return through shared
// memory so that the stores follow memory order too.
template <int NKB>
__global__ void __launch_bounds__(TT) axis_transform_kernel(const float* __restrict__ in,
                                                            float* __restrict__ out,
                                                            const float* __restrict__ Tt, int n,
                                                            int64_t I, int64_t lines, int Q,
                                                            int64_t ld) {
  extern __shared__ __align__(16) float sl[];   // TL x (n + 1)
  constexpr int kpad = 64 * NKB;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t l0 = (int64_t)blockIdx.x * TL;
  const int w = n + 1;
  for (int q = blockIdx.y; q < Q; q += gridDim.y) {
    const float* src = in + (int64_t)q * ld;
    float* dst = out + (int64_t)q * ld;
    __syncthreads();   // the previous map's results have been stored
    for (int t = threadIdx.x; t < TL * n; t += TT) {
      int l, j;
      if (I == 1) {
        l = t / n;
        j = t - l * n;
      } else {
        j = t / TL;
        l = t - j * TL;
      }
      const int64_t line = l0 + l;
      float v = 0.f;
      if (line < lines) {
        const int64_t a = line / I, i = line - a * I;
        v = src[(a * n + j) * I + i];
      }
      sl[l * w + j] = v;
    }
    __syncthreads();
    float res[NKB][2][TK];
#pragma unroll
    for (int kb = 0; kb < NKB; ++kb)
#pragma unroll
      for (int u = 0; u < TK; ++u) res[kb][0][u] = res[kb][1][u] = 0.f;
    const float* s0 = sl + lane * w;
    const float* s1 = sl + (lane + 32) * w;
    for (int j = 0; j < n; ++j) {
      const float v0 = s0[j], v1 = s1[j];
      const float* trow = Tt + (int64_t)j * kpad + grp * TK;
#pragma unroll
      for (int kb = 0; kb < NKB; ++kb) {
        const float4 c0 = __ldg(reinterpret_cast<const float4*>(trow + kb * 64));
        const float4 c1 = __ldg(reinterpret_cast<const float4*>(trow + kb * 64 + 4));
        const float c[TK] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int u = 0; u < TK; ++u) {
          res[kb][0][u] = fmaf(c[u], v0, res[kb][0][u]);
          res[kb][1][u] = fmaf(c[u], v1, res[kb][1][u]);
        }
      }
    }
    __syncthreads();   // every thread is done reading the staged lines
#pragma unroll
    for (int kb = 0; kb < NKB; ++kb)
#pragma unroll
      for (int u = 0; u < TK; ++u) {
        const int k = kb * 64 + grp * TK + u;
        if (k < n) {
          sl[lane * w + k] = res[kb][0][u];
          sl[(lane + 32) * w + k] = res[kb][1][u];
        }
      }
    __syncthreads();
    for (int t = threadIdx.x; t < TL * n; t += TT) {
      int l, j;
      if (I == 1) {
        l = t / n;
        j = t - l * n;
      } else {
        j = t / TL;
        l = t - j * TL;
      }
      const int64_t line = l0 + l;
      if (line < lines) {
        const int64_t a = line / I, i = line - a * I;
        dst[(a * n + j) * I + i] = sl[l * w + j];
      }
    }
  }
}

int ew_grid_y(int Q) { return std::min(Q, 64); }

template <int NKB>
ssm_status launch_axis(const float* in, float* out, const float* Tt, int n, int64_t I,
                       int64_t lines, int Q, int64_t ld, cudaStream_t s) {
  const size_t shm = sizeof(float) * (size_t)TL * (n + 1);
  const dim3 grid((unsigned)((lines + TL - 1) / TL), (unsigned)std::min(Q, 65535));
  axis_transform_kernel<NKB><<<grid, TT, shm, s>>>(in, out, Tt, n, I, lines, Q, ld);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status axis_transform(const ssm_plan_s* pl, const float* in, float* out, int axis, bool inverse,
                          cudaStream_t s) {
  const int64_t dims[3] = {pl->g.nx, pl->g.ny, pl->g.nz};
  const int n = (int)dims[axis];
  int64_t I = 1;
  for (int d = 0; d < axis; ++d) I *= dims[d];
  const int64_t lines = pl->g.N / n;
  const float* Tt = pl->adm_T[axis][inverse ? 1 : 0];
  switch ((n + 63) / 64) {
    case 1: return launch_axis<1>(in, out, Tt, n, I, lines, pl->Q, pl->g.ld, s);
    case 2: return launch_axis<2>(in, out, Tt, n, I, lines, pl->Q, pl->g.ld, s);
    case 3: return launch_axis<3>(in, out, Tt, n, I, lines, pl->Q, pl->g.ld, s);
    case 4: return launch_axis<4>(in, out, Tt, n, I, lines, pl->Q, pl->g.ld, s);
    default:
      set_error("ADMM form: grid axes longer than 256 are not supported");
      return SSM_EUNSUPPORTED;
  }
}

}  // namespace

// the transform matrices (orthonormal DCT-II and its transpose, stored as Tt[j][k] with
// the k dimension padded to a multiple of 64) and the spectral scaling D, formed in FP64
ssm_status admm_tables(ssm_plan_s* pl, std::vector<std::pair<float**, std::vector<float>>>* out) {
  const int64_t dims[3] = {pl->g.nx, pl->g.ny, pl->g.nz};
  std::vector<std::vector<double>> mu(3);
  for (int d = 0; d < 3; ++d) {
    const int n = (int)dims[d];
    mu[d].resize(n);
    const bool linked = d < 2 || pl->g.zlink;
    for (int k = 0; k < n; ++k) mu[d][k] = linked ? 2.0 - 2.0 * std::cos(M_PI * k / n) : 0.0;
    if (n == 1 || !linked) continue;
    if (n > 256) {
      set_error("ADMM form: grid axes longer than 256 are not supported");
      return SSM_EUNSUPPORTED;
    }
    const int kpad = 64 * ((n + 63) / 64);
    std::vector<float> fwd((size_t)n * kpad, 0.f), inv((size_t)n * kpad, 0.f);
    for (int k = 0; k < n; ++k) {
      const double a = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
      for (int j = 0; j < n; ++j) {
        const double c = a * std::cos(M_PI * (j + 0.5) * k / n);   // C[k][j]
        fwd[(size_t)j * kpad + k] = (float)c;                       // Tt_fwd[j][k] = C[k][j]
        inv[(size_t)k * kpad + j] = (float)c;                       // Tt_inv[k][j] = C[k][j]
      }
    }
    out->emplace_back(&pl->adm_T[d][0], std::move(fwd));
    out->emplace_back(&pl->adm_T[d][1], std::move(inv));
  }
  const double s = pl->lam_s;   // lambda * (stencil scale): lambda D^T D = lam_s L
  std::vector<float> D((size_t)pl->g.N);
  for (int64_t z = 0; z < dims[2]; ++z)
    for (int64_t y = 0; y < dims[1]; ++y)
      for (int64_t x = 0; x < dims[0]; ++x)
        D[(size_t)(x + dims[0] * (y + dims[1] * z))] =
            (float)(1.0 / (s * (mu[0][x] + mu[1][y] + mu[2][z]) + pl->p.beta));
  out->emplace_back(&pl->adm_D, std::move(D));
  return SSM_OK;
}

ssm_status admm_prepare() {
  const int shm = (int)(sizeof(float) * TL * (256 + 1));
  SSM_CUDA(cudaFuncSetAttribute(axis_transform_kernel<1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, shm));
  SSM_CUDA(cudaFuncSetAttribute(axis_transform_kernel<2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, shm));
  SSM_CUDA(cudaFuncSetAttribute(axis_transform_kernel<3>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, shm));
  SSM_CUDA(cudaFuncSetAttribute(axis_transform_kernel<4>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, shm));
  return SSM_OK;
}

int admm_partial_rows(const ssm_plan_s* pl) {
  return 2 * (int)(((pl->g.N + EW - 1) / EW) * ew_grid_y(pl->Q));
}

ssm_status admm_iteration(ssm_plan_s* pl, bool check, double* partial, int* nparts,
                          cudaStream_t s) {
  const AdmmState& st = pl->adm;
  const float beta = (float)pl->p.beta;
  const dim3 eg((unsigned)((pl->g.N + EW - 1) / EW), (unsigned)ew_grid_y(pl->Q));
  const int nb = (int)(eg.x * eg.y);
  if (check)
    admm_pre_kernel<true><<<eg, EW, 0, s>>>(st, pl->Q, pl->g, beta, partial);
  else
    admm_pre_kernel<false><<<eg, EW, 0, s>>>(st, pl->Q, pl->g, beta, partial);
  SSM_LAUNCHED();
  // x-step product: acc = M w
  SSM_TRY(sgemm(pl->Q, (int)pl->g.N, pl->Q, 1.f, pl->Mq32, pl->Qp, st.w, pl->g.ld, 0.f, pl->Acc,
                pl->g.ld, s));
  // z-step: forward transforms along every axis longer than 1, scaling, inverse transforms;
  // the data ping-pong between r and t and the last inverse writes z
  const int64_t dims[3] = {pl->g.nx, pl->g.ny, pl->g.nz};
  int axes[3], na = 0;
  for (int d = 0; d < 3; ++d)
    if (dims[d] > 1 && (d < 2 || pl->g.zlink)) axes[na++] = d;   // a slice stack: no z step
  if (na == 0) {
    // one voxel: D^T D = 0, z = r / beta
    SSM_CUDA(cudaMemcpyAsync(st.z, st.r, sizeof(float) * (size_t)pl->Q * pl->g.ld,
                             cudaMemcpyDeviceToDevice, s));
    scale_kernel<<<eg, EW, 0, s>>>(st.z, pl->adm_D, pl->Q, pl->g);
    SSM_LAUNCHED();
  } else {
    float* cur = st.r;
    float* other = st.t;
    for (int i = 0; i < na; ++i) {
      SSM_TRY(axis_transform(pl, cur, other, axes[i], false, s));
      std::swap(cur, other);
    }
    scale_kernel<<<eg, EW, 0, s>>>(cur, pl->adm_D, pl->Q, pl->g);
    SSM_LAUNCHED();
    for (int i = na - 1; i >= 0; --i) {
      float* dst = i == 0 ? st.z : other;
      SSM_TRY(axis_transform(pl, cur, dst, axes[i], true, s));
      other = cur;
      cur = dst;
    }
  }
  double* post = partial + (int64_t)nb * 4;
  if (check)
    admm_post_kernel<true><<<eg, EW, 0, s>>>(st, pl->H, pl->Acc, pl->Q, pl->g, beta, post);
  else
    admm_post_kernel<false><<<eg, EW, 0, s>>>(st, pl->H, pl->Acc, pl->Q, pl->g, beta, post);
  SSM_LAUNCHED();
  *nparts = nb;
  return SSM_OK;
}

}  // namespace ssm
