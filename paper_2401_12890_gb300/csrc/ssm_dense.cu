// Full-rank (Eq. 26) LADMM iteration in plain FP32, plus the kernels shared by every
// form: an FP32 SIMT matrix product, the residual reductions and the objective terms.
//
// Eq. 26 gives f_n = (K^T K + beta I)^{-1} (g_n + beta z_n - d_n). Applied literally in
// FP32 the large, nearly cancelling product M g_n dominates the rounding error, so
// the iteration uses the exact split
//     f = h + M w,   h = M g (formed once per solve),   w = beta z - d,
// and runs the Q x Q by Q x N contraction on w only. The update kernel then applies
// the z-step (Eq. 31 with the nonnegativity projection) and the dual step, and
// writes the next w (FP32 for this form, or the BF16 hi/lo pair for the tensor-core
// form), so one iteration is: sgemm (M w) -> dense_update.
#include "ssm_internal.cuh"

namespace ssm {
namespace {

// ---------------------------------------------------------------------------
// C (M x N) = alpha * A (M x K) B (K x N) + beta * C, all row-major FP32.
// 128 x 128 block tile, 8-deep k slices double-buffered in shared memory,
// 8 x 8 outputs per thread, FP32 accumulation.
// ---------------------------------------------------------------------------
constexpr int BM = 128, BN = 128, BK = 8;

__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, float alpha,
                                                    const float* __restrict__ A, int64_t lda,
                                                    const float* __restrict__ B, int64_t ldb,
                                                    float beta, float* __restrict__ C,
                                                    int64_t ldc) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // loader mapping: A tile 128 x 8 -> row tid/2, k (tid&1)*4..+4
  //                 B tile 8 x 128 -> k tid/32, col (tid&31)*4..+4
  const int ar = tid >> 1, ak = (tid & 1) * 4;
  const int bk = tid >> 5, bc = (tid & 31) * 4;
  float ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ar, gk = k0 + ak + j;
      ra[j] = (gm < M && gk < K) ? __ldg(A + (int64_t)gm * lda + gk) : 0.f;
      const int gk2 = k0 + bk, gn = n0 + bc + j;
      rb[j] = (gk2 < K && gn < N) ? __ldg(B + (int64_t)gk2 * ldb + gn) : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int j = 0; j < 4; ++j) As[buf][ak + j][ar] = ra[j];
    *reinterpret_cast<float4*>(&Bs[buf][bk][bc]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int ntile = (K + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < ntile; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ntile) load((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < ntile) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (gn >= N) continue;
      float* c = C + (int64_t)gm * ldc + gn;
      *c = beta == 0.f ? alpha * acc[i][j] : fmaf(alpha, acc[i][j], beta * *c);
    }
  }
}

// ---------------------------------------------------------------------------
// z-step (Eq. 31 + projection) and dual step for the full-rank form
//   f  = h + acc,  z' = max(0, (xi z - lambda s (deg z - sum_nbr z) + beta f + d)/(xi+beta))
//   d' = d - beta (z' - f),  w' = beta z' - d'
// block: 256 voxels x UQ compartments (loop); residual partials on check iterations.
// ---------------------------------------------------------------------------
constexpr int UV = 256, UQ = 8;

struct UpdateArgs {
  const float* __restrict__ acc;
  const float* __restrict__ H;
  const float* __restrict__ Zin;
  const float* __restrict__ Din;
  float* __restrict__ Zout;
  float* __restrict__ Dout;
  float* __restrict__ Wf;            // optional FP32 w'
  __nv_bfloat16* __restrict__ Whi;   // optional BF16 split of w'
  __nv_bfloat16* __restrict__ Wlo;
  double* __restrict__ partial;
  const uint8_t* __restrict__ mask;  // voxels inside the object (nullptr: every voxel)
  Grid g;
  int Q;
  float beta, xi, lam_s, inv_xb;
};

template <bool CHECK>
__global__ void __launch_bounds__(UV) dense_update_kernel(UpdateArgs a) {
  const int64_t n = (int64_t)blockIdx.x * UV + threadIdx.x;
  const uint8_t* mk = a.mask;
  const bool valid = n < a.g.N && (!mk || mk[n]);   // outside the object: left alone
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny, ld = a.g.ld;
  int x = 0, y = 0, zc = 0;
  if (valid) {
    x = (int)(n % nx);
    const int64_t t = n / nx;
    y = (int)(t % ny);
    zc = (int)(t / ny);
  }
  const int64_t sy_ = nx, sz_ = (int64_t)nx * ny;
  const bool hxm = valid && x > 0 && (!mk || mk[n - 1]);
  const bool hxp = valid && x < nx - 1 && (!mk || mk[n + 1]);
  const bool hym = valid && y > 0 && (!mk || mk[n - sy_]);
  const bool hyp = valid && y < ny - 1 && (!mk || mk[n + sy_]);
  const bool hzm = a.g.zlink && valid && zc > 0 && (!mk || mk[n - sz_]);
  const bool hzp = a.g.zlink && valid && zc < nz - 1 && (!mk || mk[n + sz_]);
  const float deg = (float)(hxm + hxp + hym + hyp + hzm + hzp);
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;
  const int q0 = blockIdx.y * UQ, q1 = min(a.Q, q0 + UQ);
  if (valid) {
    for (int q = q0; q < q1; ++q) {
      const int64_t o = (int64_t)q * ld + n;
      const float z = __ldg(a.Zin + o), d = __ldg(a.Din + o);
      float nb = 0.f;
      if (hxm) nb += __ldg(a.Zin + o - 1);
      if (hxp) nb += __ldg(a.Zin + o + 1);
      if (hym) nb += __ldg(a.Zin + o - sy);
      if (hyp) nb += __ldg(a.Zin + o + sy);
      if (hzm) nb += __ldg(a.Zin + o - sz);
      if (hzp) nb += __ldg(a.Zin + o + sz);
      const float f = __ldg(a.H + o) + __ldg(a.acc + o);
      const float zn = fmaxf(0.f, (a.xi * z - a.lam_s * (deg * z - nb) + a.beta * f + d) * a.inv_xb);
      const float dn = d - a.beta * (zn - f);
      const float w = a.beta * zn - dn;
      a.Zout[o] = zn;
      a.Dout[o] = dn;
      if (a.Wf) a.Wf[o] = w;
      if (a.Whi) {
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        a.Whi[o] = h;
        a.Wlo[o] = __float2bfloat16_rn(w - __bfloat162float(h));
      }
      if (CHECK) {
        const float e = zn - f, c = zn - z;
        s1 = fmaf(e, e, s1);
        s2 = fmaf(c, c, s2);
        s3 = fmaf(zn, zn, s3);
      }
    }
  }
  if (CHECK) {
    double d1 = s1, d2 = s2, d3 = s3;
    for (int off = 16; off > 0; off >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, off);
      d2 += __shfl_xor_sync(0xffffffffu, d2, off);
      d3 += __shfl_xor_sync(0xffffffffu, d3, off);
    }
    __shared__ double sm[UV / 32][3];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      sm[w][0] = d1;
      sm[w][1] = d2;
      sm[w][2] = d3;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int k = 0; k < UV / 32; ++k) t += sm[k][threadIdx.x];
      a.partial[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = t;
    }
  }
}

// sum `nparts` rows of `width` doubles (row stride 4) in a fixed order
__global__ void finish_kernel(const double* __restrict__ part, int nparts, int width,
                              double* __restrict__ out) {
  __shared__ double sm[32][4];
  double acc[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < nparts; i += blockDim.x)
    for (int j = 0; j < width; ++j) acc[j] += part[(int64_t)i * 4 + j];
  for (int j = 0; j < width; ++j)
    for (int off = 16; off > 0; off >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], off);
  if ((threadIdx.x & 31) == 0)
    for (int j = 0; j < width; ++j) sm[threadIdx.x >> 5][j] = acc[j];
  __syncthreads();
  if (threadIdx.x < width) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w][threadIdx.x];
    out[threadIdx.x] = t;
  }
}

// objective pieces: sum over the residual rows of r^2, and sum over every unordered
// neighbour pair and every map of (F_n - F_m)^2 (the forward differences)
__global__ void __launch_bounds__(UV) objective_kernel(const float* __restrict__ Res, int P,
                                                       const float* __restrict__ F, int64_t ldf,
                                                       int Q, Grid g,
                                                       const uint8_t* __restrict__ mk,
                                                       double* __restrict__ part) {
  const int64_t n = (int64_t)blockIdx.x * UV + threadIdx.x;
  double r2 = 0.0, e2 = 0.0;
  // with a mask: the data term over the voxels inside, the pairs with both ends inside
  if (n < g.N && (!mk || mk[n])) {
    for (int p = 0; p < P; ++p) {
      const float r = Res[(int64_t)p * g.ld + n];
      r2 += (double)r * r;
    }
    const int x = (int)(n % g.nx);
    const int64_t t = n / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    for (int q = 0; q < Q; ++q) {
      const float* row = F + (int64_t)q * ldf;
      const float v = row[n];
      float acc = 0.f;
      if (x + 1 < g.nx && (!mk || mk[n + 1])) {
        const float dd = v - row[n + 1];
        acc = fmaf(dd, dd, acc);
      }
      if (y + 1 < g.ny && (!mk || mk[n + sy])) {
        const float dd = v - row[n + sy];
        acc = fmaf(dd, dd, acc);
      }
      if (g.zlink && z + 1 < g.nz && (!mk || mk[n + sz])) {
        const float dd = v - row[n + sz];
        acc = fmaf(dd, dd, acc);
      }
      e2 += acc;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, off);
    e2 += __shfl_xor_sync(0xffffffffu, e2, off);
  }
  __shared__ double sm[UV / 32][2];
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5][0] = r2;
    sm[threadIdx.x >> 5][1] = e2;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < UV / 32; ++w) t += sm[w][threadIdx.x];
    part[(int64_t)blockIdx.x * 4 + threadIdx.x] = t;
  }
}

}  // namespace

ssm_status sgemm(int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                 int64_t ldb, float beta, float* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return SSM_OK;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  sgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  SSM_LAUNCHED();
  return SSM_OK;
}

int dense_max_partials(const ssm_plan_s* pl) {
  return (int)(((pl->g.N + UV - 1) / UV) * ((pl->Q + UQ - 1) / UQ));
}

ssm_status dense_update(ssm_plan_s* pl, int cur, const float* acc, bool check, bool write_fp32_w,
                        bool write_bf16_w, double* partial, int* nparts, cudaStream_t s) {
  UpdateArgs a;
  a.acc = acc;
  a.H = pl->H;
  a.Zin = pl->Z[cur];
  a.Din = pl->Dl[cur];
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.Wf = write_fp32_w ? pl->Wf : nullptr;
  a.Whi = write_bf16_w ? pl->Whi[cur ^ 1] : nullptr;
  a.Wlo = write_bf16_w ? pl->Wlo[cur ^ 1] : nullptr;
  a.partial = partial;
  a.mask = pl->mask;
  a.g = pl->g;
  a.Q = pl->Q;
  a.beta = (float)pl->p.beta;
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  dim3 grid((unsigned)((pl->g.N + UV - 1) / UV), (unsigned)((pl->Q + UQ - 1) / UQ));
  *nparts = (int)(grid.x * grid.y);
  if (check)
    dense_update_kernel<true><<<grid, UV, 0, s>>>(a);
  else
    dense_update_kernel<false><<<grid, UV, 0, s>>>(a);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status finish_partials(const double* partial, int nparts, int width, double* out,
                           cudaStream_t s) {
  finish_kernel<<<1, 1024, 0, s>>>(partial, nparts, width, out);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status objective_terms(const ssm_plan_s* pl, const float* Res, int P, const float* F,
                           int64_t ldf, double* partial, int* nparts, cudaStream_t s) {
  const unsigned nb = (unsigned)((pl->g.N + UV - 1) / UV);
  objective_kernel<<<nb, UV, 0, s>>>(Res, P, F, ldf, pl->Q, pl->g, pl->mask, partial);
  SSM_LAUNCHED();
  *nparts = (int)nb;
  return SSM_OK;
}

}  // namespace ssm
