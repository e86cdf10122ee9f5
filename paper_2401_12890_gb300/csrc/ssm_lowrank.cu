// One LADMM iteration of Algorithm 2 (rank-r f-step, Eq. 28) fused into one kernel.
//
// Per voxel n the paper's f-step is
//     c_n = g_n + beta z_n - d_n,   f_n = c_n/beta - sum_i W_i v_i (v_i^T c_n),
// W_i = sigma_i^2 / (beta^2 + beta sigma_i^2). Written literally in FP32, c_n/beta and
// the rank-r correction cancel (both ~ |g|/beta) and rounding is amplified by up to
// sigma_1^2/beta. This kernel evaluates the same f exactly rearranged. With
// g_n = V S_n (S_i = sigma_i u_i^T m_n, formed once in FP64) and V^T V = I,
//     f_n = z_n - d_n/beta + V a_n,
//     a_i = S_i/(beta + sigma_i^2) - W_i u_i,   u = V^T (beta z - d),
// none of whose terms is large against the result. u for the next iteration is
// accumulated while z^{k+1} and d^{k+1} are written, so one pass over the state does
// the whole iteration:
//     read  z^k (and its grid neighbours), d^k, a_n
//     f     = z - d/beta + sum_i V[q][i] a_i
//     z'    = max(0, (xi z - lambda s (deg z - sum_nbr z) + beta f + d)/(xi + beta))  (Eq. 31)
//     d'    = d - beta (z' - f)                                                     (step 11)
//     u'_i += V[q][i] (beta z' - d')
// D^T D z = s (deg(n) z_n - sum_{m adjacent} z_m): the free-boundary grid Laplacian,
// s = 2 for the literal Eq. 8.
//
// Mapping: a block owns 32 consecutive voxels (one per lane, coalesced) and QS warps
// split the Q compartments; the per-voxel sums u' are combined across warps through
// shared memory in a fixed order (deterministic). Traffic per state element and
// iteration: read z, d; write z', d' (16 B); neighbour reads hit L1/L2.
#include "ssm_internal.cuh"

namespace ssm {
namespace {

struct LowrankArgs {
  const float* __restrict__ Zin;
  const float* __restrict__ Din;
  float* __restrict__ Zout;
  float* __restrict__ Dout;
  const float* __restrict__ V;      // Q x R
  const float* __restrict__ S;      // R x ld
  const float* __restrict__ Uin;    // R x ld
  float* __restrict__ Uout;         // R x ld
  const float* __restrict__ coefA;  // R
  const float* __restrict__ coefW;  // R
  double* __restrict__ partial;     // 4 doubles per block (check iterations)
  Grid g;
  int Q, qchunk;
  float beta, inv_beta, xi, lam_s, inv_xb;
};

template <int R>
struct MaxThreads {
  static constexpr int value = R <= 24 ? 512 : (R <= 48 ? 256 : 128);
};

template <int R, bool CHECK>
__global__ void __launch_bounds__(MaxThreads<R>::value)
    lowrank_iter_kernel(LowrankArgs a) {
  extern __shared__ float smem[];
  const int lane = threadIdx.x;
  const int wy = threadIdx.y;
  const int QS = blockDim.y;
  const int64_t ld = a.g.ld;
  const int64_t tile0 = (int64_t)blockIdx.x * 32;
  const int64_t n = tile0 + lane;
  const bool valid = n < a.g.N;

  // a_i for the tile's 32 voxels, computed once per block
  for (int idx = wy * 32 + lane; idx < R * 32; idx += 32 * QS) {
    const int i = idx >> 5;
    const int64_t nn = tile0 + (idx & 31);
    float v = 0.f;
    if (nn < a.g.N)
      v = __ldg(a.S + i * ld + nn) * __ldg(a.coefA + i) - __ldg(a.coefW + i) * __ldg(a.Uin + i * ld + nn);
    smem[idx] = v;
  }
  __syncthreads();
  float av[R], acc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    av[i] = smem[i * 32 + lane];
    acc[i] = 0.f;
  }

  // grid coordinates and free-boundary neighbour flags
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  int x = 0, y = 0, zc = 0;
  if (valid) {
    x = (int)(n % nx);
    const int64_t t = n / nx;
    y = (int)(t % ny);
    zc = (int)(t / ny);
  }
  const bool hxm = x > 0, hxp = x < nx - 1;
  const bool hym = y > 0, hyp = y < ny - 1;
  const bool hzm = zc > 0, hzp = zc < nz - 1;
  const float deg = (float)(hxm + hxp + hym + hyp + hzm + hzp);

  const int q0 = wy * a.qchunk;
  const int q1 = min(a.Q, q0 + a.qchunk);
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if (valid) {
#pragma unroll 2
    for (int q = q0; q < q1; ++q) {
      const int64_t o = (int64_t)q * ld + n;
      const float z = __ldg(a.Zin + o);
      const float d = __ldg(a.Din + o);
      float nb = 0.f;
      if (hxm) nb += __ldg(a.Zin + o - 1);
      if (hxp) nb += __ldg(a.Zin + o + 1);
      if (hym) nb += __ldg(a.Zin + o - sy);
      if (hyp) nb += __ldg(a.Zin + o + sy);
      if (hzm) nb += __ldg(a.Zin + o - sz);
      if (hzp) nb += __ldg(a.Zin + o + sz);
      const float4* v4 = reinterpret_cast<const float4*>(a.V + (int64_t)q * R);
      float vr[R];
#pragma unroll
      for (int i = 0; i < R / 4; ++i) {
        const float4 t = __ldg(v4 + i);
        vr[4 * i] = t.x;
        vr[4 * i + 1] = t.y;
        vr[4 * i + 2] = t.z;
        vr[4 * i + 3] = t.w;
      }
      float f0 = 0.f, f1 = 0.f;
#pragma unroll
      for (int i = 0; i < R; i += 2) {
        f0 = fmaf(vr[i], av[i], f0);
        f1 = fmaf(vr[i + 1], av[i + 1], f1);
      }
      const float f = (z - d * a.inv_beta) + (f0 + f1);
      const float lap = deg * z - nb;
      const float zn = fmaxf(0.f, (a.xi * z - a.lam_s * lap + a.beta * f + d) * a.inv_xb);
      const float dn = d - a.beta * (zn - f);
      const float w = a.beta * zn - dn;
#pragma unroll
      for (int i = 0; i < R; ++i) acc[i] = fmaf(vr[i], w, acc[i]);
      a.Zout[o] = zn;
      a.Dout[o] = dn;
      if (CHECK) {
        const float e = zn - f, c = zn - z;
        s1 = fmaf(e, e, s1);
        s2 = fmaf(c, c, s2);
        s3 = fmaf(zn, zn, s3);
      }
    }
  }
  __syncthreads();
  // combine the QS partial projections per voxel (fixed order)
#pragma unroll
  for (int i = 0; i < R; ++i) smem[(wy * R + i) * 32 + lane] = acc[i];
  __syncthreads();
  for (int idx = wy * 32 + lane; idx < R * 32; idx += 32 * QS) {
    const int i = idx >> 5, l = idx & 31;
    float sum = 0.f;
    for (int y2 = 0; y2 < QS; ++y2) sum += smem[(y2 * R + i) * 32 + l];
    const int64_t nn = tile0 + l;
    if (nn < a.g.N) a.Uout[i * ld + nn] = sum;
  }
  if (CHECK) {
    double d1 = s1, d2 = s2, d3 = s3;
    for (int off = 16; off > 0; off >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, off);
      d2 += __shfl_xor_sync(0xffffffffu, d2, off);
      d3 += __shfl_xor_sync(0xffffffffu, d3, off);
    }
    __syncthreads();
    double* dsm = reinterpret_cast<double*>(smem);
    if (lane == 0) {
      dsm[wy * 3 + 0] = d1;
      dsm[wy * 3 + 1] = d2;
      dsm[wy * 3 + 2] = d3;
    }
    __syncthreads();
    if (wy == 0 && lane < 3) {
      double t = 0.0;
      for (int y2 = 0; y2 < QS; ++y2) t += dsm[y2 * 3 + lane];
      a.partial[(int64_t)blockIdx.x * 4 + lane] = t;
    }
  }
}

template <int R>
int qs_max() {
  return MaxThreads<R>::value / 32;
}

template <int R>
ssm_status launch_r(const LowrankArgs& args, bool check, int nblocks, int qs, cudaStream_t s) {
  const size_t shm = sizeof(float) * (size_t)R * 32 * qs;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(lowrank_iter_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         96 * 1024);
    cudaFuncSetAttribute(lowrank_iter_kernel<R, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    configured = true;
  }
  dim3 block(32, qs), grid(nblocks);
  if (check)
    lowrank_iter_kernel<R, true><<<grid, block, shm, s>>>(args);
  else
    lowrank_iter_kernel<R, false><<<grid, block, shm, s>>>(args);
  SSM_LAUNCHED();
  return SSM_OK;
}

// q-split: enough warps to fill the GPU (about 48 resident warps on each of the SMs),
// at least 16 compartments per warp, within the register budget of the rank.
int choose_qs(int64_t ntiles, int Q, int qsmax, int nsm) {
  const int64_t want = (int64_t)nsm * 48;
  int qs = 1;
  while (qs < qsmax && ntiles * qs < want && Q / (qs * 2) >= 16) qs *= 2;
  return qs;
}

int g_nsm = 0;

}  // namespace

int lowrank_max_partials(const ssm_plan_s* pl) { return (int)((pl->g.N + 31) / 32); }

ssm_status lowrank_iteration(ssm_plan_s* pl, int cur, bool check, double* partial, int* nparts,
                             cudaStream_t s) {
  if (g_nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (g_nsm <= 0) g_nsm = 148;
  }
  LowrankArgs a;
  a.Zin = pl->Z[cur];
  a.Din = pl->Dl[cur];
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.V = pl->V32;
  a.S = pl->S;
  a.Uin = pl->U[cur];
  a.Uout = pl->U[cur ^ 1];
  a.coefA = pl->coefA;
  a.coefW = pl->coefW;
  a.partial = partial;
  a.g = pl->g;
  a.Q = pl->Q;
  a.beta = (float)pl->p.beta;
  a.inv_beta = (float)(1.0 / pl->p.beta);
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  const int ntiles = lowrank_max_partials(pl);
  *nparts = ntiles;
  int qsmax = 1;
  switch (pl->R) {
#define SSM_QS(RR) \
  case RR:         \
    qsmax = qs_max<RR>(); \
    break;
    SSM_QS(4) SSM_QS(8) SSM_QS(12) SSM_QS(16) SSM_QS(20) SSM_QS(24) SSM_QS(28) SSM_QS(32)
    SSM_QS(40) SSM_QS(48) SSM_QS(56) SSM_QS(64)
#undef SSM_QS
    default:
      set_error("low-rank kernel: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
  const int qs = choose_qs(ntiles, pl->Q, qsmax, g_nsm);
  a.qchunk = (pl->Q + qs - 1) / qs;
  switch (pl->R) {
#define SSM_R(RR) \
  case RR:        \
    return launch_r<RR>(a, check, ntiles, qs, s);
    SSM_R(4) SSM_R(8) SSM_R(12) SSM_R(16) SSM_R(20) SSM_R(24) SSM_R(28) SSM_R(32)
    SSM_R(40) SSM_R(48) SSM_R(56) SSM_R(64)
#undef SSM_R
    default:
      set_error("low-rank kernel: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
}

}  // namespace ssm
