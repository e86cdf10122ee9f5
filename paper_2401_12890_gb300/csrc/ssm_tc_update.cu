// The bandwidth-bound half of the tensor-core full-rank iteration (the product M w is
// tc_gemm_kernel in ssm_tc.cu):
//     f  = h + acc
//     z' = max(0, (xi z - lambda s (deg z - sum_nbr z) + beta f + d) / (xi + beta))  (Eq. 31)
//     d' = d - beta (z' - f)                                                      (step 11)
//     w' = beta z' - d'   -> the BF16 pair (hi, lo), voxel-major, for the next product
#include <algorithm>

#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

namespace ssm {
namespace {

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// tc_update_kernel: the z-step, dual step and next-w split, TMA-staged (HBM-bound).
// Work items are (16-compartment chunk, voxel tile of 128) pairs ordered chunk-major and
// dealt round-robin to the CTAs (item c to CTA c mod G), so the CTAs running at the same
// time hold the same compartments of consecutive tiles: the -+nx and -+nx*ny halo rows
// one CTA loads are the rows the CTAs of the neighbouring tiles load at about the same
// time (L2 hits). One producer warp streams z (x halo), its neighbour rows, d, h and acc
// for each item with 2D TMA boxes into a 2-stage mbarrier ring; the consumer warps (8
// on 1D/2D grids, 16 on 3D grids) each own 32 voxels and one group of the chunk's
// compartments (8, or 4), store z' and d' (coalesced) and the group's new w values of
// each voxel as one 16- (8-) byte BF16 store each for hi and lo; the parts of a voxel's
// 32-byte sector are written by warps of the same CTA moments apart, so L2 merges them
// before writing the sector back.
constexpr int UTV = 128, UQC = 16, UNB = 2;
// consumer warps: 8 (2 compartment groups) on 1D/2D grids, 16 (4 groups) on 3D grids,
// whose larger stage leaves room for one CTA per SM only
template <int NCW>
struct UWarps {
  static constexpr int QG = NCW / 4;        // compartment groups of the chunk
  static constexpr int QH = UQC / QG;       // compartments per consumer warp
  static constexpr int NT = 32 * (NCW + 1); // + the producer warp
};
constexpr int UZW = UTV + 8, UNW = UTV + 4;

struct UpdMaps {
  CUtensorMap zc, zn, d, h, acc;
};

struct UpdArgs {
  float* __restrict__ Zout;
  float* __restrict__ Dout;
  __nv_bfloat16* __restrict__ Whi;
  __nv_bfloat16* __restrict__ Wlo;
  double* __restrict__ partial;
  const uint8_t* __restrict__ mask;   // voxels inside the object (nullptr: every voxel)
  int* __restrict__ err;
  Grid g;
  int Q, Qp, nqc;              // nqc = chunks per tile
  int64_t ntiles, T;           // voxel tiles, total (chunk, tile) items
  float beta, xi, lam_s, inv_xb;
};

struct ULayout {
  int zc, zn, dd, hh, aa, stage, bars, total;
  __host__ __device__ ULayout(int NR) {
    auto al = [](int b) { return (b + 127) / 128 * 128; };
    zc = 0;
    zn = al(UQC * UZW * 4);
    dd = al(zn + NR * UQC * UNW * 4);
    hh = dd + UQC * UTV * 4;
    aa = hh + UQC * UTV * 4;
    stage = al(aa + UQC * UTV * 4);
    bars = UNB * stage;
    total = bars + 4 * UNB * 8;
  }
};

__host__ __device__ __forceinline__ int64_t ufloor4(int64_t v) {
  return v >= 0 ? (v & ~(int64_t)3) : -(((-v) + 3) & ~(int64_t)3);
}

template <bool CHECK, int UNCW, bool MASKED>
__global__ void __launch_bounds__(UWarps<UNCW>::NT) tc_update_kernel(
    const __grid_constant__ UpdMaps maps, const UpdArgs a) {
  constexpr int UQH = UWarps<UNCW>::QH, UNT = UWarps<UNCW>::NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // aligned through an integer, so the staged-row reads compile as generic loads: the
  // shared-address form (an offset from smem_raw, as the other TMA-fed kernels use) ran
  // 8 % slower here (207 -> 224 us per launch on the 128x128, Q = 2500 workload)
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ld = a.g.ld, N = a.g.N;
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const bool zl = nz > 1 && a.g.zlink;   // z neighbours coupled
  const int NR = (ny > 1 ? 2 : 0) + (zl ? 2 : 0);
  const ULayout L(NR);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + UNB;
  // (the order matches the neighbour flags: y pair first when the grid has a y axis)
  const int64_t plane = (int64_t)nx * ny;
  const int64_t off[4] = {ny > 1 ? -(int64_t)nx : -plane, ny > 1 ? (int64_t)nx : plane, -plane,
                          plane};
  const int64_t G = gridDim.x;
  const unsigned stage_bytes = (unsigned)(UQC * UZW * 4 + NR * UQC * UNW * 4 + 3 * UQC * UTV * 4);
  if (tid == 0) {
    for (int b = 0; b < UNB; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], UNCW);
    }
    mbar_fence_init();
  }
  __syncthreads();
  bool failed = false;
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if (warp == UNCW) {
    if (lane == 0) {
      tma_prefetch_map(&maps.zc);
      for (int64_t c = blockIdx.x; c < a.T; c += G) {
        const int i = (int)((c - blockIdx.x) / G), b = i % UNB, k = i / UNB;
        if (i >= UNB && !mbar_wait(&empty[b], (k - 1) & 1)) {
          failed = true;
          break;
        }
        const int64_t tile = c % a.ntiles;
        const int q = (int)(c / a.ntiles) * UQC;
        const int64_t n0 = tile * UTV;
        unsigned char* st = smem + b * L.stage;
        mbar_arrive_expect_tx(&full[b], stage_bytes);
        tma_load_2d(st + L.zc, &maps.zc, (int)(n0 - 4), q, &full[b]);
        for (int j = 0; j < NR; ++j)
          tma_load_2d(st + L.zn + j * UQC * UNW * 4, &maps.zn, (int)ufloor4(n0 + off[j]), q,
                      &full[b]);
        tma_load_2d(st + L.dd, &maps.d, (int)n0, q, &full[b]);
        tma_load_2d(st + L.hh, &maps.h, (int)n0, q, &full[b]);
        tma_load_2d(st + L.aa, &maps.acc, (int)n0, q, &full[b]);
      }
    }
  } else {
    const int v = (warp & 3) * 32 + lane;   // voxel of this lane within the tile
    const int qh = (warp >> 2) * UQH;         // first compartment of this warp's group
    for (int64_t c = blockIdx.x; c < a.T; c += G) {
      const int i = (int)((c - blockIdx.x) / G), b = i % UNB, k = i / UNB;
      if (!failed && !mbar_wait(&full[b], k & 1)) failed = true;
      const int64_t tile = c % a.ntiles;
      const int q0 = (int)(c / a.ntiles) * UQC + qh;
      const int64_t n0 = tile * UTV, n = n0 + v;
      const bool valid = n < N && !failed;
      int x = 0, y = 0, zc = 0;
      if (valid) {
        x = (int)(n % nx);
        const int64_t t = n / nx;
        y = (int)(t % ny);
        zc = (int)(t / ny);
      }
      // a voxel outside the object is left alone and is nobody's neighbour
      const uint8_t* mk = MASKED ? a.mask : nullptr;   // unmasked: the checks fold away
      const bool in = valid && (!mk || mk[n]);
      const bool hxm = in && x > 0 && (!mk || mk[n - 1]);
      const bool hxp = in && x < nx - 1 && (!mk || mk[n + 1]);
      const bool hym = in && y > 0 && (!mk || mk[n - nx]);
      const bool hyp = in && y < ny - 1 && (!mk || mk[n + nx]);
      const bool hzm = zl && in && zc > 0 && (!mk || mk[n - plane]);
      const bool hzp = zl && in && zc < nz - 1 && (!mk || mk[n + plane]);
      const float deg = (float)(hxm + hxp + hym + hyp + hzm + hzp);
      const bool flags[4] = {ny > 1 ? hym : hzm, ny > 1 ? hyp : hzp, hzm, hzp};
      int nidx[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) nidx[j] = j < NR ? (int)(n + off[j] - ufloor4(n0 + off[j])) : 0;
      const unsigned char* st = smem + b * L.stage;
      const float* zr = reinterpret_cast<const float*>(st + L.zc);
      const float* znr = reinterpret_cast<const float*>(st + L.zn);
      const float* dr = reinterpret_cast<const float*>(st + L.dd);
      const float* hr = reinterpret_cast<const float*>(st + L.hh);
      const float* ar = reinterpret_cast<const float*>(st + L.aa);
      const DenseStep step{a.xi, a.lam_s, a.beta, a.inv_xb};
      float wv[UQH];
#pragma unroll
      for (int rr = 0; rr < UQH; ++rr) {
        wv[rr] = 0.f;
        const int r = qh + rr, q = q0 + rr;
        if (in && q < a.Q) {
          const float z = zr[r * UZW + 4 + v], d = dr[r * UTV + v];
          float nb = 0.f;
          if (hxm) nb += zr[r * UZW + 3 + v];
          if (hxp) nb += zr[r * UZW + 5 + v];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < NR && flags[j]) nb += znr[(j * UQC + r) * UNW + nidx[j]];
          const float f = __fadd_rn(hr[r * UTV + v], ar[r * UTV + v]);
          float dn;
          const float zn = step.apply(z, d, f, deg, nb, dn, wv[rr]);
          const int64_t o = (int64_t)q * ld + n;
          a.Zout[o] = zn;
          a.Dout[o] = dn;
          if (CHECK) {
            const float e = zn - f, ch = zn - z;
            s1 = fmaf(e, e, s1);
            s2 = fmaf(ch, ch, s2);
            s3 = fmaf(zn, zn, s3);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
      if (in) {
        // UQH values = a part (a half or a quarter) of the voxel's 32-byte sector in hi
        // and in lo
        uint32_t hh[UQH / 2], ll[UQH / 2];
#pragma unroll
        for (int e = 0; e < UQH / 2; ++e) {
          const float w0 = wv[2 * e], w1 = wv[2 * e + 1];
          hh[e] = pack_bf16(w0, w1);
          ll[e] = pack_bf16(w0 - __bfloat162float(__float2bfloat16_rn(w0)),
                            w1 - __bfloat162float(__float2bfloat16_rn(w1)));
        }
        if constexpr (UQH == 8) {
          *reinterpret_cast<uint4*>(a.Whi + n * a.Qp + q0) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
          *reinterpret_cast<uint4*>(a.Wlo + n * a.Qp + q0) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
        } else {
          *reinterpret_cast<uint2*>(a.Whi + n * a.Qp + q0) = make_uint2(hh[0], hh[1]);
          *reinterpret_cast<uint2*>(a.Wlo + n * a.Qp + q0) = make_uint2(ll[0], ll[1]);
        }
      }
    }
  }
  if (failed) atomicExch(a.err, (int)SSM_ETIMEOUT);
  if (CHECK) {
    double d1 = s1, d2 = s2, d3 = s3;
    for (int o = 16; o > 0; o >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      d3 += __shfl_xor_sync(0xffffffffu, d3, o);
    }
    __shared__ double red[UNT / 32][3];
    if (lane == 0) {
      red[warp][0] = d1;
      red[warp][1] = d2;
      red[warp][2] = d3;
    }
    __syncthreads();
    if (tid < 3) {
      double t = 0.0;
      for (int w = 0; w < UNT / 32; ++w) t += red[w][tid];
      a.partial[(int64_t)blockIdx.x * 4 + tid] = t;
    }
  }
}

int update_nr(const ssm_plan_s* pl) {
  return (pl->g.ny > 1 ? 2 : 0) + (pl->g.nz > 1 && pl->g.zlink ? 2 : 0);
}

// consumer warps of the kernel for this grid
int update_ncw(const ssm_plan_s* pl) { return update_nr(pl) == 4 ? 16 : 8; }

template <int NCW>
int update_per_sm(int nr) {
  const size_t shm = (size_t)ULayout(nr).total + 128;
  const size_t shm_max = (size_t)ULayout(4).total + 128;
  for (const void* k : {(const void*)tc_update_kernel<true, NCW, false>,
                        (const void*)tc_update_kernel<false, NCW, false>,
                        (const void*)tc_update_kernel<true, NCW, true>,
                        (const void*)tc_update_kernel<false, NCW, true>})
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_max);
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tc_update_kernel<true, NCW, false>,
                                                UWarps<NCW>::NT, shm);
  return std::max(1, b);
}

int update_grid_impl(const ssm_plan_s* pl) {
  // resident CTAs per SM, per number of halo rows (the shared-memory layout differs)
  static std::atomic<int> cached[5];
  const int nr = update_nr(pl);
  int per_sm = cached[nr].load(std::memory_order_acquire);
  if (per_sm == 0) {
    std::lock_guard<std::mutex> lock(attr_mutex());
    per_sm = cached[nr].load(std::memory_order_relaxed);
    if (per_sm == 0) {
      per_sm = update_ncw(pl) == 16 ? update_per_sm<16>(nr) : update_per_sm<8>(nr);
      cached[nr].store(per_sm, std::memory_order_release);
    }
  }
  const int64_t ntiles = (pl->g.N + UTV - 1) / UTV;
  const int64_t T = ntiles * ((pl->Q + UQC - 1) / UQC);
  return (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sm_count() * per_sm * std::max(1, pl->waves), T));
}

}  // namespace

ssm_status tc_update_prepare(ssm_plan_s* pl) {
  update_grid_impl(pl);
  return SSM_OK;
}

int tc_update_grid(const ssm_plan_s* pl) { return update_grid_impl(pl); }

ssm_status tc_update(ssm_plan_s* pl, int cur, bool check, double* partial, int* nparts,
                     cudaStream_t s) {
  const uint64_t Q = (uint64_t)pl->Q, N = (uint64_t)pl->g.N, ld = (uint64_t)pl->g.ld;
  UpdMaps m;
  const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  SSM_CUDA(encode_2d(&m.zc, f32, 4, pl->Z[cur], N, Q, ld, UZW, UQC));
  SSM_CUDA(encode_2d(&m.zn, f32, 4, pl->Z[cur], N, Q, ld, UNW, UQC));
  SSM_CUDA(encode_2d(&m.d, f32, 4, pl->Dl[cur], N, Q, ld, UTV, UQC));
  SSM_CUDA(encode_2d(&m.h, f32, 4, pl->H, N, Q, ld, UTV, UQC));
  SSM_CUDA(encode_2d(&m.acc, f32, 4, pl->Acc, N, Q, ld, UTV, UQC));
  UpdArgs a;
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.Whi = pl->Whi[cur ^ 1];
  a.Wlo = pl->Wlo[cur ^ 1];
  a.partial = partial;
  a.mask = pl->mask;
  a.err = pl->dev_err;
  a.g = pl->g;
  a.Q = pl->Q;
  a.Qp = pl->Qp;
  a.nqc = (pl->Q + UQC - 1) / UQC;
  a.ntiles = (pl->g.N + UTV - 1) / UTV;
  a.T = a.ntiles * (int64_t)a.nqc;
  a.beta = (float)pl->p.beta;
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  const int grid = update_grid_impl(pl);
  *nparts = grid;
  const size_t shm = (size_t)ULayout(update_nr(pl)).total + 128;
  const bool masked = pl->mask != nullptr;
#define SSM_UPD(C, W, MK) tc_update_kernel<C, W, MK><<<grid, UWarps<W>::NT, shm, s>>>(m, a)
  if (update_ncw(pl) == 16) {
    if (masked) {
      if (check) SSM_UPD(true, 16, true); else SSM_UPD(false, 16, true);
    } else {
      if (check) SSM_UPD(true, 16, false); else SSM_UPD(false, 16, false);
    }
  } else {
    if (masked) {
      if (check) SSM_UPD(true, 8, true); else SSM_UPD(false, 8, true);
    } else {
      if (check) SSM_UPD(true, 8, false); else SSM_UPD(false, 8, false);
    }
  }
#undef SSM_UPD
  SSM_LAUNCHED();
  return SSM_OK;
}

}  // namespace ssm
