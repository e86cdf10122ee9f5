// Full-rank (Eq. 26) LADMM iteration on the tcgen05 tensor cores, BF16 split products.
//
// The f-step of Eq. 26 is f = h + M w with M = (K^T K + beta I)^{-1} (Q x Q, formed
// once in FP64), h = M g (once per solve) and w = beta z - d. An iteration is two
// kernels:
//   tc_gemm_kernel    acc = M w on the tensor cores (tcgen05.mma, TMA-fed, FP32 in TMEM)
//   tc_update_kernel  the bandwidth-bound rest, TMA-staged (ssm_tc_update.cu):
//       f  = h + acc
//       z' = max(0, (xi z - lambda s (deg z - sum_nbr z) + beta f + d) / (xi + beta))  (Eq. 31)
//       d' = d - beta (z' - f)                                                      (step 11)
//       w' = beta z' - d'   -> stored as the BF16 pair (hi, lo) for the next product
//
// Precision ("BF16x3"): w and M are each split into BF16 hi + lo parts
// (x_hi = bf16(x), x_lo = bf16(x - x_hi)), and M w is accumulated in FP32 in tensor
// memory as M_hi w_hi + M_hi w_lo + M_lo w_hi (the lo*lo term, ~2^-16 relative, is
// dropped). z, d, h and f stay FP32.
//
// GEMM operands: w is kept voxel-major (row n holds its Q compartments, stride Qp), so
// both MMA operands are K-major: A = w tile (128 voxels x 64 compartments), B = M tile
// (BN output compartments x 64), each a 128-byte-swizzled TMA box. The accumulator
// (128 voxels x BN compartments, FP32) lives in TMEM, with TMEM lanes = voxels, so
// the epilogue's stores of acc into the map-major Q x N array coalesce. The tile width
// BN (128 .. 256) is chosen per problem shape by a small autotuner at plan time.
//
// GEMM schedule: one persistent CTA per SM walks (voxel tile, compartment tile) pairs,
// voxel-tile major so concurrently running CTAs share w tiles in L2. Warp 0 issues TMA
// loads into a smem ring; one thread of warp 1 issues the tcgen05.mma chain (3 MMAs
// per K = 16 step) and commits stage releases and accumulator completions to
// mbarriers; warps 2-5 drain the accumulator (tcgen05.ld) to global memory. Two
// accumulators (TMEM columns 0 and 256) alternate so draining one tile overlaps the
// next tile's MMAs. Every mbarrier wait is bounded.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <tuple>

#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

namespace ssm {
namespace {

constexpr int BM = 128;                         // voxels per tile (MMA M, TMEM lanes)
constexpr int BK = 64;                          // K per stage: one 128-byte swizzle atom
constexpr int UK = 16;                          // K per tcgen05.mma (kind::f16)
constexpr int NTHR = 192;                       // TMA warp, MMA warp, 4 epilogue warps
constexpr uint32_t TMEM_COLS = 512;             // two accumulators, at columns 0 and 256
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int kSmemLimit = 227 * 1024;

// Compartment-tile widths (MMA N) the autotuner chooses from: multiples of 32 (the
// drain reads 32 TMEM columns at a time) up to 256 (one accumulator). Narrower tiles
// waste fewer padded columns when Q is not a multiple of 256, and leave room for a
// deeper smem ring.
constexpr int kTileN[] = {256, 224, 192, 160, 128};

template <int BN>
struct Tile {
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int NS = (kSmemLimit - 2048) / STAGE_BYTES > 4 ? 4
                                                                  : (kSmemLimit - 2048) / STAGE_BYTES;
  static constexpr int SMEM_BYTES = NS * STAGE_BYTES + 1024 + 256;
  // kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9,
  // 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(BN % 32 == 0 && BN <= 256 && NS >= 2, "tile shape");
};

struct TcMaps {
  CUtensorMap a_hi, a_lo;   // w (voxel-major), box {BK, BM}
  CUtensorMap b_hi, b_lo;   // M, box {BK, BN}
};

struct TcArgs {
  float* __restrict__ Acc;           // M w, map-major Q x N (row stride ld)
  int* __restrict__ err;
  Grid g;
  int Q, ntv, ntq;
};

// shared-memory matrix descriptor, K-major operand in the 128-byte swizzle layout:
// start address >> 4 (bits 0-13), leading byte offset 16 B (unused for this layout),
// stride byte offset 1024 B = 8 rows x 128 B (bits 32-45), version 1 (bit 46),
// base offset 0, swizzle mode 2 = 128 B (bits 61-63)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
__global__ void __launch_bounds__(NTHR, 1) tc_gemm_kernel(const __grid_constant__ TcMaps maps,
                                                          const TcArgs a) {
  constexpr int NS = Tile<BN>::NS, STAGE_BYTES = Tile<BN>::STAGE_BYTES;
  constexpr int B_BYTES = Tile<BN>::B_BYTES;
  constexpr uint32_t IDESC = Tile<BN>::IDESC;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * STAGE_BYTES);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int ntiles = a.ntv * a.ntq;
  const int nk = (a.Q + BK - 1) / BK;
  bool failed = false;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_map(&maps.a_hi);
      tma_prefetch_map(&maps.b_hi);
      int c = 0;
      for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
        const int vt = t / a.ntq, qt = t % a.ntq;
        for (int kc = 0; kc < nk; ++kc, ++c) {
          const int s = c % NS, r = c / NS;
          if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1)) {
            failed = true;
            break;
          }
          unsigned char* st = smem + s * STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
          tma_load_2d(st, &maps.a_hi, kc * BK, vt * BM, &full[s]);
          tma_load_2d(st + A_BYTES, &maps.a_lo, kc * BK, vt * BM, &full[s]);
          tma_load_2d(st + 2 * A_BYTES, &maps.b_hi, kc * BK, qt * BN, &full[s]);
          tma_load_2d(st + 2 * A_BYTES + B_BYTES, &maps.b_lo, kc * BK, qt * BN, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int c = 0, it = 0;
      for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x, ++it) {
        const int acc = it & 1, ra = it >> 1;
        if (ra > 0 && !mbar_wait(&tempty[acc], (ra - 1) & 1)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * 256);
        for (int kc = 0; kc < nk; ++kc, ++c) {
          const int s = c % NS, r = c / NS;
          if (!mbar_wait(&full[s], r & 1)) {
            failed = true;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / UK; ++kk) {
            const uint64_t ahi = smem_desc(base + kk * 32);
            const uint64_t alo = smem_desc(base + A_BYTES + kk * 32);
            const uint64_t bhi = smem_desc(base + 2 * A_BYTES + kk * 32);
            const uint64_t blo = smem_desc(base + 2 * A_BYTES + B_BYTES + kk * 32);
            mma_bf16(d_tmem, ahi, bhi, IDESC, (kc | kk) ? 1u : 0u);
            mma_bf16(d_tmem, alo, bhi, IDESC, 1u);
            mma_bf16(d_tmem, ahi, blo, IDESC, 1u);
          }
          mma_commit(&empty[s]);      // the stage is free once these MMAs complete
        }
        mma_commit(&tfull[acc]);      // the accumulator is complete
      }
    }
  } else {
    // ------------------------------------------------------------ accumulator drain
    const int quarter = warp & 3;                  // TMEM lanes 32*quarter .. +31
    const int row = quarter * 32 + lane;           // voxel within the tile
    const int64_t ld = a.g.ld, N = a.g.N;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int acc = it & 1, ra = it >> 1;
      if (!failed && !mbar_wait(&tfull[acc], ra & 1)) failed = true;
      tc_fence_after();
      const int vt = t / a.ntq, qt = t % a.ntq;
      const int64_t n = (int64_t)vt * BM + row;
      const bool valid = n < N && !failed;
      for (int cc = 0; cc < BN / 32; ++cc) {
        const int q0 = qt * BN + cc * 32;
        if (q0 >= a.Q) break;                       // uniform across the warp
        float v[32];
        tmem_ld32(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 256 + cc * 32),
                  v);
        if (valid) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (q0 + j < a.Q) a.Acc[(int64_t)(q0 + j) * ld + n] = v[j];
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }
  if (failed) atomicExch(a.err, (int)SSM_ETIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

int gemm_grid(const ssm_plan_s* pl, int bn) {
  const int ntv = (int)((pl->g.N + BM - 1) / BM);
  const int ntq = (pl->Q + bn - 1) / bn;
  return std::max(1, std::min(sm_count() * std::max(1, pl->waves), ntv * ntq));
}

template <int BN>
ssm_status launch_gemm(const ssm_plan_s* pl, int cur, cudaStream_t s) {
  const uint64_t Q = (uint64_t)pl->Q, N = (uint64_t)pl->g.N, Qp = (uint64_t)pl->Qp;
  TcMaps m;
  const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
  SSM_CUDA(encode_2d(&m.a_hi, bf, 2, pl->Whi[cur], Q, N, Qp, BK, BM, sw));
  SSM_CUDA(encode_2d(&m.a_lo, bf, 2, pl->Wlo[cur], Q, N, Qp, BK, BM, sw));
  SSM_CUDA(encode_2d(&m.b_hi, bf, 2, pl->Mhi, Q, Q, Qp, BK, BN, sw));
  SSM_CUDA(encode_2d(&m.b_lo, bf, 2, pl->Mlo, Q, Q, Qp, BK, BN, sw));
  TcArgs a;
  a.Acc = pl->Acc;
  a.err = pl->dev_err;
  a.g = pl->g;
  a.Q = pl->Q;
  a.ntv = (int)((pl->g.N + BM - 1) / BM);
  a.ntq = (pl->Q + BN - 1) / BN;
  tc_gemm_kernel<BN><<<gemm_grid(pl, BN), NTHR, Tile<BN>::SMEM_BYTES, s>>>(m, a);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status gemm_dispatch(const ssm_plan_s* pl, int bn, int cur, cudaStream_t s) {
  switch (bn) {
    case 256: return launch_gemm<256>(pl, cur, s);
    case 224: return launch_gemm<224>(pl, cur, s);
    case 192: return launch_gemm<192>(pl, cur, s);
    case 160: return launch_gemm<160>(pl, cur, s);
    case 128: return launch_gemm<128>(pl, cur, s);
    default:
      set_error("tensor-core GEMM: unsupported tile width");
      return SSM_EUNSUPPORTED;
  }
}

template <int BN>
cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Tile<BN>::SMEM_BYTES);
}

// tile widths measured per (device, Q, N, waves), shared by every plan of the process
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int64_t, int>, int> g_tuned;

// Autotuner: time every tile width on the plan's own operands (one warm-up launch, then
// two timed launches each, CUDA events on the plan's stream) and keep the fastest.
// The choice does not change results: each output element sums the same products in
// the same K order whatever the tile width.
ssm_status tune_tile(ssm_plan_s* pl, cudaStream_t s) {
  if (const char* env = getenv("SSM_TC_BN")) {   // a fixed width (tests and sweeps)
    const int v = atoi(env);
    for (int bn : kTileN)
      if (bn == v) {
        pl->tc_bn = v;
        return SSM_OK;
      }
  }
  const auto key = std::make_tuple(pl->device, pl->Q, pl->g.N, pl->waves);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      pl->tc_bn = it->second;
      return SSM_OK;
    }
  }
  cudaEvent_t e0, e1;
  SSM_CUDA(cudaEventCreate(&e0));
  SSM_CUDA(cudaEventCreate(&e1));
  int best = 256;
  float best_ms = 0.f;
  ssm_status st = SSM_OK;
  for (int bn : kTileN) {
    // a width whose tiles do not cover fewer padded columns than a wider one cannot win
    const int pad = (pl->Q + bn - 1) / bn * bn;
    if (bn != 256 && pad >= (pl->Q + 255) / 256 * 256) continue;
    st = gemm_dispatch(pl, bn, 0, s);
    if (st != SSM_OK) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) { st = SSM_ECUDA; break; }
    for (int r = 0; r < 2 && st == SSM_OK; ++r) st = gemm_dispatch(pl, bn, 0, s);
    if (st != SSM_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = SSM_ECUDA;
      break;
    }
    if (bn == 256 || ms < best_ms) {
      best = bn;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SSM_OK) return st;
  pl->tc_bn = best;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned[key] = best;
  return SSM_OK;
}

}  // namespace

ssm_status tc_prepare(ssm_plan_s* pl, cudaStream_t s) {
  if (pl->Qp % BK != 0) {
    set_error("tensor-core form: padded Q must be a multiple of 64");
    return SSM_EUNSUPPORTED;
  }
  SSM_CUDA(set_smem_attr<256>());
  SSM_CUDA(set_smem_attr<224>());
  SSM_CUDA(set_smem_attr<192>());
  SSM_CUDA(set_smem_attr<160>());
  SSM_CUDA(set_smem_attr<128>());
  SSM_TRY(tc_update_prepare(pl));
  return tune_tile(pl, s);
}

// reduction rows: bounded with the narrowest tile (the most tiles, the largest grid)
int tc_max_partials(const ssm_plan_s* pl) {
  return std::max(gemm_grid(pl, 128), tc_update_grid(pl));
}

void tc_release(ssm_plan_s*) {}

ssm_status tc_gemm(ssm_plan_s* pl, int cur, cudaStream_t s) {
  return gemm_dispatch(pl, pl->tc_bn, cur, s);
}

int tc_gemm_grid(const ssm_plan_s* pl) { return gemm_grid(pl, pl->tc_bn); }

ssm_status tc_iteration(ssm_plan_s* pl, int cur, bool check, double* partial, int* nparts,
                        cudaStream_t s) {
  SSM_TRY(tc_gemm(pl, cur, s));
  return tc_update(pl, cur, check, partial, nparts, s);
}

}  // namespace ssm
