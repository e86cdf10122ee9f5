// Full-rank (Eq. 26) LADMM iteration on the tcgen05 tensor cores, BF16 split products.
//
// The f-step of Eq. 26 is f = h + M w with M = (K^T K + beta I)^{-1} (Q x Q, formed
// once in FP64), h = M g (once per solve) and w = beta z - d. The iteration is
//   acc = M w on the tensor cores (tcgen05.mma, TMA-fed, FP32 in TMEM), then per element
//       f  = h + acc
//       z' = max(0, (xi z - lambda s (deg z - sum_nbr z) + beta f + d) / (xi + beta))  (Eq. 31)
//       d' = d - beta (z' - f)                                                      (step 11)
//       w' = beta z' - d'   -> stored as the BF16 pair (hi, lo) for the next product
// Three forms of the iteration, chosen per problem shape by a plan-time autotuner:
//   - GEMM + update: the GEMM's epilogue stores acc to memory, and the TMA-staged update
//     kernel of ssm_tc_update.cu applies the element-wise steps;
//   - fused, staged epilogue: the epilogue warps apply the steps to each accumulator tile
//     straight out of TMEM, reading z, its neighbour rows, d and h from a shared-memory
//     ring that a producer warp fills by TMA (every width on 1D/2D grids, up to 224 on
//     3D grids; at the widest of these, d and h are prefetched into registers instead);
//   - fused, register epilogue: the same, with the reads software-pipelined in
//     registers (any width).
// In the fused forms M w never goes to memory, and the element-wise work runs while the
// MMA warp computes the next tile. All three apply the same steps (DenseStep) to the same
// accumulator values and give the same bits.
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
// mbarriers; warps 2-9 drain the accumulator (tcgen05.ld), two per TMEM lane quarter;
// warp 10 feeds the staged epilogue's ring. Two accumulators (TMEM columns 0 and 256)
// alternate so draining one tile overlaps the next tile's MMAs. Every mbarrier wait is
// bounded.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>

#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

#ifndef SSM_TC_NEPI
#define SSM_TC_NEPI 8
#endif

namespace ssm {
namespace {

constexpr int BM = 128;                         // voxels per tile (MMA M, TMEM lanes)
constexpr int BK = 64;                          // K per stage: one 128-byte swizzle atom
constexpr int UK = 16;                          // K per tcgen05.mma (kind::f16)
constexpr int NEPI = SSM_TC_NEPI;                // epilogue warps (2 per TMEM lane quarter)
constexpr int EPW = 2 + NEPI;                   // the fused epilogue's TMA producer warp
constexpr int NTHR = 96 + 32 * NEPI;            // TMA, MMA, epilogue warps, epilogue TMA
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
  // kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9,
  // 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(BN % 32 == 0 && BN <= 256 && NS >= 2, "tile shape");
};

struct TcMaps {
  CUtensorMap a_hi, a_lo;   // w (voxel-major), box {BK, BM}
  CUtensorMap b_hi, b_lo;   // M, box {BK, BN}
  // fused epilogue (map-major Q x N arrays): z with its x halo {EZW, UG}, z neighbour
  // rows {ENW, UG}, d and h {BM, UG}
  CUtensorMap ez_c, ez_n, ed, eh;
};

struct TcArgs {
  float* __restrict__ Acc;           // M w, map-major Q x N (row stride ld): store epilogue
  int* __restrict__ err;
  Grid g;
  int Q, ntv, ntq;
  // fused update epilogue
  const float* __restrict__ Zin;     // z^k, d^k, h (Q x ld)
  const float* __restrict__ Din;
  const float* __restrict__ H;
  float* __restrict__ Zout;          // z^{k+1}, d^{k+1}
  float* __restrict__ Dout;
  __nv_bfloat16* __restrict__ Whi;   // w^{k+1} split, voxel-major (row stride Qp)
  __nv_bfloat16* __restrict__ Wlo;
  double* __restrict__ partial;      // 4 doubles per CTA (residual iterations)
  const uint8_t* __restrict__ mask;  // voxels inside the object (nullptr: every voxel)
  int Qp;
  float beta, xi, lam_s, inv_xb;
};

// compartments per group of the fused epilogue: one tcgen05.ld of 8 columns and one
// 16-byte store of w each
constexpr int UG = 8;
// epilogue modes of tc_gemm_kernel
constexpr int EPI_STORE = 0;         // acc -> Acc
constexpr int EPI_UPDATE = 1;        // the element-wise steps of the iteration, reads staged
                                     // in shared memory by TMA
constexpr int EPI_UPDATE_CHECK = 2;  // ... plus the residual sums of the stopping rule
constexpr int EPI_REG = 3;           // the element-wise steps, reads software-pipelined in
                                     // registers (no shared memory: any tile width)
constexpr int EPI_REG_CHECK = 4;     // ... plus the residual sums
constexpr bool epi_check(int e) { return e == EPI_UPDATE_CHECK || e == EPI_REG_CHECK; }
constexpr bool epi_staged(int e) { return e == EPI_UPDATE || e == EPI_UPDATE_CHECK; }

// register epilogue: groups whose reads are in flight at once per thread -- two
// (software-pipelined) with up to two neighbour rows per element, one with four (3D)
template <int NRT>
constexpr int pipe_depth() { return NRT == 4 ? 1 : 2; }
constexpr int EZW = BM + 8;   // staged z row: voxels n0-4 .. n0+BM+3 (the x halo)
constexpr int ENW = BM + 4;   // staged neighbour row: 4-aligned base .. +BM+3

// One stage of the fused epilogue's ring: a group of UG compartments of a voxel tile --
// z with its x halo, NRT neighbour rows (the -+nx, -+nx*ny rows), d and h -- each a TMA
// box (128-byte-aligned offsets).
// DH = false leaves d and h out of the stage (the epilogue warps then prefetch them into
// registers one group ahead), for the configurations whose ring would not fit otherwise.
template <int NRT, bool DH = true>
struct EpiStage {
  static constexpr int zc = 0;
  static constexpr int zn = UG * EZW * 4;
  static constexpr int dd = zn + NRT * UG * ENW * 4;
  static constexpr int hh = dd + UG * BM * 4;
  static constexpr int bytes = DH ? hh + UG * BM * 4 : dd;
  static_assert(zn % 128 == 0 && dd % 128 == 0 && hh % 128 == 0 && bytes % 128 == 0, "layout");
};

// Shared memory of one kernel configuration. The store epilogue gives the GEMM's operand
// ring all of it; the fused epilogue keeps the ring at 2 stages and fills the rest with
// 2 or 4 epilogue stages. A fused configuration needs 2 of them: BN <= 224 on grids with
// 2 neighbour rows, BN <= 192 on 3D grids.
template <int BN, int EPI, int NRT>
struct Cfg {
  static constexpr bool fused = epi_staged(EPI);   // an epilogue ring in shared memory
  static constexpr int NS = fused ? 2 : Tile<BN>::NS;
  static constexpr int RESERVE = 1024 + 256;    // alignment slack, barriers, TMEM slot
  // static shared memory of the residual-test variants: the reduction array, which the
  // compiler pads to 1024 bytes to keep the 1024-aligned dynamic window aligned; the
  // per-block limit counts it with the dynamic bytes
  static constexpr int STATIC_MAX = 1024;
  static constexpr int room = kSmemLimit - RESERVE - STATIC_MAX - NS * Tile<BN>::STAGE_BYTES;
  // an even number of stages: slot = sequence index mod NBE then has the parity of the
  // sequence index, so every slot is consumed by one half of the epilogue warps and its
  // barrier phases complete in that half's order (with an odd count the halves would
  // alternate on a slot, and a half waiting by parity could pass on an older phase)
  static constexpr int even_stages(int est) { return (room / est > 4 ? 4 : room / est) & ~1; }
  // d and h are staged unless that leaves fewer than two stages
  static constexpr bool DH = even_stages(EpiStage<NRT, true>::bytes) >= 2;
  static constexpr int EST = EpiStage<NRT, DH>::bytes;
  static constexpr int NBE = fused ? even_stages(EST) : 0;
  static constexpr bool valid = !fused || NBE >= 2;
  static constexpr int SMEM_BYTES = NS * Tile<BN>::STAGE_BYTES + NBE * EST + RESERVE;
};


// round down to a multiple of 4 (toward -infinity): a 16-byte-aligned TMA x coordinate
__host__ __device__ __forceinline__ int64_t floor4i(int64_t v) {
  return v >= 0 ? (v & ~(int64_t)3) : -(((-v) + 3) & ~(int64_t)3);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

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

// 8 (or 4) consecutive FP32 columns of this warp's 32 TMEM lanes
template <int C>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float* v) {
  static_assert(C == 4 || C == 8, "columns");
  uint32_t r[8];
  if constexpr (C == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
  } else {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < C; ++i) v[i] = __uint_as_float(r[i]);
}

// NRT: staged neighbour rows the fused epilogue reads per element (2: 1D/2D grids and
// stacked slices, 4: 3D grids); the store epilogue ignores it
template <int BN, int EPI, int NRT>
__global__ void __launch_bounds__(NTHR, 1) tc_gemm_kernel(const __grid_constant__ TcMaps maps,
                                                          const TcArgs a) {
  using C = Cfg<BN, EPI, NRT>;
  using ES = EpiStage<NRT, C::DH>;
  constexpr int NS = C::NS, NBE = C::NBE, STAGE_BYTES = Tile<BN>::STAGE_BYTES;
  constexpr int B_BYTES = Tile<BN>::B_BYTES;
  constexpr uint32_t IDESC = Tile<BN>::IDESC;
  static_assert(C::valid, "fused epilogue needs two ring stages");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // aligned by an offset from the shared array itself (not through an integer), so that
  // the compiler keeps the shared address space of every pointer derived from it
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* estage = smem + NS * STAGE_BYTES;      // the epilogue ring (fused)
  uint64_t* full = reinterpret_cast<uint64_t*>(estage + NBE * C::EST);
  uint64_t* empty = full + NS;
  uint64_t* tfull = empty + NS;
  uint64_t* tempty = tfull + 2;
  uint64_t* efull = tempty + 2;     // epilogue stage loaded
  uint64_t* eempty = efull + 4;     // epilogue stage consumed (4 warps: one half)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(eempty + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], NEPI);
    }
    for (int i = 0; i < NBE; ++i) {
      mbar_init(&efull[i], 1);
      mbar_init(&eempty[i], NEPI / 2);
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
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;   // residual sums of the fused update

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
  } else if (warp == EPW) {
    // ------------------------------------------------------------ epilogue TMA producer
    // streams each (tile, group) of the CTA's sequence into the epilogue ring, running
    // up to NBE groups ahead of the epilogue warps (these reads do not depend on the MMAs)
    if constexpr (C::fused) {
      if (lane == 0) {
        const int nx = a.g.nx, ny = a.g.ny;
        const bool zl = a.g.nz > 1 && a.g.zlink;
        const int NR = (ny > 1 ? 2 : 0) + (zl ? 2 : 0);
        const int64_t plane = (int64_t)nx * ny;
        const int64_t off[4] = {ny > 1 ? -(int64_t)nx : -plane, ny > 1 ? (int64_t)nx : plane,
                                -plane, plane};
        const unsigned bytes =
            (unsigned)((UG * EZW + NR * UG * ENW + (C::DH ? 2 * UG * BM : 0)) * 4);
        tma_prefetch_map(&maps.ez_c);
        tma_prefetch_map(&maps.ez_n);
        int i = 0;
        for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
          const int vt = t / a.ntq, qt = t % a.ntq;
          const int64_t n0 = (int64_t)vt * BM;
          for (int cg = 0; cg < BN / UG; ++cg, ++i) {
            const int q0 = qt * BN + cg * UG;
            if (q0 >= a.Q) break;
            const int slot = i % NBE, k = i / NBE;
            if (k > 0 && !mbar_wait(&eempty[slot], (k - 1) & 1)) {
              failed = true;
              break;
            }
            unsigned char* st = estage + slot * C::EST;
            mbar_arrive_expect_tx(&efull[slot], bytes);
            tma_load_2d(st + ES::zc, &maps.ez_c, (int)(n0 - 4), q0, &efull[slot]);
            for (int j = 0; j < NR; ++j)
              tma_load_2d(st + ES::zn + j * UG * ENW * 4, &maps.ez_n,
                          (int)floor4i(n0 + off[j]), q0, &efull[slot]);
            if constexpr (C::DH) {
              tma_load_2d(st + ES::dd, &maps.ed, (int)n0, q0, &efull[slot]);
              tma_load_2d(st + ES::hh, &maps.eh, (int)n0, q0, &efull[slot]);
            }
          }
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
    const int half = NEPI == 8 ? (warp - 2) >> 2 : 0;   // which column groups this warp takes
    const int64_t ld = a.g.ld, N = a.g.N;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const bool zl = nz > 1 && a.g.zlink;           // z neighbours coupled
    const int NR = (ny > 1 ? 2 : 0) + (zl ? 2 : 0);
    const int64_t plane = (int64_t)nx * ny;
    // neighbour offsets beyond x: -nx, +nx, -nx*ny, +nx*ny (the axes the grid has; the y
    // pair first when there is a y axis)
    const int64_t off[4] = {ny > 1 ? -(int64_t)nx : -plane, ny > 1 ? (int64_t)nx : plane,
                            -plane, plane};
    // staged epilogue whose stages leave d and h out: those of this warp's next group are
    // prefetched into registers one group ahead; (pt, pcg) walks the CTA's (tile, group)
    // sequence in the order the epilogue producer stages it, two positions per group of
    // this half
    float dnext[UG], hnext[UG];
    int pt = blockIdx.x, pcg = 0;
    auto ngroups = [&](int tt) {
      const int rest = a.Q - (tt % a.ntq) * BN;
      return min(BN / UG, (rest + UG - 1) / UG);
    };
    auto step_seq = [&]() {
      if (++pcg >= ngroups(pt)) {
        pcg = 0;
        pt += gridDim.x;
      }
    };
    auto load_dh = [&]() {
      if (pt < ntiles) {
        const int64_t nn = (int64_t)(pt / a.ntq) * BM + row;   // < ld: a valid address
        const int q0n = (pt % a.ntq) * BN + pcg * UG;
#pragma unroll
        for (int j = 0; j < UG; ++j) {
          const int64_t o = (int64_t)min(q0n + j, a.Q - 1) * ld + nn;
          dnext[j] = __ldg(a.Din + o);
          hnext[j] = __ldg(a.H + o);
        }
      }
    };
    if constexpr (epi_staged(EPI) && !C::DH) {
      if (half == 1) step_seq();
      load_dh();
    }
    int it = 0;
    int gseq = 0;   // position in the CTA's sequence of (tile, group) (fused epilogue)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int acc = it & 1, ra = it >> 1;
      // every epilogue warp waits for each tile's accumulator (also one whose half has no
      // group in the tile), so no warp's release of an accumulator runs a phase ahead
      if (!failed && !mbar_wait(&tfull[acc], ra & 1)) failed = true;
      tc_fence_after();
      const int vt = t / a.ntq, qt = t % a.ntq;
      const int64_t n = (int64_t)vt * BM + row;
      const bool valid = n < N && !failed;
      if constexpr (EPI != EPI_STORE) {
        // the voxel's neighbours on the grid graph (the one the mask induces: a voxel
        // outside the object is left alone and is nobody's neighbour)
        int x = 0, y = 0, zc = 0;
        if (valid) {
          x = (int)(n % nx);
          const int64_t tt = n / nx;
          y = (int)(tt % ny);
          zc = (int)(tt / ny);
        }
        const uint8_t* mk = a.mask;
        const bool in = valid && (!mk || mk[n]);
        const bool hxm = in && x > 0 && (!mk || mk[n - 1]);
        const bool hxp = in && x < nx - 1 && (!mk || mk[n + 1]);
        const bool hym = in && y > 0 && (!mk || mk[n - nx]);
        const bool hyp = in && y < ny - 1 && (!mk || mk[n + nx]);
        const bool hzm = zl && in && zc > 0 && (!mk || mk[n - plane]);
        const bool hzp = zl && in && zc < nz - 1 && (!mk || mk[n + plane]);
        const float deg = (float)(hxm + hxp + hym + hyp + hzm + hzp);
        const bool flags[4] = {ny > 1 ? hym : hzm, ny > 1 ? hyp : hzp, hzm, hzp};
        if constexpr (epi_staged(EPI)) {
          bool nok[4];
          int rem[4];   // staged neighbour row k holds voxel v at index v + rem[k]
          const int64_t n0 = (int64_t)vt * BM;
  #pragma unroll
          for (int j = 0; j < 4; ++j) {
            nok[j] = j < NR && flags[j];
            rem[j] = (int)(n0 + off[j] - floor4i(n0 + off[j]));
          }
          const DenseStep step{a.xi, a.lam_s, a.beta, a.inv_xb};
          // the tile's groups of UG compartments in the CTA's sequence (the order the
          // epilogue producer stages them): this warp's half takes every other one
          for (int cg = 0; cg < BN / UG; ++cg, ++gseq) {
            const int q0 = qt * BN + cg * UG;
            if (q0 >= a.Q) break;                     // uniform across the warp
            if ((gseq & 1) != half) continue;
            const int slot = gseq % NBE, k = gseq / NBE;
            if (!failed && !mbar_wait(&efull[slot], k & 1)) failed = true;
            float v[UG];
            tmem_ld_cols<UG>(
                tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 256 + cg * UG), v);
            const unsigned char* st = estage + slot * C::EST;
            const float* zc_ = reinterpret_cast<const float*>(st + ES::zc);
            const float* zn_ = reinterpret_cast<const float*>(st + ES::zn);
            const float* dd_ = reinterpret_cast<const float*>(st + ES::dd);
            const float* hh_ = reinterpret_cast<const float*>(st + ES::hh);
            float dcur[UG], hcur[UG];
            if constexpr (!C::DH) {
#pragma unroll
              for (int j = 0; j < UG; ++j) {
                dcur[j] = dnext[j];
                hcur[j] = hnext[j];
              }
              step_seq();
              step_seq();
              load_dh();
            }
            if (!failed) {
  #pragma unroll
              for (int j = 0; j < UG; ++j) {
                const float z = zc_[j * EZW + 4 + row];
                float nb = 0.f;
                nb += hxm ? zc_[j * EZW + 3 + row] : 0.f;
                nb += hxp ? zc_[j * EZW + 5 + row] : 0.f;
  #pragma unroll
                for (int kk = 0; kk < NRT; ++kk)
                  nb += nok[kk] ? zn_[(kk * UG + j) * ENW + row + rem[kk]] : 0.f;
                const int q = q0 + j;
                const float f = __fadd_rn(C::DH ? hh_[j * BM + row] : hcur[j], v[j]);
                float dn, w;
                const float zn =
                    step.apply(z, C::DH ? dd_[j * BM + row] : dcur[j], f, deg, nb, dn, w);
                if (in && q < a.Q) {
                  const int64_t o = (int64_t)q * ld + n;
                  a.Zout[o] = zn;
                  a.Dout[o] = dn;
                  if constexpr (epi_check(EPI)) {
                    const float e = zn - f, ch = zn - z;
                    s1 = fmaf(e, e, s1);
                    s2 = fmaf(ch, ch, s2);
                    s3 = fmaf(zn, zn, s3);
                  }
                }
                v[j] = q < a.Q ? w : 0.f;             // padding columns stay zero
              }
              if (in) {
                uint32_t hh[UG / 2], ll[UG / 2];
  #pragma unroll
                for (int e = 0; e < UG / 2; ++e) {
                  const float w0 = v[2 * e], w1 = v[2 * e + 1];
                  hh[e] = pack_bf16x2(w0, w1);
                  ll[e] = pack_bf16x2(w0 - __bfloat162float(__float2bfloat16_rn(w0)),
                                      w1 - __bfloat162float(__float2bfloat16_rn(w1)));
                }
                *reinterpret_cast<uint4*>(a.Whi + n * a.Qp + q0) =
                    make_uint4(hh[0], hh[1], hh[2], hh[3]);
                *reinterpret_cast<uint4*>(a.Wlo + n * a.Qp + q0) =
                    make_uint4(ll[0], ll[1], ll[2], ll[3]);
              }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&eempty[slot]);
          }
        } else {
          bool nok[4];
          int64_t dk[4];
  #pragma unroll
          for (int j = 0; j < 4; ++j) {
            nok[j] = j < NR && flags[j];
            dk[j] = nok[j] ? off[j] : 0;
          }
          // groups of UG compartments of voxel n: a group's loads (coalesced across the
          // warp's 32 voxels; the neighbours are L1/L2 hits) are issued before its stores
          const DenseStep step{a.xi, a.lam_s, a.beta, a.inv_xb};
          // The warp's groups cg = half, half + NEPI/4, ... are software-pipelined over two
          // register buffers (1D/2D grids): the loads of the next group are issued before
          // the current group is computed, so two groups' reads are in flight. x neighbours
          // come from the adjacent lanes (shuffles); the two values beyond the warp's 32
          // voxels of each compartment are one register per group (lanes 0 .. UG-1: voxel
          // n0w - 1, lanes UG .. 2 UG - 1: n0w + 32, for compartments q0 .. q0 + UG - 1);
          // on 3D grids a single buffer, and x neighbours loaded (L1 hits).
          constexpr int GS = NEPI / 4;
          const int64_t n0w = n - lane;
          // x neighbours: shuffles where the two-buffer pipeline needs the registers (1D/2D),
          // L1-hit loads otherwise (3D)
          constexpr bool XSHFL = pipe_depth<NRT>() == 2;
          const int dxm = hxm ? -1 : 0, dxp = hxp ? 1 : 0;
          struct Buf {
            float z[UG], d[UG], h[UG], zk[NRT][UG], xm[UG], xp[UG], edge;
          };
          auto have = [&](int cg) { return cg < BN / UG && qt * BN + cg * UG < a.Q; };
          auto load = [&](int cg, Buf& b) {
            const int q0 = qt * BN + cg * UG;
  #pragma unroll
            for (int j = 0; j < UG; ++j) {
              // a padding column reads the last compartment's row (in bounds), unused;
              // absent neighbours read the voxel's own value and are dropped
              const int64_t o = (int64_t)min(q0 + j, a.Q - 1) * ld + n;
              b.z[j] = __ldg(a.Zin + o);
              b.d[j] = __ldg(a.Din + o);
              b.h[j] = __ldg(a.H + o);
  #pragma unroll
              for (int k = 0; k < NRT; ++k) b.zk[k][j] = __ldg(a.Zin + o + dk[k]);
              if constexpr (!XSHFL) {
                b.xm[j] = __ldg(a.Zin + o + dxm);
                b.xp[j] = __ldg(a.Zin + o + dxp);
              }
            }
            if constexpr (XSHFL) {
              const int je = lane % UG, side = lane / UG;
              const int64_t ne = side == 0 ? (n0w > 0 ? n0w - 1 : n0w)
                                           : side == 1 ? min(n0w + 32, ld - 1) : n0w;
              b.edge = __ldg(a.Zin + (int64_t)min(q0 + je, a.Q - 1) * ld + ne);
            }
          };
          auto process = [&](int cg, Buf& b) {
            const int q0 = qt * BN + cg * UG;
            float v[UG];
            tmem_ld_cols<UG>(
                tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 256 + cg * UG), v);
  #pragma unroll
            for (int j = 0; j < UG; ++j) {
              float zl, zr;
              if constexpr (XSHFL) {
                zl = __shfl_up_sync(0xffffffffu, b.z[j], 1);
                zr = __shfl_down_sync(0xffffffffu, b.z[j], 1);
                const float el = __shfl_sync(0xffffffffu, b.edge, j);
                const float er = __shfl_sync(0xffffffffu, b.edge, UG + j);
                if (lane == 0) zl = el;
                if (lane == 31) zr = er;
              } else {
                zl = b.xm[j];
                zr = b.xp[j];
              }
              float nb = 0.f;
              nb += hxm ? zl : 0.f;
              nb += hxp ? zr : 0.f;
  #pragma unroll
              for (int k = 0; k < NRT; ++k) nb += nok[k] ? b.zk[k][j] : 0.f;
              const int q = q0 + j;
              const float f = __fadd_rn(b.h[j], v[j]);
              float dn, w;
              const float zn = step.apply(b.z[j], b.d[j], f, deg, nb, dn, w);
              if (in && q < a.Q) {
                const int64_t o = (int64_t)q * ld + n;
                a.Zout[o] = zn;
                a.Dout[o] = dn;
                if constexpr (epi_check(EPI)) {
                  const float e = zn - f, ch = zn - b.z[j];
                  s1 = fmaf(e, e, s1);
                  s2 = fmaf(ch, ch, s2);
                  s3 = fmaf(zn, zn, s3);
                }
              }
              v[j] = q < a.Q ? w : 0.f;               // padding columns stay zero
            }
            if (in) {
              uint32_t hh[UG / 2], ll[UG / 2];
  #pragma unroll
              for (int e = 0; e < UG / 2; ++e) {
                const float w0 = v[2 * e], w1 = v[2 * e + 1];
                hh[e] = pack_bf16x2(w0, w1);
                ll[e] = pack_bf16x2(w0 - __bfloat162float(__float2bfloat16_rn(w0)),
                                    w1 - __bfloat162float(__float2bfloat16_rn(w1)));
              }
              *reinterpret_cast<uint4*>(a.Whi + n * a.Qp + q0) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
              *reinterpret_cast<uint4*>(a.Wlo + n * a.Qp + q0) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
            }
            __syncwarp();
          };
          if constexpr (pipe_depth<NRT>() == 2) {
            Buf b0, b1;
            int cg = half;
            if (have(cg)) load(cg, b0);
  #pragma unroll 1
            while (have(cg)) {
              if (have(cg + GS)) load(cg + GS, b1);
              process(cg, b0);
              cg += GS;
              if (!have(cg)) break;
              if (have(cg + GS)) load(cg + GS, b0);
              process(cg, b1);
              cg += GS;
            }
          } else {
            Buf b0;
  #pragma unroll 1
            for (int cg = half; have(cg); cg += GS) {
              load(cg, b0);
              process(cg, b0);
            }
          }
        }
      } else
      for (int cc = half; cc < BN / 32; cc += NEPI / 4) {
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
  if constexpr (epi_check(EPI)) {
    double d1 = s1, d2 = s2, d3 = s3;
    for (int o = 16; o > 0; o >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      d3 += __shfl_xor_sync(0xffffffffu, d3, o);
    }
    __shared__ double red[NTHR / 32][3];
    if (lane == 0) {
      red[warp][0] = d1;
      red[warp][1] = d2;
      red[warp][2] = d3;
    }
    __syncthreads();
    if (tid < 3) {
      double t = 0.0;
      for (int w = 0; w < NTHR / 32; ++w) t += red[w][tid];
      a.partial[(int64_t)blockIdx.x * 4 + tid] = t;
    }
  }
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

template <int BN, int EPI, int NRT>
ssm_status launch_gemm(const ssm_plan_s* pl, int cur, double* partial, cudaStream_t s) {
  const uint64_t Q = (uint64_t)pl->Q, N = (uint64_t)pl->g.N, Qp = (uint64_t)pl->Qp;
  using C = Cfg<BN, EPI, NRT>;
  TcMaps m;
  std::memset(&m, 0, sizeof(m));
  const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
  SSM_CUDA(encode_2d(&m.a_hi, bf, 2, pl->Whi[cur], Q, N, Qp, BK, BM, sw));
  SSM_CUDA(encode_2d(&m.a_lo, bf, 2, pl->Wlo[cur], Q, N, Qp, BK, BM, sw));
  SSM_CUDA(encode_2d(&m.b_hi, bf, 2, pl->Mhi, Q, Q, Qp, BK, BN, sw));
  SSM_CUDA(encode_2d(&m.b_lo, bf, 2, pl->Mlo, Q, Q, Qp, BK, BN, sw));
  if constexpr (C::fused) {
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const uint64_t ld = (uint64_t)pl->g.ld;
    SSM_CUDA(encode_2d(&m.ez_c, f32, 4, pl->Z[cur], N, Q, ld, EZW, UG));
    SSM_CUDA(encode_2d(&m.ez_n, f32, 4, pl->Z[cur], N, Q, ld, ENW, UG));
    SSM_CUDA(encode_2d(&m.ed, f32, 4, pl->Dl[cur], N, Q, ld, BM, UG));
    SSM_CUDA(encode_2d(&m.eh, f32, 4, pl->H, N, Q, ld, BM, UG));
  }
  TcArgs a;
  a.Acc = pl->Acc;
  a.err = pl->dev_err;
  a.g = pl->g;
  a.Q = pl->Q;
  a.ntv = (int)((pl->g.N + BM - 1) / BM);
  a.ntq = (pl->Q + BN - 1) / BN;
  a.Zin = pl->Z[cur];
  a.Din = pl->Dl[cur];
  a.H = pl->H;
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.Whi = pl->Whi[cur ^ 1];
  a.Wlo = pl->Wlo[cur ^ 1];
  a.partial = partial;
  a.mask = pl->mask;
  a.Qp = pl->Qp;
  a.beta = (float)pl->p.beta;
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  tc_gemm_kernel<BN, EPI, NRT><<<gemm_grid(pl, BN), NTHR, C::SMEM_BYTES, s>>>(m, a);
  SSM_LAUNCHED();
  return SSM_OK;
}

// staged neighbour rows of the plan's grid: 4 on 3D grids, else at most 2
int fused_nrt(const ssm_plan_s* pl) { return pl->g.ny > 1 && pl->g.nz > 1 && pl->g.zlink ? 4 : 2; }

template <int BN, int EPI, int NRT>
ssm_status launch_if_valid(const ssm_plan_s* pl, int cur, double* partial, cudaStream_t s) {
  if constexpr (Cfg<BN, EPI, NRT>::valid) {
    return launch_gemm<BN, EPI, NRT>(pl, cur, partial, s);
  } else {
    set_error("tensor-core GEMM: tile width too wide for the fused epilogue's shared memory");
    return SSM_EUNSUPPORTED;
  }
}

template <int EPI, int NRT>
ssm_status gemm_dispatch_n(const ssm_plan_s* pl, int bn, int cur, double* partial, cudaStream_t s) {
  switch (bn) {
    case 256: return launch_if_valid<256, EPI, NRT>(pl, cur, partial, s);
    case 224: return launch_if_valid<224, EPI, NRT>(pl, cur, partial, s);
    case 192: return launch_if_valid<192, EPI, NRT>(pl, cur, partial, s);
    case 160: return launch_if_valid<160, EPI, NRT>(pl, cur, partial, s);
    case 128: return launch_if_valid<128, EPI, NRT>(pl, cur, partial, s);
    default:
      set_error("tensor-core GEMM: unsupported tile width");
      return SSM_EUNSUPPORTED;
  }
}

// whether a tile width has a fused configuration on this plan's grid
bool fused_width_ok(const ssm_plan_s* pl, int bn) {
  const bool four = fused_nrt(pl) == 4;
  switch (bn) {
    case 256: return four ? Cfg<256, 1, 4>::valid : Cfg<256, 1, 2>::valid;
    case 224: return four ? Cfg<224, 1, 4>::valid : Cfg<224, 1, 2>::valid;
    case 192: return four ? Cfg<192, 1, 4>::valid : Cfg<192, 1, 2>::valid;
    case 160: return four ? Cfg<160, 1, 4>::valid : Cfg<160, 1, 2>::valid;
    case 128: return four ? Cfg<128, 1, 4>::valid : Cfg<128, 1, 2>::valid;
    default: return false;
  }
}

template <int EPI>
ssm_status gemm_dispatch(const ssm_plan_s* pl, int bn, int cur, double* partial, cudaStream_t s) {
  if constexpr (EPI != EPI_STORE) {
    if (fused_nrt(pl) == 4) return gemm_dispatch_n<EPI, 4>(pl, bn, cur, partial, s);
  }
  return gemm_dispatch_n<EPI, 2>(pl, bn, cur, partial, s);
}

ssm_status gemm_dispatch(const ssm_plan_s* pl, int bn, int cur, cudaStream_t s) {
  return gemm_dispatch<EPI_STORE>(pl, bn, cur, nullptr, s);
}

template <int BN, int EPI, int NRT>
cudaError_t set_attr_one() {
  if constexpr (Cfg<BN, EPI, NRT>::valid) {
    return cudaFuncSetAttribute(tc_gemm_kernel<BN, EPI, NRT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Cfg<BN, EPI, NRT>::SMEM_BYTES);
  } else {
    return cudaSuccess;
  }
}

template <int BN>
cudaError_t set_smem_attr() {
  for (cudaError_t e : {set_attr_one<BN, EPI_STORE, 2>(), set_attr_one<BN, EPI_UPDATE, 2>(),
                        set_attr_one<BN, EPI_UPDATE_CHECK, 2>(), set_attr_one<BN, EPI_UPDATE, 4>(),
                        set_attr_one<BN, EPI_UPDATE_CHECK, 4>(), set_attr_one<BN, EPI_REG, 2>(),
                        set_attr_one<BN, EPI_REG_CHECK, 2>(), set_attr_one<BN, EPI_REG, 4>(),
                        set_attr_one<BN, EPI_REG_CHECK, 4>()})
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

// choices measured per (device, Q, N, waves, halo rows, fixed tile width), shared by every
// plan of the process
struct TcChoice {
  int bn;        // GEMM width of the two-kernel form and of the register-epilogue kernel
  int bn_fused;  // width of the staged-epilogue kernel (0: none fits)
  int form;      // 0: GEMM + update, 1: fused (staged epilogue), 2: fused (register)
};
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int64_t, int, int, int>, TcChoice> g_tuned;

// Autotuner, on the plan's own operands and state buffers (the solve initialises the
// state, so what these launches write is overwritten): (1) the tile width, timing the
// GEMM alone at every width that pads Q to fewer columns than a wider one; (2) at that
// width, the fused iteration kernel against the GEMM + update pair -- the fused kernel
// wins where its epilogue hides under the tensor-core time (large Q) and loses where the
// element-wise work outweighs the product (small Q). Each candidate gets one warm-up
// launch and two timed ones (CUDA events on the plan's stream). Neither choice changes
// results: each output element sums the same products in the same K order whatever the
// width, and both iteration forms apply the same steps to the same accumulator values.
// SSM_TC_BN / SSM_TC_FUSED fix a choice (tests and sweeps).
ssm_status tune_tile(ssm_plan_s* pl, cudaStream_t s) {
  int fixed_bn = 0, fixed_fused = -1;
  if (const char* env = getenv("SSM_TC_BN")) {
    const int v = atoi(env);
    for (int bn : kTileN)
      if (bn == v) fixed_bn = v;
  }
  if (const char* env = getenv("SSM_TC_FUSED")) {   // 0, 1 (staged) or 2 (register)
    const int v = atoi(env);
    fixed_fused = v >= 0 && v <= 2 ? v : 0;
  }
  if (fixed_bn != 0 && fixed_fused >= 0) {
    if (fixed_fused == 1 && !fused_width_ok(pl, fixed_bn)) {
      set_error("SSM_TC_BN: no fused configuration at this tile width for this grid");
      return SSM_EUNSUPPORTED;
    }
    pl->tc_bn = pl->tc_bn_fused = fixed_bn;
    pl->tc_fused = fixed_fused != 0;
    pl->tc_fused_reg = fixed_fused == 2;
    return SSM_OK;
  }
  const int nr = (pl->g.ny > 1 ? 2 : 0) + (pl->g.nz > 1 && pl->g.zlink ? 2 : 0);
  const auto key = std::make_tuple(pl->device, pl->Q, pl->g.N, pl->waves, nr, fixed_bn);
  auto apply = [&](const TcChoice& c) {
    pl->tc_bn = c.bn;
    pl->tc_bn_fused = c.bn_fused;
    int form = fixed_fused >= 0 ? fixed_fused : c.form;
    if (form == 1 && c.bn_fused == 0) form = 2;   // no staged configuration fits
    pl->tc_fused = form != 0;
    pl->tc_fused_reg = form == 2;
  };
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      apply(it->second);
      return SSM_OK;
    }
  }
  cudaEvent_t e0, e1;
  SSM_CUDA(cudaEventCreate(&e0));
  SSM_CUDA(cudaEventCreate(&e1));
  // one warm-up launch of `run`, then the time of two
  auto timed = [&](auto&& run, float* ms) -> ssm_status {
    SSM_TRY(run());
    SSM_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 2; ++r) SSM_TRY(run());
    SSM_CUDA(cudaEventRecord(e1, s));
    SSM_CUDA(cudaEventSynchronize(e1));
    SSM_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return SSM_OK;
  };
  TcChoice c{fixed_bn != 0 ? fixed_bn : 256, 0, 0};
  ssm_status st = SSM_OK;
  if (fixed_bn == 0) {
    float best_ms = 0.f;
    for (int bn : kTileN) {
      // a width whose tiles do not cover fewer padded columns than a wider one cannot win
      const int pad = (pl->Q + bn - 1) / bn * bn;
      if (bn != 256 && pad >= (pl->Q + 255) / 256 * 256) continue;
      float ms = 0.f;
      st = timed([&] { return gemm_dispatch(pl, bn, 0, s); }, &ms);
      if (st != SSM_OK) break;
      if (bn == 256 || ms < best_ms) {
        c.bn = bn;
        best_ms = ms;
      }
    }
  }
  if (st == SSM_OK) {
    float two_ms = 0.f, fused_ms = 0.f;
    int parts = 0;
    st = timed(
        [&] {
          SSM_TRY(gemm_dispatch(pl, c.bn, 0, s));
          return tc_update(pl, 0, false, nullptr, &parts, s);
        },
        &two_ms);
    // the fused kernel at every width whose configuration fits (its operand ring is
    // shallower, so its best width can differ from the GEMM's)
    for (int bn : kTileN) {
      if (st != SSM_OK) break;
      if (fixed_bn != 0 && bn != fixed_bn) continue;
      if (!fused_width_ok(pl, bn)) continue;
      float ms = 0.f;
      st = timed([&] { return gemm_dispatch<EPI_UPDATE>(pl, bn, 0, nullptr, s); }, &ms);
      if (st == SSM_OK && (c.bn_fused == 0 || ms < fused_ms)) {
        c.bn_fused = bn;
        fused_ms = ms;
      }
    }
    // the register-epilogue kernel at the GEMM's width (it needs no shared memory)
    float reg_ms = 0.f;
    if (st == SSM_OK)
      st = timed([&] { return gemm_dispatch<EPI_REG>(pl, c.bn, 0, nullptr, s); }, &reg_ms);
    c.form = 0;
    float best = two_ms;
    if (c.bn_fused != 0 && fused_ms < best) {
      c.form = 1;
      best = fused_ms;
    }
    if (reg_ms < best) c.form = 2;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SSM_OK) return st;
  apply(c);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned[key] = c;
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

int tc_tile_width(const ssm_plan_s* pl) {
  return pl->tc_fused && !pl->tc_fused_reg ? pl->tc_bn_fused : pl->tc_bn;
}

int tc_gemm_grid(const ssm_plan_s* pl) { return gemm_grid(pl, tc_tile_width(pl)); }

ssm_status tc_iteration(ssm_plan_s* pl, int cur, bool check, double* partial, int* nparts,
                        cudaStream_t s) {
  if (!pl->tc_fused) {
    SSM_TRY(tc_gemm(pl, cur, s));
    return tc_update(pl, cur, check, partial, nparts, s);
  }
  if (pl->tc_fused_reg) {
    *nparts = gemm_grid(pl, pl->tc_bn);
    return check ? gemm_dispatch<EPI_REG_CHECK>(pl, pl->tc_bn, cur, partial, s)
                 : gemm_dispatch<EPI_REG>(pl, pl->tc_bn, cur, partial, s);
  }
  *nparts = gemm_grid(pl, pl->tc_bn_fused);
  return check ? gemm_dispatch<EPI_UPDATE_CHECK>(pl, pl->tc_bn_fused, cur, partial, s)
               : gemm_dispatch<EPI_UPDATE>(pl, pl->tc_bn_fused, cur, partial, s);
}

}  // namespace ssm
