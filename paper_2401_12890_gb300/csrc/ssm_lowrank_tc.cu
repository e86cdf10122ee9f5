// One LADMM iteration of Algorithm 2 (rank-r f-step, Eq. 28) with its two rank-r products
// on the tcgen05 tensor cores ("TF32x3").
//
// The iteration is the d-free recurrence of ssm_lowrank.cu (the algebra is derived there):
// with a_i = S_i/(beta + sigma_i^2) - W_i u_i per voxel (u summed from the previous
// iteration's partial products),
//     t  = z + V a                                              (rank-r product 1)
//     z' = max(0, e1 z + c2 sum_nbr z + c3 (V a))               (Eq. 31)
//     d' = beta (t - z')                                        (step 11)
//     w  = beta (2 z' - t)            (= beta z' - d')
//     u' = V^T w                                                (rank-r product 2)
// For a tile of 128 voxels and a chunk of QC = 32 compartments both products are matrix
// products with the voxels as the M dimension:
//     VA [128 x 32] = A [128 x RP] . V_c^T [RP x 32]      (K = rank, padded to RP = 32/64)
//     U  [128 x RP] = W [128 x 32] . V_c   [32 x RP]      (K = the chunk's compartments)
// Both run as tcgen05.mma kind::tf32 with FP32 accumulation in tensor memory (TMEM). The
// A operands live in TMEM too: the epilogue warps own one voxel (= one TMEM lane) each
// and write a (once per tile segment) and w (per chunk) with tcgen05.st; the B operands
// (the chunk's rows of V and of V^T) are TMA boxes in the 128-byte-swizzled K-major layout.
//
// Precision (TF32x3): each operand x is split as x_hi = tf32(x), x_lo = tf32(x - x_hi)
// (round to nearest), and each product is formed as hi.hi + (hi.lo + lo.hi) (the dropped
// lo.lo term is ~2^-22 relative). The tensor core's FP32 accumulation does not round to
// nearest, so every chain of MMAs into one accumulator is kept short and the two parts
// go to separate accumulators: the main term hi.hi (one MMA per K step of 8) and the
// correction hi.lo + lo.hi (~2^-11 smaller, so its own accumulation error is negligible),
// added in FP32 registers with round-to-nearest. Product 2 starts from zero for every
// chunk and its 32-compartment partial sums are added into registers the same way (a
// chain over all Q compartments would bias u').
//
// Schedule (one CTA per SM): the work units are (segment, tile) pairs, segment-major,
// dealt round-robin to the CTAs; a segment is a contiguous run of a tile's chunks (one
// segment per tile when there are at least as many tiles as CTAs, several otherwise).
// CTAs running together therefore hold the same chunks of consecutive tiles, and the
// neighbour rows each of them stages were just read by another: L2 hits. With between
// half as many tiles as CTAs and as many, each tile is one main unit and one tail unit
// instead, the tails going to the CTAs that would otherwise idle (see layout()). Each segment
// writes its partial u' to its own slot; the next iteration sums a tile's slots in
// segment order (fixed, hence deterministic). Warp roles:
//   warp 0      TMA: per chunk, z with its x halo, the -+nx (-+nx*ny) neighbour rows and
//               the chunk's V / V^T boxes (hi and lo) into a ring of NS stages
//   warp 1      MMA: product 1 of chunk g, then product 2 of chunk g - (NVA - 1) (so the
//               tensor core works ahead of the epilogue); commits release stages and buffers
//   warps 2-9   epilogue (2-17 on 3D grids and in residual-test iterations), two (four)
//               per TMEM lane quarter, each a half (quarter) of a chunk's compartments:
//               tcgen05.ld of V a, the z-step and dual step, z' (and d') stores, w split
//               into TMEM, and the running sum of product 2 in registers
// Waiting warps sleep in mbarrier.try_wait (with a suspend-time hint) instead of polling.
// TMEM: V a (main, correction) and w (hi, lo) are double-buffered by chunk parity, a is
// per segment, U (main, correction) is double-buffered for RP = 32 and single for 64.
// HBM traffic per state element and iteration: read z, write z' (8 B); per voxel and rank:
// S, the partial u in and out. Every mbarrier wait is bounded and reports SSM_ETIMEOUT
// through the plan's device error word; the TMA warp waits (bounded) for its last copies
// and the MMA warp for its last products before the CTA frees its TMEM and exits.
#include <algorithm>
#include <cstdlib>

#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

namespace ssm {
namespace {

constexpr int TV = 128;              // voxels per tile: MMA M, TMEM lanes
constexpr int QC = 32;               // compartments per chunk
// epilogue warps: 8 on 1D/2D grids, 16 on 3D grids (whose elements read four neighbour
// rows: more warps hide their longer latency chains) and in residual-test iterations
// (which also load d^k per element); EPQ per TMEM lane quarter, each taking GC
// compartments of a chunk
template <int NR, bool CHECK> struct Epi {
  static constexpr int NEPI = (NR == 4 || CHECK) ? 16 : 8;
  static constexpr int EPQ = NEPI / 4;
  static constexpr int GC = 32 / EPQ;
  static constexpr int NT = 32 * (2 + NEPI);
  static_assert(NEPI % 4 == 0 && GC % 8 == 0, "epilogue split");
};
constexpr int ZW = TV + 8;           // staged z row: voxels n0-4 .. n0+TV+3
constexpr int NW = TV + 4;           // staged neighbour row: 4-aligned base .. +TV+3
constexpr uint32_t TMEM_COLS = 512;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kPrefetch = 8;         // chunks of a tile's own z rows prefetched into L2 ahead

// Rings, buffers and tensor-memory columns of one kernel configuration.
//   V ring (NSV stages): the chunk's V boxes (B of product 1) and V^T boxes (B of product
//     2), hi and lo; a stage is held from its load until product 2 of its chunk completes
//   z ring (NSZ stages): z with its x halo and the NR neighbour rows; held until the
//     epilogue warps have read it
//   TMEM: V a in NVA buffers (main and correction, 64 columns each), w in 2 (hi and lo),
//     a (hi and lo, per segment), U in UB buffers (main and correction, 2 RP columns)
// Product 1 runs NVA - 1 chunks ahead of the epilogue and the epilogue reads product 2's
// sums two chunks late, so neither MMA latency is on the epilogue's path.
template <int RP, int NR>
struct Lay {
  static constexpr int NVA = RP == 32 ? 3 : 2;
  static constexpr int UB = RP == 32 ? 2 : 1;
  static constexpr int V1 = RP / 32 * QC * 128;   // V rows of the chunk: RP/32 swizzle atoms
  static constexpr int V2 = RP * 128;            // V^T rows (RP) x the chunk (128 bytes)
  static constexpr int v1h = 0, v1l = V1, v2h = 2 * V1, v2l = 2 * V1 + V2;
  static constexpr int VST = 2 * V1 + 2 * V2;    // V stage (a multiple of 1024)
  static constexpr int zc = 0;
  static constexpr int zn = QC * ZW * 4;
  static constexpr int ZST = (zn + NR * QC * NW * 4 + 1023) / 1024 * 1024;
  static constexpr int RESERVE = 1024 + 512;     // alignment slack, barriers, TMEM slot
  static constexpr int STATIC_MAX = 1024;       // the residual variant's reduction array
  static constexpr int budget = kSmemLimit - RESERVE - STATIC_MAX;
  static constexpr int nsz_with(int nsv) { return (budget - nsv * VST) / ZST; }
  static constexpr int NSV = nsz_with(NVA + 1) >= 2 ? NVA + 1 : NVA;
  static constexpr int NSZ = nsz_with(NSV) > 4 ? 4 : nsz_with(NSV);
  static constexpr bool valid = NSZ >= 2 && NSV >= 2;
  static constexpr int zbase = NSV * VST;        // the z ring after the V ring
  static constexpr int bytes = (valid ? zbase + NSZ * ZST : 0) + RESERVE;
  static constexpr unsigned VBYTES = (unsigned)VST;
  static constexpr unsigned ZBYTES = (unsigned)(QC * ZW * 4 + NR * QC * NW * 4);
  static constexpr uint32_t T_VA = 0;                     // buffer b: main 64 b, corr +32
  static constexpr uint32_t T_W = 64 * NVA;               // buffer p: hi 64 p, lo +32
  static constexpr uint32_t T_A = T_W + 128;              // hi, lo at + RP
  static constexpr uint32_t T_U = T_A + 2 * RP;           // buffer b: main 2 RP b, corr + RP
  // kind::tf32 instruction descriptors: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9,
  // 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC1 = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(QC >> 3) << 17) | ((uint32_t)(TV >> 4) << 24);
  static constexpr uint32_t IDESC2 = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(RP >> 3) << 17) | ((uint32_t)(TV >> 4) << 24);
  static_assert(VST % 1024 == 0 && ZST % 1024 == 0 && zn % 128 == 0 && v1l % 1024 == 0 &&
                    v2h % 1024 == 0 && v2l % 1024 == 0,
                "layout");
  static_assert(T_U + 2 * RP * UB <= TMEM_COLS, "tensor memory");
};

struct LrtcMaps {
  CUtensorMap v1h, v1l;   // V (Q x RP), box {32, QC}, 128-byte swizzle
  CUtensorMap v2h, v2l;   // V^T (RP x Qs), box {QC, RP}, 128-byte swizzle
  CUtensorMap zc, zn;     // z^k (Q x N), boxes {ZW, QC} and {NW, QC}
  CUtensorMap dd;         // d^k (Q x N), box {TV, QC}: prefetched into L2 before a residual
                          // test reads it
};

struct LrtcArgs {
  float* __restrict__ Zout;
  float* __restrict__ Dout;         // d^{k+1} (iterations before a residual test)
  const float* __restrict__ Din;    // d^k (residual-test iterations)
  const float* __restrict__ S;      // RP x ld
  const float* __restrict__ Pin;    // partial u of the previous iteration [tile][seg][RP][TV]
  float* __restrict__ Pout;         // partial u of this iteration
  int64_t ntiles;                   // voxel tiles
  int nch;                          // compartment chunks per tile
  int spc;                          // segments per tile (each a contiguous run of chunks)
  int split;                        // > 0: main/tail layout, the chunk where tails start
  int kr;                           // K steps of 8 ranks holding the rank r (<= RP / 8)
  const float* __restrict__ coefA;  // RP
  const float* __restrict__ coefW;  // RP
  double* __restrict__ partial;     // 4 doubles per block (check iterations)
  const uint8_t* __restrict__ mask; // voxels inside the object (nullptr: every voxel)
  int* __restrict__ err;            // device error word
  Grid g;
  int Q;
  float beta, inv_beta, xi, lam_s, inv_xb;
};

__host__ __device__ __forceinline__ int64_t floor4(int64_t v) {
  return v >= 0 ? (v & ~(int64_t)3) : -(((-v) + 3) & ~(int64_t)3);
}

// x rounded to TF32 (10 stored mantissa bits), to nearest with ties away from zero: add
// half a unit of the last kept place to the magnitude bits and clear the 13 bits below
// (a carry into the exponent is the correct rounding up; finite inputs of magnitude
// below 2^128 (1 - 2^-12) stay finite)
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// shared-memory descriptor, K-major operand in the 128-byte swizzle layout (8 rows x
// 128 B atoms, 1024 B apart): start >> 4, leading byte offset 16 B (unused here),
// stride byte offset 1024 B, version 1 (bit 46), swizzle mode 2 = 128 B (bits 61-63)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// D (TMEM) (+)= A (TMEM) . B (shared memory), kind::tf32
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                         uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tst8(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
      : "memory");
}
__device__ __forceinline__ void tst_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// C consecutive 32-bit columns at each of two TMEM addresses (one lane per thread): both
// loads are in flight together and one wait covers them (the outputs are defined by the
// statement that waits, so no use of them can be scheduled before the wait)
template <int C>
__device__ __forceinline__ void tld2(uint32_t t0, uint32_t t1, float* v0, float* v1) {
  static_assert(C == 8 || C == 16, "columns per load");
  uint32_t r[2 * C];
  if constexpr (C == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t0), "r"(t1)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, "
        "%25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(t0), "r"(t1)
        : "memory");
  }
#pragma unroll
  for (int i = 0; i < C; ++i) {
    v0[i] = __uint_as_float(r[i]);
    v1[i] = __uint_as_float(r[C + i]);
  }
}

// C columns (a multiple of 8) at each of two TMEM addresses, 16 (or 8) per wait
template <int C>
__device__ __forceinline__ void tld2_cols(uint32_t t0, uint32_t t1, float* v0, float* v1) {
  static_assert(C % 8 == 0, "columns");
  constexpr int S = C % 16 == 0 ? 16 : 8;
#pragma unroll
  for (int k = 0; k < C; k += S) tld2<S>(t0 + k, t1 + k, v0 + k, v1 + k);
}

template <int RP, int NR, bool CHECK, bool WD>
__global__ void __launch_bounds__(Epi<NR, CHECK>::NT, 1) lrtc_kernel(const __grid_constant__ LrtcMaps maps,
                                                              const LrtcArgs a) {
  using L = Lay<RP, NR>;
  using E = Epi<NR, CHECK>;
  constexpr int NEPI = E::NEPI, EPQ = E::EPQ, GC = E::GC, NT = E::NT;
  constexpr int NSV = L::NSV, NSZ = L::NSZ, NVA = L::NVA, UB = L::UB;
  constexpr int D1 = NVA - 1;         // chunks product 1 runs ahead of product 2
  constexpr int RQ = RP / EPQ;        // ranks per epilogue warp of a lane quarter
  static_assert(L::valid, "two ring stages");
  static_assert(RQ % 8 == 0, "rank split");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // aligned by an offset from the shared array itself (not through an integer), so that
  // the compiler keeps the shared address space of every pointer derived from it
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* vring = smem;
  unsigned char* zring = smem + L::zbase;
  uint64_t* vfull = reinterpret_cast<uint64_t*>(zring + NSZ * L::ZST);
  uint64_t* vempty = vfull + NSV;
  uint64_t* zfull = vempty + NSV;
  uint64_t* zempty = zfull + NSZ;
  uint64_t* va_full = zempty + NSZ;
  uint64_t* va_free = va_full + NVA;
  uint64_t* w_full = va_free + NVA;
  uint64_t* u_full = w_full + 2;
  uint64_t* u_free = u_full + 2;
  uint64_t* a_ready = u_free + 2;
  uint64_t* a_free = a_ready + 1;
  uint64_t* fin = a_free + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nunits = a.ntiles * a.spc;
  const int nch = a.nch, spc = a.spc;

  if (tid == 0) {
    for (int s = 0; s < NSV; ++s) {
      mbar_init(&vfull[s], 1);
      mbar_init(&vempty[s], 1);
    }
    for (int s = 0; s < NSZ; ++s) {
      mbar_init(&zfull[s], 1);
      mbar_init(&zempty[s], NEPI);
    }
    for (int i = 0; i < NVA; ++i) {
      mbar_init(&va_full[i], 1);
      mbar_init(&va_free[i], NEPI);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&w_full[i], NEPI);
      mbar_init(&u_full[i], 1);
      mbar_init(&u_free[i], NEPI);
    }
    mbar_init(a_ready, NEPI);
    mbar_init(a_free, 1);
    mbar_init(fin, 1);
    mbar_fence_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;

  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int64_t plane = (int64_t)nx * ny;
  // neighbour rows beyond x: -nx, +nx, -nx*ny, +nx*ny (the y pair first when there is one)
  const int64_t off[4] = {ny > 1 ? -(int64_t)nx : -plane, ny > 1 ? (int64_t)nx : plane, -plane,
                          plane};
  // unit u = (segment s, tile t), segment-major: the CTAs running together hold the
  // same chunks of consecutive tiles, so the neighbour rows they stage are L2 hits
  auto unit_of = [&](int64_t u, int64_t& tile, int& c0, int& c1, int& sg) {
    sg = (int)(u / a.ntiles);
    tile = u - (int64_t)sg * a.ntiles;
    c0 = (int)((int64_t)sg * nch / spc);
    c1 = (int)((int64_t)(sg + 1) * nch / spc);
  };
  // the k-th unit of this CTA. Main/tail layout (a.split > 0, fewer tiles than CTAs but
  // more than half as many): CTA j < ntiles owns chunks [0, split) of tile j; the other
  // CTAs take the tails [split, nch) of tiles j - ntiles, j - ntiles + (G - ntiles), ...
  // (concurrent tails are of consecutive tiles too). Otherwise units are dealt
  // round-robin in segment-major order.
  auto unit_at = [&](int k, int64_t& tile, int& c0, int& c1, int& sg) -> bool {
    if (a.split > 0) {
      const int64_t j = blockIdx.x, G = gridDim.x;
      if (j < a.ntiles) {
        if (k > 0) return false;
        tile = j;
        sg = 0;
        c0 = 0;
        c1 = a.split;
        return true;
      }
      tile = j - a.ntiles + (int64_t)k * (G - a.ntiles);
      if (tile >= a.ntiles) return false;
      sg = 1;
      c0 = a.split;
      c1 = nch;
      return true;
    }
    const int64_t u = blockIdx.x + (int64_t)k * gridDim.x;
    if (u >= nunits) return false;
    unit_of(u, tile, c0, c1, sg);
    return true;
  };

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_map(&maps.zc);
      tma_prefetch_map(&maps.zn);
      tma_prefetch_map(&maps.v1h);
      tma_prefetch_map(&maps.v2h);
      if (CHECK) tma_prefetch_map(&maps.dd);
      int g = 0;
      int64_t tile;
      int c0, c1, sg;
      for (int k = 0; !failed && unit_at(k, tile, c0, c1, sg); ++k) {
        const int64_t n0 = tile * TV;
        // the tile's own z rows come from HBM: they are prefetched into L2 kPrefetch chunks
        // ahead of their staged loads, so that enough bytes are in flight per SM (the
        // staged loads and the neighbour rows, which other CTAs prefetched, hit L2)
        for (int c = c0 + 1; c < c0 + kPrefetch && c < c1; ++c)
          tma_prefetch_2d(&maps.zc, (int)(n0 - 4), c * QC);
        // a residual test also reads d^k, element by element in the epilogue: its rows
        // are prefetched into L2 the same way (the first kPrefetch chunks at once)
        if (CHECK)
          for (int c = c0; c < c0 + kPrefetch && c < c1; ++c)
            tma_prefetch_2d(&maps.dd, (int)n0, c * QC);
        for (int c = c0; c < c1; ++c, ++g) {
          const int q0 = c * QC;
          if (c + kPrefetch < c1) tma_prefetch_2d(&maps.zc, (int)(n0 - 4), q0 + kPrefetch * QC);
          if (CHECK && c + kPrefetch < c1)
            tma_prefetch_2d(&maps.dd, (int)n0, q0 + kPrefetch * QC);
          // the chunk's V boxes (product 1 needs them first)
          const int sv = g % NSV, kv = g / NSV;
          if (kv > 0 && !mbar_wait_sleep(&vempty[sv], (kv - 1) & 1)) {
            failed = true;
            break;
          }
          unsigned char* vs = vring + sv * L::VST;
          mbar_arrive_expect_tx(&vfull[sv], L::VBYTES);
#pragma unroll
          for (int at = 0; at < RP / 32; ++at) {
            tma_load_2d(vs + L::v1h + at * QC * 128, &maps.v1h, at * 32, q0, &vfull[sv]);
            tma_load_2d(vs + L::v1l + at * QC * 128, &maps.v1l, at * 32, q0, &vfull[sv]);
          }
          tma_load_2d(vs + L::v2h, &maps.v2h, q0, 0, &vfull[sv]);
          tma_load_2d(vs + L::v2l, &maps.v2l, q0, 0, &vfull[sv]);
          // z with its x halo and the neighbour rows
          const int sz = g % NSZ, kz = g / NSZ;
          if (kz > 0 && !mbar_wait_sleep(&zempty[sz], (kz - 1) & 1)) {
            failed = true;
            ++g;          // the V copies of this chunk were issued
            break;
          }
          unsigned char* zs = zring + sz * L::ZST;
          mbar_arrive_expect_tx(&zfull[sz], L::ZBYTES);
          tma_load_2d(zs + L::zc, &maps.zc, (int)(n0 - 4), q0, &zfull[sz]);
#pragma unroll
          for (int j = 0; j < NR; ++j)
            tma_load_2d(zs + L::zn + j * QC * NW * 4, &maps.zn, (int)floor4(n0 + off[j]), q0,
                        &zfull[sz]);
        }
      }
      // no copy may still be in flight when the CTA exits: wait (bounded) for the last
      // phase issued into every stage
      for (int s = 0; s < NSV && s < g; ++s)
        mbar_wait_sleep(&vfull[s], ((s + ((g - 1 - s) / NSV) * NSV) / NSV) & 1);
      for (int s = 0; s < NSZ && s < g; ++s)
        mbar_wait_sleep(&zfull[s], ((s + ((g - 1 - s) / NSZ) * NSZ) / NSZ) & 1);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t a_hi = tmem + L::T_A, a_lo = tmem + L::T_A + RP;
      // product 2 of chunk gg: U (main, correction) = w (hi, lo) . V_c (hi, lo)
      auto product2 = [&](int gg) {
        const int p = gg & 1;
        if (!failed && !mbar_wait_sleep(&w_full[p], (gg >> 1) & 1)) failed = true;
        // the U buffer is free once the epilogue has read chunk gg - UB's
        const int gp = gg - UB;
        if (!failed && gp >= 0 && !mbar_wait_sleep(&u_free[gp & 1], (gp >> 1) & 1))
          failed = true;
        if (failed) return;
        fence_after();
        const uint32_t vs = smem_u32(vring + (gg % NSV) * L::VST);
        const uint32_t dm = tmem + L::T_U + 2 * RP * (gg % UB), dc = dm + RP;
        const uint32_t w_hi = tmem + L::T_W + 64 * p, w_lo = w_hi + 32;
#pragma unroll
        for (int k = 0; k < QC / 8; ++k) {
          const uint64_t bh = sdesc(vs + L::v2h + k * 32), bl = sdesc(vs + L::v2l + k * 32);
          mma_tf32(dm, w_hi + 8 * k, bh, L::IDESC2, k > 0 ? 1u : 0u);
          mma_tf32(dc, w_hi + 8 * k, bl, L::IDESC2, k > 0 ? 1u : 0u);
          mma_tf32(dc, w_lo + 8 * k, bh, L::IDESC2, 1u);
        }
        commit(&u_full[p]);
        commit(&vempty[gg % NSV]);    // the V stage is free once these complete
      };
      int g = 0, si = 0;
      int64_t tile;
      int c0, c1, sg;
      for (int k = 0; !failed && unit_at(k, tile, c0, c1, sg); ++k) {
        const int nchk = c1 - c0;
        if (!mbar_wait_sleep(a_ready, si & 1)) {
          failed = true;
          break;
        }
        fence_after();
        for (int i = 0; i < nchk && !failed; ++i) {
          // product 1 of chunk gg: V a (main, correction) = a (hi, lo) . V_c^T (hi, lo)
          const int gg = g + i, b = gg % NVA;
          if (!mbar_wait_sleep(&vfull[gg % NSV], (gg / NSV) & 1)) failed = true;
          if (!failed && gg >= NVA && !mbar_wait_sleep(&va_free[b], ((gg / NVA) - 1) & 1))
            failed = true;
          if (failed) break;
          fence_after();
          const uint32_t vs = smem_u32(vring + (gg % NSV) * L::VST);
          const uint32_t dm = tmem + L::T_VA + 64 * b, dc = dm + 32;
          // the padding ranks beyond r carry zero a: their K steps are skipped
#pragma unroll 4
          for (int k = 0; k < a.kr; ++k) {
            const int at = k / 4, o = (k % 4) * 32;
            const uint64_t bh = sdesc(vs + L::v1h + at * QC * 128 + o);
            const uint64_t bl = sdesc(vs + L::v1l + at * QC * 128 + o);
            mma_tf32(dm, a_hi + 8 * k, bh, L::IDESC1, k > 0 ? 1u : 0u);
            mma_tf32(dc, a_hi + 8 * k, bl, L::IDESC1, k > 0 ? 1u : 0u);
            mma_tf32(dc, a_lo + 8 * k, bh, L::IDESC1, 1u);
          }
          commit(&va_full[b]);
          if (i == nchk - 1) commit(a_free);     // a may be rewritten once these complete
          if (i >= D1) product2(gg - D1);
        }
        // the segment's last products 2
        for (int j = (nchk > D1 ? nchk - D1 : 0); j < nchk && !failed; ++j) product2(g + j);
        g += nchk;
        ++si;
      }
      // every product issued has completed before the TMEM is freed
      commit(fin);
      mbar_wait_sleep(fin, 0);
    }
  } else {
    // ------------------------------------------------------------------ epilogue warps
    const int quarter = warp & 3;
    const int grp = (warp - 2) >> 2;                 // compartments grp*GC .. of a chunk
    const int v = quarter * 32 + lane;               // voxel within the tile = TMEM lane
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int64_t ld = a.g.ld, N = a.g.N;
    const int Q = a.Q;
    const bool zl = nz > 1 && a.g.zlink;
    const float c2 = a.lam_s * a.inv_xb;             // weight of the neighbour sum
    const float c3 = a.beta * a.inv_xb;              // weight of V a
    const float beta = a.beta, inv_beta = a.inv_beta;
    const float2 c2_2 = make_float2(c2, c2), c3_2 = make_float2(c3, c3);
    const float2 beta2 = make_float2(beta, beta), two2 = make_float2(2.f, 2.f);
    int g = 0, si = 0;
    int64_t tile;
    int c0, c1, sg;
    for (int k = 0; unit_at(k, tile, c0, c1, sg); ++k) {
      const int nchk = c1 - c0;
      const int64_t n0 = tile * TV;
      const int64_t n = n0 + v;
      const bool valid = n < N;
      // voxel coordinates in 32-bit arithmetic (N < 2^31)
      int x = 0, y = 0, zc = 0;
      if (valid) {
        const unsigned nn = (unsigned)n, t = nn / (unsigned)nx;
        x = (int)(nn - t * (unsigned)nx);
        y = (int)(t % (unsigned)ny);
        zc = (int)(t / (unsigned)ny);
      }
      // a voxel outside the object is left alone (its z stays 0) and is nobody's neighbour
      const uint8_t* mk = a.mask;
      const bool in = valid && (!mk || mk[n]);
      const bool hxm = in && x > 0 && (!mk || mk[n - 1]);
      const bool hxp = in && x < nx - 1 && (!mk || mk[n + 1]);
      const bool hym = in && y > 0 && (!mk || mk[n - nx]);
      const bool hyp = in && y < ny - 1 && (!mk || mk[n + nx]);
      const bool hzm = zl && in && zc > 0 && (!mk || mk[n - plane]);
      const bool hzp = zl && in && zc < nz - 1 && (!mk || mk[n + plane]);
      const float deg = (float)(hxm + hxp + hym + hyp + hzm + hzp);
      const float e1 = (a.xi + a.beta - a.lam_s * deg) * a.inv_xb;   // weight of z
      // neighbour presence as 0/1 weights: the staged rows are always readable (finite
      // z values or the copy's zero fill), so every neighbour term is a fused add
      const float fxm = hxm ? 1.f : 0.f, fxp = hxp ? 1.f : 0.f;
      const float2 fxm2 = make_float2(fxm, fxm), fxp2 = make_float2(fxp, fxp);
      const float2 e1_2 = make_float2(e1, e1);
      int nidx[4];
      float fk[4];
      {
        const bool flags[4] = {ny > 1 ? hym : hzm, ny > 1 ? hyp : hzp, hzm, hzp};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          nidx[j] = j < NR ? (int)(n + off[j] - floor4(n0 + off[j])) : 0;
          fk[j] = (j < NR && flags[j]) ? 1.f : 0.f;
        }
      }
      float2 fk2[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) fk2[j] = make_float2(fk[j], fk[j]);
      // a for this warp's ranks: a_i = S_i/(beta + sigma_i^2) - W_i u_i, u_i summed over
      // the tile's segment slots of the previous iteration in segment order
      if (si > 0 && !failed && !mbar_wait_sleep(a_free, (si - 1) & 1)) failed = true;
      fence_after();
      {
        float ah[RQ], al[RQ];
        const float* pt = a.Pin + (tile * spc) * (int64_t)(RP * TV) + grp * RQ * TV + v;
        const float* sp = a.S + (int64_t)(grp * RQ) * ld + n;
        // every load of the a-vector is issued before any is used
        float us[RQ], sv[RQ];
#pragma unroll
        for (int i = 0; i < RQ; ++i) {
          sv[i] = in ? __ldg(sp + i * ld) : 0.f;
          us[i] = in ? pt[i * TV] : 0.f;
        }
        for (int k = 1; k < spc; ++k) {
#pragma unroll
          for (int i = 0; i < RQ; ++i) us[i] += in ? pt[(k * RP + i) * TV] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < RQ; ++i) {
          const int r = grp * RQ + i;
          const float av = in ? sv[i] * __ldg(a.coefA + r) - __ldg(a.coefW + r) * us[i] : 0.f;
          ah[i] = tf32_rna(av);
          al[i] = tf32_rna(av - ah[i]);
        }
#pragma unroll
        for (int i = 0; i < RQ; i += 8) {
          tst8(tmem + lane_base + L::T_A + grp * RQ + i, ah + i);
          tst8(tmem + lane_base + L::T_A + RP + grp * RQ + i, al + i);
        }
        tst_wait();
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_ready);
      float uacc[RQ];
#pragma unroll
      for (int i = 0; i < RQ; ++i) uacc[i] = 0.f;
      // product 2's sums of chunk gg (main + correction, rounded to nearest in registers)
      auto consume_u = [&](int gg) {
        const int p = gg & 1;
        if (!failed && !mbar_wait_sleep(&u_full[p], (gg >> 1) & 1)) failed = true;
        fence_after();
        const uint32_t ub = tmem + lane_base + L::T_U + 2 * RP * (gg % UB) + grp * RQ;
        {
          float um[RQ], uc[RQ];
          tld2_cols<RQ>(ub, ub + RP, um, uc);
#pragma unroll
          for (int j = 0; j < RQ; j += 2) {
            const float2 t2 = __fadd2_rn(make_float2(um[j], um[j + 1]), make_float2(uc[j], uc[j + 1]));
            const float2 s2 = __fadd2_rn(make_float2(uacc[j], uacc[j + 1]), t2);
            uacc[j] = s2.x;
            uacc[j + 1] = s2.y;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&u_free[p]);
      };
      for (int i = 0; i < nchk; ++i) {
        const int gg = g + i, sz = gg % NSZ, b = gg % NVA, p = gg & 1;
        const int qg = (c0 + i) * QC + grp * GC;   // this warp's first compartment
        // a residual test needs d^k, read from global memory element by element: the
        // chunk's loads are issued before the waits, so that their latency overlaps the
        // chunk's processing (loading them where they are used cost 2.7x per iteration)
        float dkc[CHECK ? GC : 1];
        if constexpr (CHECK) {
          const int jn0 = min(GC, Q - qg);
          const float* dq = a.Din + (int64_t)qg * ld + n;
#pragma unroll
          for (int j = 0; j < GC; ++j) dkc[j] = (in && j < jn0) ? __ldg(dq + j * ld) : 0.f;
        }
        if (!failed && !mbar_wait_sleep(&zfull[sz], (gg / NSZ) & 1)) failed = true;
        if (!failed && !mbar_wait_sleep(&va_full[b], (gg / NVA) & 1)) failed = true;
        fence_after();
        float va[GC];
        {
          float vc[GC];
          const uint32_t tb = tmem + lane_base + L::T_VA + 64 * b + grp * GC;
          tld2_cols<GC>(tb, tb + 32, va, vc);
#pragma unroll
          for (int k = 0; k < GC; k += 2) {
            const float2 s2 = __fadd2_rn(make_float2(va[k], va[k + 1]), make_float2(vc[k], vc[k + 1]));
            va[k] = s2.x;
            va[k + 1] = s2.y;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&va_free[b]);
        const bool work = in && !failed;
        const int jn = min(GC, Q - qg);              // the same for every lane
        const float* zcr = reinterpret_cast<const float*>(zring + sz * L::ZST + L::zc) +
                           grp * GC * ZW + 4 + v;
        const float* znr = reinterpret_cast<const float*>(zring + sz * L::ZST + L::zn) +
                           grp * GC * NW;
        float w[GC];
        float* zp = a.Zout + (int64_t)qg * ld + n;
        if (work) {
          // in halves of 8 compartments: the staged rows first (all shared-memory loads of
          // the half in flight at once, before any store to global memory), then the
          // arithmetic, then the stores
#pragma unroll
          for (int h = 0; h < GC; h += 8) {
            // compartments in pairs, in packed FP32x2 arithmetic: each half of an FP32x2
            // operation rounds as the scalar one, so the values are those of scalar code
            float2 zz2[4], nb2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = h + 2 * j;
              zz2[j] = make_float2(zcr[r * ZW], zcr[(r + 1) * ZW]);
              nb2[j] = __fmul2_rn(fxm2, make_float2(zcr[r * ZW - 1], zcr[(r + 1) * ZW - 1]));
              nb2[j] = __ffma2_rn(fxp2, make_float2(zcr[r * ZW + 1], zcr[(r + 1) * ZW + 1]), nb2[j]);
#pragma unroll
              for (int k = 0; k < NR; ++k)
                nb2[j] = __ffma2_rn(fk2[k],
                                    make_float2(znr[(k * QC + r) * NW + nidx[k]],
                                                znr[(k * QC + r + 1) * NW + nidx[k]]),
                                    nb2[j]);
            }
            float zz[8], zn[8], tt[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = h + 2 * j;
              const float2 va2 = make_float2(va[r], va[r + 1]);
              const float2 y = __ffma2_rn(e1_2, zz2[j], __ffma2_rn(c2_2, nb2[j], __fmul2_rn(c3_2, va2)));
              const float2 z2 = make_float2(fmaxf(0.f, y.x), fmaxf(0.f, y.y));
              const float2 t2 = __fadd2_rn(zz2[j], va2);
              const float2 w2 =
                  __fmul2_rn(beta2, __ffma2_rn(two2, z2, make_float2(-t2.x, -t2.y)));
              zz[2 * j] = zz2[j].x;
              zz[2 * j + 1] = zz2[j].y;
              zn[2 * j] = z2.x;
              zn[2 * j + 1] = z2.y;
              tt[2 * j] = t2.x;
              tt[2 * j + 1] = t2.y;
              // compartments past Q read the copies' zero fill (z) and zero rows of V
              // (V a): their w is exactly 0 without a test
              w[r] = w2.x;
              w[r + 1] = w2.y;
            }
            if constexpr (CHECK) {
              // f^{k+1} = t - d^k / beta needs d^k
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (h + j < jn) {
                  const float f = tt[j] - dkc[h + j] * inv_beta;
                  const float e = zn[j] - f, ch = zn[j] - zz[j];
                  s1 = fmaf(e, e, s1);
                  s2 = fmaf(ch, ch, s2);
                  s3 = fmaf(zn[j], zn[j], s3);
                }
            }
            if (jn == GC) {
#pragma unroll
              for (int j = 0; j < 8; ++j) __stcs(zp + (h + j) * ld, zn[j]);
              if constexpr (WD) {
                float* dp = a.Dout + (zp - a.Zout);
#pragma unroll
                for (int j = 0; j < 8; ++j) dp[(h + j) * ld] = beta * (tt[j] - zn[j]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (h + j < jn) {
                  zp[(h + j) * ld] = zn[j];
                  if constexpr (WD) a.Dout[(zp - a.Zout) + (h + j) * ld] = beta * (tt[j] - zn[j]);
                }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < GC; ++j) w[j] = 0.f;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&zempty[sz]);   // the staged rows are no longer read
        // product 2 of chunk gg - 2 has completed (it read the w buffer about to be
        // rewritten); its sums join the running u'
        if (i >= 2) consume_u(gg - 2);
#pragma unroll
        for (int j = 0; j < GC; j += 8) {
          float wh[8], wl[8];
#pragma unroll
          for (int k = 0; k < 8; k += 2) {
            wh[k] = tf32_rna(w[j + k]);
            wh[k + 1] = tf32_rna(w[j + k + 1]);
            const float2 l2 = __fadd2_rn(make_float2(w[j + k], w[j + k + 1]),
                                         make_float2(-wh[k], -wh[k + 1]));
            wl[k] = tf32_rna(l2.x);
            wl[k + 1] = tf32_rna(l2.y);
          }
          tst8(tmem + lane_base + L::T_W + 64 * p + grp * GC + j, wh);
          tst8(tmem + lane_base + L::T_W + 64 * p + 32 + grp * GC + j, wl);
        }
        tst_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&w_full[p]);
      }
      for (int j = (nchk > 2 ? nchk - 2 : 0); j < nchk; ++j) consume_u(g + j);
      // this segment's partial u' (zero for voxels past the grid or outside the object)
      float* po = a.Pout + ((tile * spc + sg) * (int64_t)RP) * TV;
#pragma unroll
      for (int i = 0; i < RQ; ++i) po[(grp * RQ + i) * TV + v] = in ? uacc[i] : 0.f;
      g += nchk;
      ++si;
    }
  }
  if (failed) atomicExch(a.err, (int)SSM_ETIMEOUT);
  if constexpr (CHECK) {
    double d1 = s1, d2 = s2, d3 = s3;
    for (int o = 16; o > 0; o >>= 1) {
      d1 += __shfl_xor_sync(0xffffffffu, d1, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      d3 += __shfl_xor_sync(0xffffffffu, d3, o);
    }
    __shared__ double red[NT / 32][3];
    if (lane == 0) {
      red[warp][0] = d1;
      red[warp][1] = d2;
      red[warp][2] = d3;
    }
    __syncthreads();
    if (tid < 3) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += red[w][tid];
      a.partial[(int64_t)blockIdx.x * 4 + tid] = t;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// V (Q x RP) and V^T (RP x Qs), each split into TF32 hi/lo parts (round to nearest)
__global__ void split_basis_kernel(const float* __restrict__ V32, int Q, int RP, int Qs,
                                   float* __restrict__ v1h, float* __restrict__ v1l,
                                   float* __restrict__ v2h, float* __restrict__ v2l) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)RP * Qs) return;
  const int i = (int)(idx / Qs), q = (int)(idx % Qs);
  const float x = q < Q ? V32[(int64_t)q * RP + i] : 0.f;
  const float h = tf32_rna(x);
  const float l = tf32_rna(x - h);
  v2h[idx] = h;
  v2l[idx] = l;
  if (q < Q) {
    v1h[(int64_t)q * RP + i] = h;
    v1l[(int64_t)q * RP + i] = l;
  }
}

template <int RP, int NR, bool CHECK, bool WD>
ssm_status set_attr() {
  return cudaFuncSetAttribute(lrtc_kernel<RP, NR, CHECK, WD>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Lay<RP, NR>::bytes) == cudaSuccess
             ? SSM_OK
             : SSM_ECUDA;
}

template <int RP, int NR>
ssm_status prepare_rn() {
  if constexpr (Lay<RP, NR>::valid) {
    SSM_TRY((set_attr<RP, NR, false, false>()));
    SSM_TRY((set_attr<RP, NR, false, true>()));
    SSM_TRY((set_attr<RP, NR, true, false>()));
    SSM_TRY((set_attr<RP, NR, true, true>()));
  }
  return SSM_OK;
}

template <int RP, int NR>
ssm_status launch_rn(const LrtcMaps& maps, const LrtcArgs& args, bool check, bool write_d,
                     int64_t grid, cudaStream_t s) {
  if constexpr (!Lay<RP, NR>::valid) {
    set_error("tensor-core low-rank form: this rank does not fit on 3D grids (r <= 32)");
    return SSM_EUNSUPPORTED;
  } else {
    const size_t shm = Lay<RP, NR>::bytes;
    const unsigned gr = (unsigned)grid;
    if (check && write_d)
      lrtc_kernel<RP, NR, true, true><<<gr, Epi<NR, true>::NT, shm, s>>>(maps, args);
    else if (check)
      lrtc_kernel<RP, NR, true, false><<<gr, Epi<NR, true>::NT, shm, s>>>(maps, args);
    else if (write_d)
      lrtc_kernel<RP, NR, false, true><<<gr, Epi<NR, false>::NT, shm, s>>>(maps, args);
    else
      lrtc_kernel<RP, NR, false, false><<<gr, Epi<NR, false>::NT, shm, s>>>(maps, args);
    SSM_LAUNCHED();
    return SSM_OK;
  }
}

int grid_nr(const ssm_plan_s* pl) {
  return (pl->g.ny > 1 ? 2 : 0) + (pl->g.nz > 1 && pl->g.zlink ? 2 : 0);
}

int64_t ntiles_of(const ssm_plan_s* pl) { return (pl->g.N + TV - 1) / TV; }
int64_t chunks_of(const ssm_plan_s* pl) { return (pl->Q + QC - 1) / QC; }

// Launch layout: the CTAs' budget G0 (one per SM per launch wave).
//  - At least G0 tiles: every tile is one unit (its whole Q range) and the grid is the
//    fewest CTAs that keep the rounds of G tiles equal.
//  - Between G0/2 and G0 tiles (the 128x128 slice: 128 tiles, 152 SMs): one segment per
//    tile would leave G0 - ntiles SMs idle, two would give some CTAs two whole-Q-halves
//    of work; instead CTA j < ntiles takes chunks [0, split) of tile j and the spare
//    CTAs take the tails, `split` chosen so that both kinds finish together (counting a
//    unit's start as one chunk). On the slice: 126 us per launch at split 69 (150 CTAs)
//    against 136 us with one segment per tile (128 CTAs); splits of 60 and 64 overload
//    the tail CTAs (209 and 172 us).
//  - Fewer tiles: each tile is split into spc equal segments so that all CTAs have work.
void layout(const ssm_plan_s* pl, int64_t* grid, int* spc, int* split) {
  const int64_t ntiles = ntiles_of(pl), nch = chunks_of(pl);
  int64_t g0 = (int64_t)sm_count() * std::max(1, pl->waves);
  if (const char* env = getenv("SSM_LRTC_GRID")) {   // launch-shape override for sweeps
    const long v = atol(env);
    if (v >= 1 && v <= 65536) g0 = v;
  }
  int64_t force_split = -1;
  if (const char* env = getenv("SSM_LRTC_SPLIT")) {  // 0: no main/tail layout (sweeps)
    const long v = atol(env);
    if (v >= 0 && v < nch) force_split = v;
  }
  *split = 0;
  if (ntiles >= g0) {
    const int64_t rounds = (ntiles + g0 - 1) / g0;
    *spc = 1;
    *grid = (ntiles + rounds - 1) / rounds;
  } else if (2 * ntiles > g0 && nch >= 4 && force_split != 0) {
    const int64_t spare = g0 - ntiles;
    const int64_t per = (ntiles + spare - 1) / spare;   // tails per spare CTA
    int64_t best = 1, cost = INT64_MAX;
    for (int64_t c = 1; c < nch; ++c) {
      const int64_t t = std::max(c + 1, per * (nch - c + 1));
      if (t < cost) {
        cost = t;
        best = c;
      }
    }
    if (force_split > 0) best = force_split;
    *split = (int)best;
    *spc = 2;
    *grid = ntiles + (ntiles + per - 1) / per;
  } else {
    *spc = (int)std::max<int64_t>(1, std::min(nch, g0 / ntiles));
    *grid = ntiles * *spc;
  }
}

}  // namespace

// padded rank of the tensor-core low-rank form: 32 or 64 (0: not supported)
int lrtc_padded_rank(int r, bool three_d) {
  if (r <= 32) return 32;
  if (r <= 64 && !three_d) return 64;
  return 0;
}

int64_t lrtc_grid(const ssm_plan_s* pl) {
  int64_t grid;
  int spc, split;
  layout(pl, &grid, &spc, &split);
  return grid;
}

int64_t lrtc_partial_floats(const ssm_plan_s* pl, int64_t grid) {
  (void)grid;
  int64_t g;
  int spc, split;
  layout(pl, &g, &spc, &split);
  return ntiles_of(pl) * spc * (int64_t)pl->R * TV;
}

// once per process and device: the kernels' shared-memory limits
ssm_status lrtc_prepare() {
  std::lock_guard<std::mutex> lock(attr_mutex());
  SSM_TRY((prepare_rn<32, 0>()));
  SSM_TRY((prepare_rn<32, 2>()));
  SSM_TRY((prepare_rn<32, 4>()));
  SSM_TRY((prepare_rn<64, 0>()));
  SSM_TRY((prepare_rn<64, 2>()));
  return SSM_OK;
}

// the TF32 hi/lo parts of V and V^T from the plan's FP32 basis V32 (Q x R)
ssm_status lrtc_split_basis(ssm_plan_s* pl, cudaStream_t s) {
  const int Qs = pl->lrtc_qs;
  const int64_t cnt = (int64_t)pl->R * Qs;
  split_basis_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(
      pl->V32, pl->Q, pl->R, Qs, pl->V1h, pl->V1l, pl->V2h, pl->V2l);
  SSM_LAUNCHED();
  return SSM_OK;
}

ssm_status lrtc_iteration(ssm_plan_s* pl, int cur, bool check, bool write_d, double* partial,
                          int* nparts, cudaStream_t s) {
  const uint64_t N = (uint64_t)pl->g.N, Q = (uint64_t)pl->Q, ld = (uint64_t)pl->g.ld;
  const uint64_t RP = (uint64_t)pl->R, Qs = (uint64_t)pl->lrtc_qs;
  LrtcMaps m;
  const auto SW = CU_TENSOR_MAP_SWIZZLE_128B;
  const auto F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  SSM_CUDA(encode_2d(&m.v1h, F32, 4, pl->V1h, RP, Q, RP, 32, QC, SW));
  SSM_CUDA(encode_2d(&m.v1l, F32, 4, pl->V1l, RP, Q, RP, 32, QC, SW));
  SSM_CUDA(encode_2d(&m.v2h, F32, 4, pl->V2h, Q, RP, Qs, QC, (unsigned)RP, SW));
  SSM_CUDA(encode_2d(&m.v2l, F32, 4, pl->V2l, Q, RP, Qs, QC, (unsigned)RP, SW));
  SSM_CUDA(encode_2d(&m.zc, F32, 4, pl->Z[cur], N, Q, ld, ZW, QC));
  SSM_CUDA(encode_2d(&m.zn, F32, 4, pl->Z[cur], N, Q, ld, NW, QC));
  SSM_CUDA(encode_2d(&m.dd, F32, 4, pl->Dl[cur], N, Q, ld, TV, QC));
  int64_t grid;
  int spc, split;
  layout(pl, &grid, &spc, &split);
  if (grid != pl->lr_grid) {
    set_error("tensor-core low-rank form: launch layout changed since planning");
    return SSM_ECUDA;
  }
  LrtcArgs a;
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.Din = pl->Dl[cur];
  a.S = pl->S;
  a.Pin = pl->U[cur];
  a.Pout = pl->U[cur ^ 1];
  a.ntiles = ntiles_of(pl);
  a.nch = (int)chunks_of(pl);
  a.spc = spc;
  a.split = split;
  a.kr = std::max(1, std::min((int)RP / 8, (pl->r + 7) / 8));
  a.coefA = pl->coefA;
  a.coefW = pl->coefW;
  a.partial = partial;
  a.mask = pl->mask;
  a.err = pl->dev_err;
  a.g = pl->g;
  a.Q = pl->Q;
  a.beta = (float)pl->p.beta;
  a.inv_beta = (float)(1.0 / pl->p.beta);
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  *nparts = (int)grid;
  const int nr = grid_nr(pl);
  if (pl->R == 32) {
    if (nr == 0) return launch_rn<32, 0>(m, a, check, write_d, grid, s);
    if (nr == 2) return launch_rn<32, 2>(m, a, check, write_d, grid, s);
    return launch_rn<32, 4>(m, a, check, write_d, grid, s);
  }
  if (pl->R == 64) {
    if (nr == 0) return launch_rn<64, 0>(m, a, check, write_d, grid, s);
    if (nr == 2) return launch_rn<64, 2>(m, a, check, write_d, grid, s);
    return launch_rn<64, 4>(m, a, check, write_d, grid, s);
  }
  set_error("tensor-core low-rank form: unsupported padded rank");
  return SSM_EUNSUPPORTED;
}

}  // namespace ssm
