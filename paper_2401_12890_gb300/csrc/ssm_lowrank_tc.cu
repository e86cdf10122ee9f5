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
// (round to nearest), and each product is accumulated as hi.hi + hi.lo + lo.hi (the
// dropped lo.lo term is ~2^-22 relative). The chain of MMAs into one accumulator is kept
// short: product 1 sums RP ranks; product 2 starts from zero for every chunk, and its
// 32-compartment partial sums are added into FP32 registers with round-to-nearest
// (the tensor core's accumulation does not round to nearest, and a chain over all Q
// compartments would bias u').
//
// Schedule (persistent, one CTA per SM): the work is the flattened list of (voxel tile,
// compartment chunk) units; each CTA takes an equal contiguous share, split into
// segments at tile boundaries. Warp roles:
//   warp 0      TMA: per chunk, z with its x halo, the -+nx (-+nx*ny) neighbour rows and
//               the chunk's V / V^T boxes (hi and lo) into a ring of NS stages
//   warp 1      MMA: product 1 of chunk g, then product 2 of chunk g-1 (so the tensor
//               core works ahead of the epilogue); commits release stages and buffers
//   warps 2-9   epilogue, two per TMEM lane quarter, each half of a chunk's compartments:
//               tcgen05.ld of V a, the z-step and dual step, z' (and d') stores, w split
//               into TMEM, and the running sum of product 2 in registers
// TMEM: V a and w are double-buffered by chunk parity, a is per segment, U by parity.
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
constexpr int HC = QC / 2;           // compartments per epilogue warp and chunk
constexpr int NEPI = 8;              // epilogue warps (two per TMEM lane quarter)
constexpr int NT = 32 * (2 + NEPI);
constexpr int ZW = TV + 8;           // staged z row: voxels n0-4 .. n0+TV+3
constexpr int NW = TV + 4;           // staged neighbour row: 4-aligned base .. +TV+3
constexpr uint32_t TMEM_COLS = 512;
constexpr int kSmemLimit = 227 * 1024;

// TMEM column map (RP-independent part)
constexpr uint32_t T_VA = 0;         // V a: chunk parity p at 32 p
constexpr uint32_t T_W = 64;         // w: parity p at 64 + 64 p (hi), +32 (lo)
constexpr uint32_t T_A = 192;        // a: hi at 192, lo at 192 + RP

template <int RP, int NR>
struct Lay {
  static constexpr int V1 = RP / 32 * QC * 128;   // V rows of the chunk: RP/32 swizzle atoms
  static constexpr int V2 = RP * 128;            // V^T rows (RP) x the chunk (128 bytes)
  static constexpr int v1h = 0, v1l = V1, v2h = 2 * V1, v2l = 2 * V1 + V2;
  static constexpr int zc = 2 * V1 + 2 * V2;
  static constexpr int zn = zc + QC * ZW * 4;
  static constexpr int raw = zn + NR * QC * NW * 4;
  static constexpr int stage = (raw + 1023) / 1024 * 1024;
  static constexpr int RESERVE = 1024 + 512;     // alignment slack, barriers, TMEM slot
  static constexpr int STATIC_MAX = 1024;       // the residual variant's reduction array
  static constexpr int ns_fit = (kSmemLimit - RESERVE - STATIC_MAX) / stage;
  static constexpr int NS = ns_fit > 4 ? 4 : ns_fit;
  static constexpr bool valid = NS >= 2;
  static constexpr int bytes = (NS < 1 ? 1 : NS) * stage + RESERVE;
  static constexpr uint32_t T_U = T_A + 2 * RP;  // U: parity p at T_U + RP p
  // kind::tf32 instruction descriptors: D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9,
  // 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC1 = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(QC >> 3) << 17) | ((uint32_t)(TV >> 4) << 24);
  static constexpr uint32_t IDESC2 = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(RP >> 3) << 17) | ((uint32_t)(TV >> 4) << 24);
  static_assert(zc % 1024 == 0 && zn % 128 == 0 && v1l % 1024 == 0 && v2h % 1024 == 0 &&
                    v2l % 1024 == 0,
                "layout");
  static_assert(T_U + 2 * RP <= TMEM_COLS, "tensor memory");
};

struct LrtcMaps {
  CUtensorMap v1h, v1l;   // V (Q x RP), box {32, QC}, 128-byte swizzle
  CUtensorMap v2h, v2l;   // V^T (RP x Qs), box {QC, RP}, 128-byte swizzle
  CUtensorMap zc, zn;     // z^k (Q x N), boxes {ZW, QC} and {NW, QC}
};

struct LrtcArgs {
  float* __restrict__ Zout;
  float* __restrict__ Dout;         // d^{k+1}, written when write_d != 0
  const float* __restrict__ Din;    // d^k (residual-test iterations)
  const float* __restrict__ S;      // RP x ld
  const float* __restrict__ Pin;    // partial u of the previous iteration [tile][seg][RP][TV]
  float* __restrict__ Pout;         // partial u of this iteration
  int64_t ntiles, T;                // tiles, units (ntiles * nch)
  int nch;                          // chunks per tile
  int maxseg;                       // segment slots per tile
  const float* __restrict__ coefA;  // RP
  const float* __restrict__ coefW;  // RP
  double* __restrict__ partial;     // 4 doubles per block (check iterations)
  const uint8_t* __restrict__ mask; // voxels inside the object (nullptr: every voxel)
  int* __restrict__ err;            // device error word
  Grid g;
  int Q;
  int write_d;
  float beta, inv_beta, xi, lam_s, inv_xb;
};

__host__ __device__ __forceinline__ int64_t floor4(int64_t v) {
  return v >= 0 ? (v & ~(int64_t)3) : -(((-v) + 3) & ~(int64_t)3);
}
__host__ __device__ __forceinline__ int64_t share_lo(int64_t T, int64_t j, int64_t G) {
  return (T * j) / G;
}
// the first CTA whose share contains unit u
__host__ __device__ __forceinline__ int64_t owner_of(int64_t u, int64_t T, int64_t G) {
  return ((u + 1) * G + T - 1) / T - 1;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
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

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes (one lane per thread)
__device__ __forceinline__ void tld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tst16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tst_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int RP, int NR, bool CHECK>
__global__ void __launch_bounds__(NT, 1) lrtc_kernel(const __grid_constant__ LrtcMaps maps,
                                                     const LrtcArgs a) {
  using L = Lay<RP, NR>;
  constexpr int NS = L::NS;
  constexpr int RH = RP / 2;          // ranks per epilogue half
  static_assert(L::valid, "two ring stages");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * L::stage);
  uint64_t* empty = full + NS;
  uint64_t* va_full = empty + NS;
  uint64_t* va_free = va_full + 2;
  uint64_t* w_full = va_free + 2;
  uint64_t* u_full = w_full + 2;
  uint64_t* u_free = u_full + 2;
  uint64_t* a_ready = u_free + 2;
  uint64_t* a_free = a_ready + 1;
  uint64_t* fin = a_free + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t G = gridDim.x;
  const int64_t lo = share_lo(a.T, blockIdx.x, G);
  const int64_t hi = share_lo(a.T, blockIdx.x + 1, G);
  const int nch = a.nch;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + NEPI);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&va_full[i], 1);
      mbar_init(&va_free[i], NEPI);
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

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_map(&maps.zc);
      tma_prefetch_map(&maps.zn);
      tma_prefetch_map(&maps.v1h);
      tma_prefetch_map(&maps.v2h);
      constexpr unsigned bytes = (unsigned)(2 * L::V1 + 2 * L::V2 + QC * ZW * 4 + NR * QC * NW * 4);
      int g = 0;
      for (int64_t u = lo; u < hi && !failed;) {
        const int64_t tile = u / nch;
        const int c0 = (int)(u - tile * nch);
        const int cend = (int)(min(hi - tile * nch, (int64_t)nch));
        const int64_t n0 = tile * TV;
        for (int c = c0; c < cend; ++c, ++g) {
          const int s = g % NS, k = g / NS;
          if (k > 0 && !mbar_wait(&empty[s], (k - 1) & 1)) {
            failed = true;
            break;
          }
          unsigned char* st = smem + s * L::stage;
          const int q0 = c * QC;
          mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
          for (int at = 0; at < RP / 32; ++at) {
            tma_load_2d(st + L::v1h + at * QC * 128, &maps.v1h, at * 32, q0, &full[s]);
            tma_load_2d(st + L::v1l + at * QC * 128, &maps.v1l, at * 32, q0, &full[s]);
          }
          tma_load_2d(st + L::v2h, &maps.v2h, q0, 0, &full[s]);
          tma_load_2d(st + L::v2l, &maps.v2l, q0, 0, &full[s]);
          tma_load_2d(st + L::zc, &maps.zc, (int)(n0 - 4), q0, &full[s]);
#pragma unroll
          for (int j = 0; j < NR; ++j)
            tma_load_2d(st + L::zn + j * QC * NW * 4, &maps.zn, (int)floor4(n0 + off[j]), q0,
                        &full[s]);
        }
        u = tile * nch + cend;
      }
      // no copy may still be in flight when the CTA exits: wait (bounded) for the last
      // phase issued into every stage
      for (int s = 0; s < NS && s < g; ++s) {
        const int last = s + ((g - 1 - s) / NS) * NS;
        mbar_wait(&full[s], (last / NS) & 1);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t a_hi = tmem + T_A, a_lo = tmem + T_A + RP;
      auto product2 = [&](int gg) {
        const int p = gg & 1, ph = gg >> 1;
        if (!failed && !mbar_wait(&w_full[p], ph & 1)) failed = true;
        if (!failed && gg >= 2 && !mbar_wait(&u_free[p], (ph - 1) & 1)) failed = true;
        if (failed) return;
        fence_after();
        const uint32_t st = smem_u32(smem + (gg % NS) * L::stage);
        const uint32_t d = tmem + L::T_U + RP * p;
        const uint32_t w_hi = tmem + T_W + 64 * p, w_lo = w_hi + 32;
#pragma unroll
        for (int k = 0; k < QC / 8; ++k) {
          const uint64_t bh = sdesc(st + L::v2h + k * 32), bl = sdesc(st + L::v2l + k * 32);
          mma_tf32(d, w_hi + 8 * k, bh, L::IDESC2, k > 0 ? 1u : 0u);
          mma_tf32(d, w_hi + 8 * k, bl, L::IDESC2, 1u);
          mma_tf32(d, w_lo + 8 * k, bh, L::IDESC2, 1u);
        }
        commit(&u_full[p]);
        commit(&empty[gg % NS]);
      };
      int g = 0, si = 0;
      for (int64_t u = lo; u < hi && !failed;) {
        const int64_t tile = u / nch;
        const int c0 = (int)(u - tile * nch);
        const int cend = (int)(min(hi - tile * nch, (int64_t)nch));
        const int nchk = cend - c0;
        if (!mbar_wait(a_ready, si & 1)) {
          failed = true;
          break;
        }
        fence_after();
        for (int i = 0; i < nchk && !failed; ++i) {
          const int gg = g + i, s = gg % NS, p = gg & 1, ph = gg >> 1;
          if (!mbar_wait(&full[s], (gg / NS) & 1)) failed = true;
          if (!failed && gg >= 2 && !mbar_wait(&va_free[p], (ph - 1) & 1)) failed = true;
          if (failed) break;
          fence_after();
          const uint32_t st = smem_u32(smem + s * L::stage);
          const uint32_t d = tmem + T_VA + 32 * p;
#pragma unroll
          for (int k = 0; k < RP / 8; ++k) {
            const int at = k / 4, o = (k % 4) * 32;
            const uint64_t bh = sdesc(st + L::v1h + at * QC * 128 + o);
            const uint64_t bl = sdesc(st + L::v1l + at * QC * 128 + o);
            mma_tf32(d, a_hi + 8 * k, bh, L::IDESC1, k > 0 ? 1u : 0u);
            mma_tf32(d, a_hi + 8 * k, bl, L::IDESC1, 1u);
            mma_tf32(d, a_lo + 8 * k, bh, L::IDESC1, 1u);
          }
          commit(&va_full[p]);
          if (i == nchk - 1) commit(a_free);     // a may be rewritten once these complete
          if (i > 0) product2(gg - 1);
        }
        if (!failed) product2(g + nchk - 1);
        g += nchk;
        ++si;
        u = tile * nch + cend;
      }
      // every product issued has completed before the TMEM is freed
      commit(fin);
      mbar_wait(fin, 0);
    }
  } else {
    // ------------------------------------------------------------------ epilogue warps
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int v = quarter * 32 + lane;               // voxel within the tile = TMEM lane
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int64_t ld = a.g.ld, N = a.g.N;
    const int Q = a.Q;
    const bool zl = nz > 1 && a.g.zlink;
    const float c2 = a.lam_s * a.inv_xb;             // weight of the neighbour sum
    const float c3 = a.beta * a.inv_xb;              // weight of V a
    int g = 0, si = 0;
    for (int64_t u = lo; u < hi;) {
      const int64_t tile = u / nch;
      const int c0 = (int)(u - tile * nch);
      const int cend = (int)(min(hi - tile * nch, (int64_t)nch));
      const int nchk = cend - c0;
      const int64_t n0 = tile * TV;
      const int64_t n = n0 + v;
      const bool valid = n < N;
      int x = 0, y = 0, zc = 0;
      if (valid) {
        x = (int)(n % nx);
        const int64_t t = n / nx;
        y = (int)(t % ny);
        zc = (int)(t / ny);
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
      int nidx[4];
      bool nok[4];
      {
        const bool flags[4] = {ny > 1 ? hym : hzm, ny > 1 ? hyp : hzp, hzm, hzp};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          nidx[j] = j < NR ? (int)(n + off[j] - floor4(n0 + off[j])) : 0;
          nok[j] = j < NR && flags[j];
        }
      }
      // a for this half's ranks: a_i = S_i/(beta + sigma_i^2) - W_i u_i, u_i summed over
      // the tile's segment slots of the previous iteration in segment order
      const int64_t j0 = owner_of(tile * nch, a.T, G);
      const int nseg = (int)(owner_of(tile * nch + nch - 1, a.T, G) - j0 + 1);
      const int sidx = (int)(blockIdx.x - j0);
      if (si > 0 && !failed && !mbar_wait(a_free, (si - 1) & 1)) failed = true;
      fence_after();
      {
        float ah[RH], al[RH];
        const float* pt = a.Pin + (tile * a.maxseg) * (int64_t)(RP * TV);
#pragma unroll
        for (int i = 0; i < RH; ++i) {
          const int r = half * RH + i;
          float av = 0.f;
          if (in) {
            float us = 0.f;
            for (int sg = 0; sg < nseg; ++sg) us += pt[(sg * RP + r) * TV + v];
            av = __ldg(a.S + r * ld + n) * __ldg(a.coefA + r) - __ldg(a.coefW + r) * us;
          }
          ah[i] = tf32_rna(av);
          al[i] = tf32_rna(av - ah[i]);
        }
#pragma unroll
        for (int i = 0; i < RH; i += 16) {
          tst16(tmem + lane_base + T_A + half * RH + i, ah + i);
          tst16(tmem + lane_base + T_A + RP + half * RH + i, al + i);
        }
        tst_wait();
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(a_ready);
      float uacc[RH];
#pragma unroll
      for (int i = 0; i < RH; ++i) uacc[i] = 0.f;
      auto consume_u = [&](int gg) {
        const int p = gg & 1;
        if (!failed && !mbar_wait(&u_full[p], (gg >> 1) & 1)) failed = true;
        fence_after();
#pragma unroll
        for (int i = 0; i < RH; i += 16) {
          float uu[16];
          tld16(tmem + lane_base + L::T_U + RP * p + half * RH + i, uu);
#pragma unroll
          for (int j = 0; j < 16; ++j) uacc[i + j] += uu[j];
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&u_free[p]);
      };
      for (int i = 0; i < nchk; ++i) {
        const int gg = g + i, s = gg % NS, p = gg & 1;
        const int qh = (c0 + i) * QC + half * HC;   // this warp's first compartment
        if (!failed && !mbar_wait(&full[s], (gg / NS) & 1)) failed = true;
        if (!failed && !mbar_wait(&va_full[p], (gg >> 1) & 1)) failed = true;
        fence_after();
        float va[HC];
        tld16(tmem + lane_base + T_VA + 32 * p + half * HC, va);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&va_free[p]);
        float dk[HC];
        if constexpr (CHECK) {
#pragma unroll
          for (int j = 0; j < HC; ++j)
            dk[j] = (in && qh + j < Q) ? __ldg(a.Din + (int64_t)(qh + j) * ld + n) : 0.f;
        }
        const unsigned char* st = smem + s * L::stage;
        const float* zcr = reinterpret_cast<const float*>(st + L::zc) + half * HC * ZW;
        const float* znr = reinterpret_cast<const float*>(st + L::zn) + half * HC * NW;
        float wh[HC], wl[HC];
#pragma unroll
        for (int j = 0; j < HC; ++j) {
          const int q = qh + j;
          float w = 0.f;
          if (!failed && in && q < Q) {
            const float z = zcr[j * ZW + 4 + v];
            float nb = 0.f;
            if (hxm) nb += zcr[j * ZW + 3 + v];
            if (hxp) nb += zcr[j * ZW + 5 + v];
#pragma unroll
            for (int k = 0; k < NR; ++k)
              if (nok[k]) nb += znr[(k * QC + j) * NW + nidx[k]];
            const float zn = fmaxf(0.f, fmaf(e1, z, fmaf(c2, nb, c3 * va[j])));
            const float t = z + va[j];
            w = a.beta * (2.f * zn - t);
            const int64_t o = (int64_t)q * ld + n;
            a.Zout[o] = zn;
            if (a.write_d) a.Dout[o] = a.beta * (t - zn);
            if constexpr (CHECK) {
              const float f = t - dk[j] * a.inv_beta;   // f^{k+1}
              const float e = zn - f, ch = zn - z;
              s1 = fmaf(e, e, s1);
              s2 = fmaf(ch, ch, s2);
              s3 = fmaf(zn, zn, s3);
            }
          }
          wh[j] = tf32_rna(w);
          wl[j] = tf32_rna(w - wh[j]);
        }
        tst16(tmem + lane_base + T_W + 64 * p + half * HC, wh);
        tst16(tmem + lane_base + T_W + 64 * p + 32 + half * HC, wl);
        tst_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&w_full[p]);
          mbar_arrive(&empty[s]);
        }
        if (i > 0) consume_u(gg - 1);
      }
      consume_u(g + nchk - 1);
      // this segment's partial u' (zero for voxels past the grid or outside the object)
      float* po = a.Pout + ((tile * a.maxseg + sidx) * (int64_t)RP) * TV;
#pragma unroll
      for (int i = 0; i < RH; ++i) po[(half * RH + i) * TV + v] = in ? uacc[i] : 0.f;
      g += nchk;
      ++si;
      u = tile * nch + cend;
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

template <int RP, int NR, bool CHECK>
ssm_status set_attr() {
  return cudaFuncSetAttribute(lrtc_kernel<RP, NR, CHECK>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Lay<RP, NR>::bytes) == cudaSuccess
             ? SSM_OK
             : SSM_ECUDA;
}

template <int RP, int NR>
ssm_status prepare_rn() {
  if constexpr (Lay<RP, NR>::valid) {
    SSM_TRY((set_attr<RP, NR, false>()));
    SSM_TRY((set_attr<RP, NR, true>()));
  }
  return SSM_OK;
}

template <int RP, int NR>
ssm_status launch_rn(const LrtcMaps& maps, const LrtcArgs& args, bool check, int64_t grid,
                     cudaStream_t s) {
  if constexpr (!Lay<RP, NR>::valid) {
    set_error("tensor-core low-rank form: this rank does not fit on 3D grids (r <= 32)");
    return SSM_EUNSUPPORTED;
  } else {
    const size_t shm = Lay<RP, NR>::bytes;
    if (check)
      lrtc_kernel<RP, NR, true><<<(unsigned)grid, NT, shm, s>>>(maps, args);
    else
      lrtc_kernel<RP, NR, false><<<(unsigned)grid, NT, shm, s>>>(maps, args);
    SSM_LAUNCHED();
    return SSM_OK;
  }
}

int grid_nr(const ssm_plan_s* pl) {
  return (pl->g.ny > 1 ? 2 : 0) + (pl->g.nz > 1 && pl->g.zlink ? 2 : 0);
}

}  // namespace

// padded rank of the tensor-core low-rank form: 32 or 64 (0: not supported)
int lrtc_padded_rank(int r, bool three_d) {
  if (r <= 32) return 32;
  if (r <= 64 && !three_d) return 64;
  return 0;
}

int64_t lrtc_chunks(const ssm_plan_s* pl) { return (pl->Q + QC - 1) / QC; }

int64_t lrtc_grid(const ssm_plan_s* pl) {
  const int64_t ntiles = (pl->g.N + TV - 1) / TV;
  const int64_t T = ntiles * lrtc_chunks(pl);
  int64_t grid = (int64_t)sm_count() * std::max(1, pl->waves);
  if (const char* env = getenv("SSM_LRTC_GRID")) {   // launch-shape override for sweeps
    const long v = atol(env);
    if (v >= 1 && v <= 65536) grid = v;
  }
  return std::max<int64_t>(1, std::min(grid, T));
}

int lrtc_maxseg(const ssm_plan_s* pl, int64_t grid) {
  const int64_t ntiles = (pl->g.N + TV - 1) / TV;
  return (int)((grid + ntiles - 1) / ntiles + 1);
}

int64_t lrtc_partial_floats(const ssm_plan_s* pl, int64_t grid) {
  const int64_t ntiles = (pl->g.N + TV - 1) / TV;
  return ntiles * lrtc_maxseg(pl, grid) * (int64_t)pl->R * TV;
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
  const int64_t grid = pl->lr_grid;
  LrtcArgs a;
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.Din = pl->Dl[cur];
  a.S = pl->S;
  a.Pin = pl->U[cur];
  a.Pout = pl->U[cur ^ 1];
  a.ntiles = (pl->g.N + TV - 1) / TV;
  a.nch = (int)lrtc_chunks(pl);
  a.T = a.ntiles * a.nch;
  a.maxseg = lrtc_maxseg(pl, grid);
  a.coefA = pl->coefA;
  a.coefW = pl->coefW;
  a.partial = partial;
  a.mask = pl->mask;
  a.err = pl->dev_err;
  a.g = pl->g;
  a.Q = pl->Q;
  a.write_d = write_d ? 1 : 0;
  a.beta = (float)pl->p.beta;
  a.inv_beta = (float)(1.0 / pl->p.beta);
  a.xi = (float)pl->xi;
  a.lam_s = (float)pl->lam_s;
  a.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  *nparts = (int)grid;
  const int nr = grid_nr(pl);
  if (pl->R == 32) {
    if (nr == 0) return launch_rn<32, 0>(m, a, check, grid, s);
    if (nr == 2) return launch_rn<32, 2>(m, a, check, grid, s);
    return launch_rn<32, 4>(m, a, check, grid, s);
  }
  if (pl->R == 64) {
    if (nr == 0) return launch_rn<64, 0>(m, a, check, grid, s);
    if (nr == 2) return launch_rn<64, 2>(m, a, check, grid, s);
    return launch_rn<64, 4>(m, a, check, grid, s);
  }
  set_error("tensor-core low-rank form: unsupported padded rank");
  return SSM_EUNSUPPORTED;
}

}  // namespace ssm
