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
// none of whose terms is large against the result. Substituting this f into the
// z-step and the dual step, d cancels from both:
//     beta f + d = beta (z + V a),   d^{k+1} = beta (z^k + V a^k - z^{k+1}),
// so the iteration's state is z and the r-vector u per voxel; d is only
// materialised where the stopping test needs it. One pass over z does the whole
// iteration:
//     t     = z + V a                                                (rank-r product)
//     z'    = max(0, ((xi + beta - lambda s deg) z + lambda s sum_nbr z + beta (V a))
//                    / (xi + beta))                                  (Eq. 31)
//     d'    = beta (t - z')                                          (step 11)
//     u'    = V^T (beta z' - d') = V^T beta (2 z' - t)               (rank-r product)
// D^T D z = s (deg(n) z_n - sum_{m adjacent} z_m): the free-boundary grid Laplacian,
// s = 2 for the literal Eq. 8.
//
// Mapping (HBM-streaming, TMA-fed, persistent). The work units are (segment, voxel tile
// of 128) pairs, a segment being one of nseg equal compartment ranges; the units are
// dealt round-robin in segment-major order to a grid sized to the resident capacity, so
// the CTAs of one round stream the same compartments of consecutive tiles and each
// one's neighbour rows were just read by another (L2 hits); nseg is chosen by layout().
// One producer warp streams a unit's rows in stages of QC compartments with 2D TMA
// box loads -- z with its x halo, the -+nx (-+nx*ny) neighbour rows, d and the
// matching rows of V -- into a ring of shared-memory stages guarded by mbarriers.
// Four consumer warps own one voxel per lane: for every staged compartment they
// compute f (packed f32x2 FMAs over the rank index), the z-step and the dual step,
// store z' and d' (coalesced), and fold beta z' - d' into the voxel's u' accumulators
// kept in registers. At the end of a unit the partial u' goes to its (tile, segment)
// slot; the next iteration sums a tile's slots in segment order (fixed, hence
// deterministic) when it forms a. HBM traffic per state element and iteration:
// read z, write z' (8 B); d is read/written only around residual tests; the halo rows
// are L2 hits. Every mbarrier wait is
// bounded and reports SSM_ETIMEOUT through the plan's device error word.
#include <algorithm>
#include <cstdlib>

#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

namespace ssm {
namespace {

constexpr int TV = 128;            // voxels per tile (4 consumer warps x 32 lanes)
constexpr int NCW = 4;             // consumer warps
constexpr int NT = 32 * (NCW + 1); // + one producer warp
constexpr int QC = 8;              // compartments per stage
constexpr int NB = 3;              // stages in the ring
constexpr int ZW = TV + 8;         // staged z row: voxels n0-4 .. n0+TV+3
constexpr int NW = TV + 4;         // staged neighbour row: 4-aligned base .. +TV+4

struct LowrankMaps {
  CUtensorMap zc;   // z^k, box {ZW, QC}
  CUtensorMap zn;   // z^k, box {NW, QC}
  CUtensorMap d;    // d^k, box {TV, QC}
  CUtensorMap v;    // V (Q x R), box {R, QC}
};

struct LowrankArgs {
  float* __restrict__ Zout;
  float* __restrict__ Dout;         // d^{k+1}, written when write_d != 0
  const float* __restrict__ S;      // R x ld
  const float* __restrict__ Pin;    // partial u of the previous iteration [tile][seg][R][TV]
  float* __restrict__ Pout;         // partial u of this iteration
  int64_t ntiles;                   // voxel tiles
  int nseg;                         // compartment segments per tile (units = ntiles nseg)
  const float* __restrict__ coefA;  // R
  const float* __restrict__ coefW;  // R
  double* __restrict__ partial;     // 4 doubles per block (check iterations)
  const uint8_t* __restrict__ mask; // voxels inside the object (nullptr: every voxel)
  int* __restrict__ err;            // device error word (SSM_ETIMEOUT on a failed wait)
  Grid g;
  int Q;
  int write_d;
  float beta, inv_beta, xi, lam_s, inv_xb;
};

// shared-memory layout (bytes), every TMA destination 128-byte aligned
struct Layout {
  int zc, zn, dd, vv, stage;   // offsets inside one stage, stage size
  int bars, total;             // mbarriers after the stages, total bytes
  __host__ __device__ Layout(int R, int NR) {
    auto al = [](int b) { return (b + 127) / 128 * 128; };
    zc = 0;
    zn = al(zc + QC * ZW * 4);
    dd = al(zn + NR * QC * NW * 4);
    vv = al(dd + QC * TV * 4);
    stage = al(vv + QC * R * 4);
    bars = NB * stage;
    total = bars + 2 * NB * 8;
  }
};

__host__ __device__ __forceinline__ int64_t floor4(int64_t v) {
  return v >= 0 ? (v & ~(int64_t)3) : -(((-v) + 3) & ~(int64_t)3);
}


template <int R, bool CHECK>
__global__ void __launch_bounds__(NT) lowrank_iter_kernel(const __grid_constant__ LowrankMaps maps,
                                                          const LowrankArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: align the dynamic window explicitly
  // aligned by an offset from the shared array itself (not through an integer), so that
  // the compiler keeps the shared address space of every pointer derived from it
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int64_t ld = a.g.ld;
  const int64_t N = a.g.N;
  const int Q = a.Q;
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const bool zl = nz > 1 && a.g.zlink;   // z neighbours coupled
  const int NR = (ny > 1 ? 2 : 0) + (zl ? 2 : 0);
  const Layout L(R, NR);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* empty = full + NB;
  // neighbour row offsets in flat index: -nx, +nx, -nx*ny, +nx*ny (present axes only)
  // (the order matches the neighbour flags: y pair first when the grid has a y axis)
  const int64_t plane = (int64_t)nx * ny;
  const int64_t off[4] = {ny > 1 ? -(int64_t)nx : -plane, ny > 1 ? (int64_t)nx : plane, -plane,
                          plane};
  const int64_t G = gridDim.x;
  const int64_t nunits = a.ntiles * a.nseg;
  // unit u = (segment u / ntiles, tile u % ntiles), dealt round-robin: the CTAs of one
  // round hold the same compartments of consecutive tiles, so the neighbour rows each
  // stages were just streamed by another (L2 hits)
  auto unit_rows = [&](int64_t u, int64_t& tile, int& sg, int& q0, int& q1) {
    sg = (int)(u / a.ntiles);
    tile = u - (int64_t)sg * a.ntiles;
    q0 = (int)(((int64_t)Q * sg) / a.nseg);
    q1 = (int)(((int64_t)Q * (sg + 1)) / a.nseg);
  };
  // d^k is staged only on residual-test iterations (it enters f, not z' or u')
  const unsigned stage_bytes = (unsigned)(QC * ZW * 4 + NR * QC * NW * 4 +
                                          (CHECK ? QC * TV * 4 : 0) + QC * R * 4);

  if (tid == 0) {
    for (int b = 0; b < NB; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], NCW);
    }
    mbar_fence_init();
  }
  __syncthreads();
  bool failed = false;
  float s1 = 0.f, s2 = 0.f, s3 = 0.f;
  const float c2 = a.lam_s * a.inv_xb;     // weight of the neighbour sum
  const float c3 = a.beta * a.inv_xb;      // weight of V a

  if (warp == NCW) {
    // ------------------------------- producer warp: one elected lane issues TMA
    if (lane == 0) {
      tma_prefetch_map(&maps.zc);
      tma_prefetch_map(&maps.d);
      int c = 0;   // running stage counter over all units
      for (int64_t u = blockIdx.x; u < nunits && !failed; u += G) {
        int64_t tile;
        int sg, q0, qend;
        unit_rows(u, tile, sg, q0, qend);
        const int64_t n0 = tile * TV;
        for (int q = q0; q < qend; q += QC, ++c) {
          const int b = c % NB;
          const int k = c / NB;
          if (c >= NB && !mbar_wait(&empty[b], (k - 1) & 1)) {
            failed = true;
            break;
          }
          unsigned char* st = smem + b * L.stage;
          mbar_arrive_expect_tx(&full[b], stage_bytes);
          tma_load_2d(st + L.zc, &maps.zc, (int)(n0 - 4), q, &full[b]);
          for (int j = 0; j < NR; ++j)
            tma_load_2d(st + L.zn + j * QC * NW * 4, &maps.zn, (int)floor4(n0 + off[j]), q,
                        &full[b]);
          if (CHECK) tma_load_2d(st + L.dd, &maps.d, (int)n0, q, &full[b]);
          tma_load_2d(st + L.vv, &maps.v, 0, q, &full[b]);
        }
      }
    }
  } else {
    // ------------------------------- consumer warps: one voxel per lane
    const int v = warp * 32 + lane;
    int c = 0;
    for (int64_t u = blockIdx.x; u < nunits; u += G) {
      int64_t tile;
      int sidx, q0, qend;
      unit_rows(u, tile, sidx, q0, qend);
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
      // a voxel outside the object is left alone (its z stays 0) and is nobody's
      // neighbour: the grid graph is the one the mask induces
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
      // a_i = S_i/(beta + sigma_i^2) - W_i u_i, u_i summed over the tile's segment
      // slots of the previous iteration in segment order
      const int nseg = a.nseg;
      float2 av[R / 2];
      {
        // slot by slot, all R loads of a slot in flight together (each u_i still sums
        // the slots in segment order)
        float us[R];
#pragma unroll
        for (int i = 0; i < R; ++i) us[i] = 0.f;
        if (in) {
          const float* pt = a.Pin + (tile * nseg) * (int64_t)(R * TV) + v;
          for (int sg = 0; sg < nseg; ++sg) {
#pragma unroll
            for (int i = 0; i < R; ++i) us[i] += pt[(sg * R + i) * TV];
          }
        }
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
          float a0 = 0.f, a1 = 0.f;
          if (in) {
            a0 = __ldg(a.S + (2 * i) * ld + n) * __ldg(a.coefA + 2 * i) -
                 __ldg(a.coefW + 2 * i) * us[2 * i];
            a1 = __ldg(a.S + (2 * i + 1) * ld + n) * __ldg(a.coefA + 2 * i + 1) -
                 __ldg(a.coefW + 2 * i + 1) * us[2 * i + 1];
          }
          av[i] = make_float2(a0, a1);
        }
      }
      float2 uacc[R / 2];
#pragma unroll
      for (int i = 0; i < R / 2; ++i) uacc[i] = make_float2(0.f, 0.f);
      for (int qc0 = q0; qc0 < qend; qc0 += QC, ++c) {
        const int b = c % NB;
        const int k = c / NB;
        if (!failed && !mbar_wait(&full[b], k & 1)) failed = true;
        const unsigned char* st = smem + b * L.stage;
        const float* zcr = reinterpret_cast<const float*>(st + L.zc);
        const float* znr = reinterpret_cast<const float*>(st + L.zn);
        const float* ddr = reinterpret_cast<const float*>(st + L.dd);
        const float* vvr = reinterpret_cast<const float*>(st + L.vv);
        const int qn = min(QC, qend - qc0);
        if (!failed && in) {
#pragma unroll
          for (int row = 0; row < QC; ++row) {
            if (row >= qn) break;
            const float z = zcr[row * ZW + 4 + v];
            float nb = 0.f;
            if (hxm) nb += zcr[row * ZW + 3 + v];
            if (hxp) nb += zcr[row * ZW + 5 + v];
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (nok[j]) nb += znr[(j * QC + row) * NW + nidx[j]];
            const float4* v4 = reinterpret_cast<const float4*>(vvr + row * R);
            float2 p0 = make_float2(0.f, 0.f), p1 = make_float2(0.f, 0.f);
            float4 vr[R / 4];
#pragma unroll
            for (int i = 0; i < R / 4; ++i) {
              vr[i] = v4[i];
              p0 = __ffma2_rn(make_float2(vr[i].x, vr[i].y), av[2 * i], p0);
              p1 = __ffma2_rn(make_float2(vr[i].z, vr[i].w), av[2 * i + 1], p1);
            }
            const float va = (p0.x + p0.y) + (p1.x + p1.y);     // (V a)_q
            const float zn = fmaxf(0.f, fmaf(e1, z, fmaf(c2, nb, c3 * va)));
            const float t = z + va;
            const float w = a.beta * (2.f * zn - t);            // beta z' - d'
            const float2 ww = make_float2(w, w);
#pragma unroll
            for (int i = 0; i < R / 4; ++i) {
              uacc[2 * i] = __ffma2_rn(make_float2(vr[i].x, vr[i].y), ww, uacc[2 * i]);
              uacc[2 * i + 1] = __ffma2_rn(make_float2(vr[i].z, vr[i].w), ww, uacc[2 * i + 1]);
            }
            const int64_t o = (int64_t)(qc0 + row) * ld + n;
            a.Zout[o] = zn;
            if (a.write_d) a.Dout[o] = a.beta * (t - zn);
            if (CHECK) {
              const float f = t - ddr[row * TV + v] * a.inv_beta;   // f^{k+1}
              const float e = zn - f, ch = zn - z;
              s1 = fmaf(e, e, s1);
              s2 = fmaf(ch, ch, s2);
              s3 = fmaf(zn, zn, s3);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
      }
      // this segment's partial u' (zero for voxels past the grid)
      float* po = a.Pout + ((tile * nseg + sidx) * (int64_t)R) * TV;
#pragma unroll
      for (int i = 0; i < R / 2; ++i) {
        po[(2 * i) * TV + v] = in ? uacc[i].x : 0.f;
        po[(2 * i + 1) * TV + v] = in ? uacc[i].y : 0.f;
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
}


template <int R>
size_t smem_for(int nr) { return (size_t)Layout(R, nr).total + 128; }

template <int R>
ssm_status launch_r(const LowrankMaps& maps, const LowrankArgs& args, bool check, int64_t grid,
                    cudaStream_t s) {
  const size_t shm =
      smem_for<R>((args.g.ny > 1 ? 2 : 0) + (args.g.nz > 1 && args.g.zlink ? 2 : 0));
  if (check)
    lowrank_iter_kernel<R, true><<<(unsigned)grid, NT, shm, s>>>(maps, args);
  else
    lowrank_iter_kernel<R, false><<<(unsigned)grid, NT, shm, s>>>(maps, args);
  SSM_LAUNCHED();
  return SSM_OK;
}

// resident CTAs per SM for rank R (registers and shared memory), set up once per R
template <int R>
int blocks_per_sm(int nr) {
  static std::atomic<int> cached[5];
  int v = cached[nr].load(std::memory_order_acquire);
  if (v != 0) return v;
  std::lock_guard<std::mutex> lock(attr_mutex());
  v = cached[nr].load(std::memory_order_relaxed);
  if (v != 0) return v;
  // the attribute belongs to the kernel, not to the halo layout: allow the largest
  // layout's size (3D, 4 halo rows), which every grid's launch fits in
  const size_t shm = smem_for<R>(nr);
  const size_t shm_max = smem_for<R>(4);
  cudaFuncSetAttribute(lowrank_iter_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)shm_max);
  cudaFuncSetAttribute(lowrank_iter_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)shm_max);
  int b1 = 0, b2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, lowrank_iter_kernel<R, true>, NT, shm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, lowrank_iter_kernel<R, false>, NT, shm);
  v = std::max(1, std::min(b1, b2));
  cached[nr].store(v, std::memory_order_release);
  return v;
}

// tensor maps of the current ping-pong state (encoding is a ~1 us host computation)
ssm_status build_maps(const ssm_plan_s* pl, int cur, LowrankMaps* m) {
  const uint64_t N = (uint64_t)pl->g.N, Q = (uint64_t)pl->Q, ld = (uint64_t)pl->g.ld;
  SSM_CUDA(encode_2d(&m->zc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pl->Z[cur], N, Q, ld, ZW, QC));
  SSM_CUDA(encode_2d(&m->zn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pl->Z[cur], N, Q, ld, NW, QC));
  SSM_CUDA(encode_2d(&m->d, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pl->Dl[cur], N, Q, ld, TV, QC));
  SSM_CUDA(encode_2d(&m->v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pl->V32, (uint64_t)pl->R, Q,
                     (uint64_t)pl->R, (unsigned)pl->R, QC));
  return SSM_OK;
}


int bpsm_for(int R, int nr) {
  switch (R) {
#define SSM_R(RR) \
  case RR:        \
    return blocks_per_sm<RR>(nr);
    SSM_R(4) SSM_R(8) SSM_R(12) SSM_R(16) SSM_R(20) SSM_R(24) SSM_R(28) SSM_R(32)
    SSM_R(40) SSM_R(48) SSM_R(56) SSM_R(64)
#undef SSM_R
    default:
      return 1;
  }
}

}  // namespace

namespace {

// a unit's start (the a-vector from the segment slots, the partial u' at its end) costs
// about as much as this many compartment rows
constexpr int kUnitRows = 16;

// Launch layout: G CTAs (every resident slot, times the launch waves) and nseg segments
// per tile, the units (segment, tile) dealt round-robin. nseg minimises rounds x (rows
// per unit + a unit's start), rounds = ceil(ntiles nseg / G): on the 128x128 slice
// (128 tiles, 456 CTAs) 7 segments make 896 units, two rounds of 357 rows, against the
// 702 rows per CTA of an even split that cannot keep neighbouring tiles in step.
void layout(const ssm_plan_s* pl, int64_t* grid, int* nseg) {
  const int nr = (pl->g.ny > 1 ? 2 : 0) + (pl->g.nz > 1 && pl->g.zlink ? 2 : 0);
  const int64_t ntiles = (pl->g.N + TV - 1) / TV;
  const int Q = pl->Q;
  int64_t g0 = (int64_t)sm_count() * bpsm_for(pl->R, nr) * std::max(1, pl->waves);
  if (const char* env = getenv("SSM_LOWRANK_GRID")) {   // launch-shape override for sweeps
    const long v = atol(env);
    if (v >= 1 && v <= 65536) g0 = v;
  }
  const int smax = std::max(1, std::min(64, Q / (2 * QC)));   // at least two stages a unit
  int best = 1;
  int64_t cost = INT64_MAX;
  for (int sg = 1; sg <= smax; ++sg) {
    const int64_t rounds = (ntiles * sg + g0 - 1) / g0;
    const int64_t c = rounds * ((Q + sg - 1) / sg + kUnitRows);
    if (c < cost) {
      cost = c;
      best = sg;
    }
  }
  *nseg = best;
  *grid = std::max<int64_t>(1, std::min<int64_t>(g0, ntiles * best));
}

}  // namespace

int64_t lowrank_grid(const ssm_plan_s* pl) {
  int64_t grid;
  int nseg;
  layout(pl, &grid, &nseg);
  return grid;
}

int64_t lowrank_partial_floats(const ssm_plan_s* pl, int64_t grid) {
  (void)grid;
  int64_t g;
  int nseg;
  layout(pl, &g, &nseg);
  const int64_t ntiles = (pl->g.N + TV - 1) / TV;
  return ntiles * nseg * (int64_t)pl->R * TV;
}

int lowrank_max_partials(const ssm_plan_s* pl) { return (int)lowrank_grid(pl); }

ssm_status lowrank_iteration(ssm_plan_s* pl, int cur, bool check, bool write_d, double* partial,
                             int* nparts, cudaStream_t s) {
  LowrankMaps maps;
  SSM_TRY(build_maps(pl, cur, &maps));
  int64_t grid;
  int nseg;
  layout(pl, &grid, &nseg);
  if (grid != pl->lr_grid) {
    set_error("low-rank form: launch layout changed since planning");
    return SSM_ECUDA;
  }
  LowrankArgs a;
  a.Zout = pl->Z[cur ^ 1];
  a.Dout = pl->Dl[cur ^ 1];
  a.S = pl->S;
  a.Pin = pl->U[cur];
  a.Pout = pl->U[cur ^ 1];
  a.ntiles = (pl->g.N + TV - 1) / TV;
  a.nseg = nseg;
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
  switch (pl->R) {
#define SSM_R(RR) \
  case RR:        \
    return launch_r<RR>(maps, a, check, grid, s);
    SSM_R(4) SSM_R(8) SSM_R(12) SSM_R(16) SSM_R(20) SSM_R(24) SSM_R(28) SSM_R(32)
    SSM_R(40) SSM_R(48) SSM_R(56) SSM_R(64)
#undef SSM_R
    default:
      set_error("low-rank kernel: unsupported padded rank");
      return SSM_EUNSUPPORTED;
  }
}

}  // namespace ssm
