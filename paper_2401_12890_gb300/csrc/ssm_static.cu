// Objective evaluation that allocates no device memory (ssm_objective_noalloc).
//
// Some callers cannot allocate device memory at the point where they want the
// objective: real-time pipelines that forbid allocation once they are running,
// processes where another allocator has reserved the device memory, and code on a
// busy device where cudaMalloc/cudaFree would synchronise the device and stall other
// streams. For them this entry point evaluates Eq. 7 / Eq. 8 from the caller's own
// buffers; its only scratch (per-block partial sums) lives in a fixed, file-scope
// device array, so nothing is allocated or freed.
//
// Limits and sharing: the array holds the partial sums of at most kMaxBlocks blocks
// of kThreads voxels, i.e. N <= 4,194,304 voxels (256 KB per device that loads the
// library, held until the process exits). Every call on a device uses the same array
// and leaves its contents behind; each call overwrites every slot it reads, and calls
// whose work overlaps on the GPU (two streams at once) would race on it.
#include <mutex>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

constexpr int kThreads = 256;                    // voxels per block
constexpr int kMaxBlocks = 16384;                // => N <= 4,194,304
constexpr int kPTile = 32;                       // residual rows per pass
constexpr int kQTile = 64;                       // dictionary columns per smem tile

// [0, 2*kMaxBlocks): per-block (data term, roughness term); then the finished pair
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks + 2];

// per voxel: sum_p (m_p - (K f)_p)^2 and sum over forward neighbour pairs of the map
// differences squared; the dictionary is staged through shared memory in tiles
__global__ void __launch_bounds__(kThreads) objective_noalloc_kernel(
    const float* __restrict__ K, int P, int Q, const float* __restrict__ M, int64_t ldm,
    const float* __restrict__ F, int64_t ldf, Grid g, double* __restrict__ part) {
  __shared__ float ks[kPTile][kQTile];
  const int64_t n = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool valid = n < g.N;
  double r2 = 0.0, e2 = 0.0;
  for (int p0 = 0; p0 < P; p0 += kPTile) {
    float acc[kPTile];
#pragma unroll
    for (int j = 0; j < kPTile; ++j) acc[j] = 0.f;
    for (int q0 = 0; q0 < Q; q0 += kQTile) {
      __syncthreads();
      for (int t = threadIdx.x; t < kPTile * kQTile; t += kThreads) {
        const int pp = t / kQTile, qq = t % kQTile;
        ks[pp][qq] = (p0 + pp < P && q0 + qq < Q) ? K[(int64_t)(p0 + pp) * Q + q0 + qq] : 0.f;
      }
      __syncthreads();
      if (valid) {
        const int qn = min(kQTile, Q - q0);
        for (int qq = 0; qq < qn; ++qq) {
          const float fv = F[(int64_t)(q0 + qq) * ldf + n];
#pragma unroll
          for (int j = 0; j < kPTile; ++j) acc[j] = fmaf(ks[j][qq], fv, acc[j]);
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < kPTile; ++j)
        if (p0 + j < P) {
          const double r = (double)M[(int64_t)(p0 + j) * ldm + n] - (double)acc[j];
          r2 += r * r;
        }
    }
  }
  if (valid) {
    const int x = (int)(n % g.nx);
    const int64_t t = n / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    for (int q = 0; q < Q; ++q) {
      const float* row = F + (int64_t)q * ldf;
      const float v = row[n];
      float s = 0.f;
      if (x + 1 < g.nx) { const float d = v - row[n + 1]; s = fmaf(d, d, s); }
      if (y + 1 < g.ny) { const float d = v - row[n + sy]; s = fmaf(d, d, s); }
      if (z + 1 < g.nz) { const float d = v - row[n + sz]; s = fmaf(d, d, s); }
      e2 += s;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  }
  __shared__ double red[kThreads / 32][2];
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = r2;
    red[threadIdx.x >> 5][1] = e2;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    part[2 * blockIdx.x + threadIdx.x] = s;
  }
}

// fixed-order sum of the block partials into the last two slots
__global__ void objective_noalloc_finish(double* part, int nblocks) {
  __shared__ double sm[32][2];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sm[threadIdx.x >> 5][0] = a;
    sm[threadIdx.x >> 5][1] = b;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm[w][threadIdx.x];
    part[2 * kMaxBlocks + threadIdx.x] = s;
  }
}

// device address of the scratch array, looked up once per device with that device
// current (the array's name is only a host-side stand-in for it)
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[256] = {};

ssm_status noalloc_scratch(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (device < 0 || device >= 256) {
    set_error("device index out of range");
    return SSM_EINVAL;
  }
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return SSM_ECUDA;
    }
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return SSM_OK;
}

}  // namespace
}  // namespace ssm

using namespace ssm;

extern "C" ssm_status ssm_objective_noalloc(const float* K_dev, int P, int Q, const float* M_dev,
                                            int64_t ldm, const float* F_dev, int64_t ldf,
                                            int ndim, const int64_t* dims, double lambda,
                                            int stencil_pairs, double* J_host, void* stream) {
  if (!K_dev || !M_dev || !F_dev || !dims || !J_host) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  if (P < 1 || Q < 1 || ndim < 1 || ndim > 3 || !(lambda >= 0.0) ||
      (stencil_pairs != 1 && stencil_pairs != 2)) {
    set_error("invalid sizes or parameters");
    return SSM_EINVAL;
  }
  // the voxel count is checked on the 64-bit sizes, axis by axis, before any is
  // narrowed to int (a dimension of 2^32 + 5 must not pass as 5)
  const int64_t max_voxels = (int64_t)kThreads * kMaxBlocks;
  int64_t nvox = 1;
  for (int d = 0; d < ndim; ++d) {
    if (dims[d] < 1) {
      set_error("grid dimensions must be >= 1");
      return SSM_EINVAL;
    }
    if (dims[d] > max_voxels || nvox * dims[d] > max_voxels) {
      set_error("ssm_objective_noalloc: at most 4194304 voxels (fixed scratch of 16384 blocks)");
      return SSM_EINVAL;
    }
    nvox *= dims[d];
  }
  Grid g;
  g.nx = (int)dims[0];
  g.ny = ndim >= 2 ? (int)dims[1] : 1;
  g.nz = ndim >= 3 ? (int)dims[2] : 1;
  g.N = nvox;
  g.ld = g.N;
  if (ldm < g.N || ldf < g.N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  int device = 0;
  SSM_CUDA(cudaGetDevice(&device));
  double* part = nullptr;
  SSM_TRY(noalloc_scratch(device, &part));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblocks = (int)((g.N + kThreads - 1) / kThreads);
  objective_noalloc_kernel<<<nblocks, kThreads, 0, s>>>(K_dev, P, Q, M_dev, ldm, F_dev, ldf, g,
                                                        part);
  SSM_LAUNCHED();
  objective_noalloc_finish<<<1, 1024, 0, s>>>(part, nblocks);
  SSM_LAUNCHED();
  double sums[2];
  SSM_CUDA(cudaMemcpyAsync(sums, part + 2 * kMaxBlocks, sizeof(sums), cudaMemcpyDeviceToHost, s));
  SSM_CUDA(cudaStreamSynchronize(s));
  // 1/2 ||M - K F||^2 + lambda * 1/2 ||D F||^2, 1/2 ||D F||^2 = (s/2) sum_edges (F_n - F_m)^2
  *J_host = 0.5 * sums[0] + lambda * (stencil_pairs == 2 ? 1.0 : 0.5) * sums[1];
  return SSM_OK;
}
