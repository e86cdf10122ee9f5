// Self-test of the bounded waits (ssm_selftest_wait_timeout in include/ssm.h).
//
// Every mbarrier wait in the solver's kernels gives up after a fixed number of polls and
// reports SSM_ETIMEOUT through a device error word instead of hanging the GPU. This
// entry point exercises that path on purpose and safely: one CTA initialises an
// mbarrier that expects one arrival, no thread ever arrives, and the waiting thread
// polls it with the caller's (small) limit through the same mbar_wait the solver uses,
// then records the timeout and returns. Nothing faults and nothing spins unbounded.
#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

namespace ssm {
namespace {

__global__ void wait_timeout_kernel(unsigned polls, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, polls)) atomicExch(err, (int)SSM_ETIMEOUT);
  __syncthreads();   // nobody leaves with the barrier pending in use
}

}  // namespace
}  // namespace ssm

using namespace ssm;

extern "C" ssm_status ssm_selftest_wait_timeout(unsigned polls, void* stream) {
  if (polls < 1 || polls > (1u << 20)) {
    set_error("polls must be in [1, 2^20]");
    return SSM_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  SSM_CUDA(cudaMallocAsync(&err, sizeof(int), s));
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32, 0, s>>>(polls, err);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(err, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  SSM_CUDA(e);
  if (h != 0) {
    set_error("a bounded device-side wait timed out (self-test: expected)");
    return (ssm_status)h;
  }
  return SSM_OK;
}
