// beta heuristic of Sec. III-E (ssm_tune_beta in include/ssm.h).
//
// The paper tunes beta once on a small patch of the image (3 x 3 voxels, 3 x 3 x 3 in
// 3D) for the fastest convergence and reuses it on the whole image. Here "fastest" is
// the lowest objective J(z^k) of Eq. 7 (with the dictionary the iteration uses) after a
// fixed budget of k iterations from the zero start; candidates are sigma_1^2 times a
// log-spaced grid. The spectral factors of K do not depend on beta, so one plan on the
// patch is made and each candidate only re-forms the beta-dependent weights
// (ssm_plan_set_beta) before its solve: one eigendecomposition for the whole search.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ssm_internal.cuh"

using namespace ssm;

extern "C" ssm_status ssm_tune_beta(const ssm_params* p, const double* K_host,
                                    const float* M_host, int64_t ldm, int iters, int n_grid,
                                    double grid_lo, double grid_hi, int device, void* stream,
                                    double* beta_out, double* betas, double* J) {
  if (!p || !K_host || !M_host || !beta_out) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  SSM_TRY(validate_params(p));
  if (iters < 1 || n_grid < 1 || n_grid > 4096 || !(grid_hi >= grid_lo) ||
      !std::isfinite(grid_lo) || !std::isfinite(grid_hi)) {
    set_error("need iters >= 1, 1 <= n_grid <= 4096 and grid_lo <= grid_hi");
    return SSM_EINVAL;
  }
  int64_t N = 1;
  for (int d = 0; d < p->ndim; ++d) N *= p->dims[d];
  if (ldm < N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  // the centre patch: up to 3 voxels per axis, starting at dims/2 - 1
  int64_t start[3] = {0, 0, 0}, size[3] = {1, 1, 1};
  for (int d = 0; d < p->ndim; ++d) {
    size[d] = std::min<int64_t>(3, p->dims[d]);
    start[d] = std::max<int64_t>(0, p->dims[d] / 2 - 1);
  }
  const int64_t np = size[0] * size[1] * size[2];
  std::vector<float> Mp((size_t)p->P * np);
  {
    int64_t c = 0;
    for (int64_t z = 0; z < size[2]; ++z)
      for (int64_t y = 0; y < size[1]; ++y)
        for (int64_t x = 0; x < size[0]; ++x, ++c) {
          const int64_t flat = (start[0] + x) + p->dims[0] * ((start[1] + y) +
                               (p->ndim >= 2 ? p->dims[1] : 1) * (start[2] + z));
          for (int r = 0; r < p->P; ++r) Mp[(size_t)r * np + c] = M_host[(size_t)r * ldm + flat];
        }
  }
  ssm_params pp = *p;
  for (int d = 0; d < p->ndim; ++d) pp.dims[d] = size[d];
  pp.form = SSM_FORM_LOWRANK;
  pp.precision = SSM_FP32;
  pp.beta = 1.0;
  pp.max_iter = iters;
  pp.check_every = 0;
  pp.tol_primal = pp.tol_change = 0.0;
  SSM_CUDA(cudaSetDevice(device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ssm_plan_t pl = nullptr;
  SSM_TRY(ssm_plan(&pl, &pp, K_host, device, stream));
  float *Md = nullptr, *Fd = nullptr;
  ssm_status st = SSM_OK;
  const cudaError_t e1 = cudaMallocAsync(&Md, sizeof(float) * p->P * np, s);
  const cudaError_t e2 = cudaMallocAsync(&Fd, sizeof(float) * p->Q * np, s);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    set_error("cudaMallocAsync failed");
    st = SSM_ENOMEM;
  }
  if (st == SSM_OK &&
      cudaMemcpyAsync(Md, Mp.data(), sizeof(float) * Mp.size(), cudaMemcpyHostToDevice, s) !=
          cudaSuccess) {
    set_error("cudaMemcpyAsync failed");
    st = SSM_ECUDA;
  }
  const double s1sq = pl->sigma1 * pl->sigma1;
  double best_b = 0.0, best_J = INFINITY;
  for (int k = 0; k < n_grid && st == SSM_OK; ++k) {
    const double ex = n_grid == 1 ? grid_lo : grid_lo + (grid_hi - grid_lo) * k / (n_grid - 1);
    const double b = s1sq * std::pow(10.0, ex);
    double Jk = 0.0;
    st = ssm_plan_set_beta(pl, b, stream);
    if (st == SSM_OK) st = ssm_solve(pl, Md, np, Fd, np, nullptr, stream);
    if (st == SSM_OK) st = ssm_objective(pl, Md, np, Fd, np, 0, &Jk, stream);
    if (st != SSM_OK) break;
    if (betas) betas[k] = b;
    if (J) J[k] = Jk;
    // lowest J; among equal J the smaller beta
    if (Jk < best_J || (Jk == best_J && b < best_b)) {
      best_J = Jk;
      best_b = b;
    }
  }
  if (Md) cudaFreeAsync(Md, s);
  if (Fd) cudaFreeAsync(Fd, s);
  cudaStreamSynchronize(s);
  ssm_destroy(pl);
  if (st != SSM_OK) return st;
  *beta_out = best_b;
  return SSM_OK;
}
