// Groups of independent low-rank problems in one launch per iteration (ssm_group_*).
//
// Each problem is a plan (its own dictionary, grid, lambda, beta and stopping rule) and
// runs Algorithm 2's low-rank iteration exactly as ssm_solve does; the group runs them
// together through the work-table kernel of ssm_table.cu, whose table lists the active
// problems' (tile, segment) entries. A problem leaves the table after the residual test
// that stops it (or its last iteration); the others go on. The group owns what the table
// kernel reads at its own layout: S, V_r and the weights padded to the group's rank R,
// sigma_i u_i for the projections, the partial-u buffers; z and d stay in the plans.
//
// Per iteration: one table launch. Per residual test: one launch that sums each active
// problem's residual rows in row order, and one host read of 3 doubles per problem.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ssm_internal.cuh"

struct ssm_group_s {
  int device = 0;
  int R = 0;
  std::vector<ssm_plan_t> plans;
  std::vector<int64_t> ntiles;
  std::vector<int> nseg;
  std::vector<float*> S, V, cA, cW, U0, U1;
  std::vector<double*> B;
  ssm::TableProblem* probs = nullptr;   // nplans descriptors (device)
  int4* table = nullptr;                // entries of the active problems (device)
  int64_t table_cap = 0;
  int64_t* ranges = nullptr;            // per active problem: first row, rows (device)
  double* red = nullptr;                // residual partial rows (4 doubles per entry)
  double* sums = nullptr;               // 3 doubles per problem (device)
  std::vector<double> sums_host;        // their host copy
  cudaStream_t stream = nullptr;        // the stream of the last create/solve call
  int64_t bytes = 0;
};

namespace ssm {
namespace {

constexpr int FT = 256;   // threads of the residual finish kernel

// out[3 j + c] = sum over rows [first, first + rows) of red[4 row + c], c < 3, in a fixed
// order: thread t sums rows t, t + FT, ... in order, then a fixed tree
__global__ void __launch_bounds__(FT) group_finish_kernel(const double* __restrict__ red,
                                                          const int64_t* __restrict__ ranges,
                                                          double* __restrict__ out) {
  __shared__ double sh[3][FT];
  const int64_t first = ranges[2 * blockIdx.x], rows = ranges[2 * blockIdx.x + 1];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += FT) {
    const double* p = red + (first + r) * 4;
    a0 += p[0];
    a1 += p[1];
    a2 += p[2];
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int h = FT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[3 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

template <typename T>
ssm_status galloc(ssm_group_s* g, T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) return SSM_OK;
  SSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(T) * count, s));
  g->bytes += (int64_t)(sizeof(T) * count);
  return SSM_OK;
}

// frees stream-ordered on the stream the group last ran on, so that releasing a group
// waits for nothing else on the device (a device-wide synchronisation here would hold a
// serving worker behind every other worker's solve)
void group_release(ssm_group_s* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  cudaStream_t s = g->stream;
  for (auto* v : {&g->S, &g->V, &g->cA, &g->cW, &g->U0, &g->U1})
    for (float* p : *v)
      if (p) cudaFreeAsync(p, s);
  for (double* p : g->B)
    if (p) cudaFreeAsync(p, s);
  for (void* p : {(void*)g->probs, (void*)g->table, (void*)g->ranges, (void*)g->red,
                  (void*)g->sums})
    if (p) cudaFreeAsync(p, s);
  cudaStreamSynchronize(s);
  delete g;
}

ssm_status check_plan(const ssm_plan_s* pl, int device) {
  if (!pl) {
    set_error("a plan of the group is NULL");
    return SSM_EINVAL;
  }
  if (pl->device != device) {
    set_error("the plans of a group must share one device");
    return SSM_EINVAL;
  }
  if (pl->p.form != SSM_FORM_LOWRANK || pl->p.precision != SSM_FP32 || pl->ndict > 0 ||
      pl->mask) {
    set_error("a group takes low-rank FP32 plans with one dictionary and no mask");
    return SSM_EUNSUPPORTED;
  }
  if (table_padded_rank(pl->r) == 0) {
    set_error("a group takes plans of rank <= 32");
    return SSM_EUNSUPPORTED;
  }
  return SSM_OK;
}

ssm_status create_impl(ssm_group_s* g, cudaStream_t s) {
  const int np = (int)g->plans.size();
  int R = 4;
  for (ssm_plan_t pl : g->plans) R = std::max(R, table_padded_rank(pl->r));
  g->R = R;
  for (auto* v : {&g->S, &g->V, &g->cA, &g->cW, &g->U0, &g->U1}) v->assign(np, nullptr);
  g->B.assign(np, nullptr);
  g->ntiles.assign(np, 0);
  g->nseg.assign(np, 1);
  std::vector<TableProblem> tp(np);
  int64_t entries = 0;
  for (int i = 0; i < np; ++i) {
    ssm_plan_s* pl = g->plans[i];
    const int P = pl->P, Q = pl->Q, r = pl->r;
    const int64_t ld = pl->g.ld;
    g->ntiles[i] = (pl->g.N + kTableTile - 1) / kTableTile;
    // segments from the problem's own Q alone (at least 32 compartments per warp: the
    // group, not the segments, fills the device), so its launch shape and summation
    // order do not depend on the other problems
    g->nseg[i] = std::max(1, std::min(8, Q / 128));
    entries += g->ntiles[i] * g->nseg[i];
    SSM_TRY(galloc(g, &g->S[i], (size_t)R * ld, s));
    SSM_TRY(galloc(g, &g->V[i], (size_t)Q * R, s));
    SSM_TRY(galloc(g, &g->cA[i], (size_t)R, s));
    SSM_TRY(galloc(g, &g->cW[i], (size_t)R, s));
    SSM_TRY(galloc(g, &g->B[i], (size_t)P * R, s));
    const size_t uf = (size_t)table_state_floats(pl->g.N, g->nseg[i], R);
    SSM_TRY(galloc(g, &g->U0[i], uf, s));
    SSM_TRY(galloc(g, &g->U1[i], uf, s));
    // V_r, the weights and sigma_i u_i at stride R (zero past the rank)
    SSM_CUDA(cudaMemsetAsync(g->V[i], 0, sizeof(float) * Q * R, s));
    SSM_CUDA(cudaMemcpy2DAsync(g->V[i], sizeof(float) * R, pl->V32, sizeof(float) * pl->R,
                               sizeof(float) * r, Q, cudaMemcpyDeviceToDevice, s));
    SSM_CUDA(cudaMemsetAsync(g->cA[i], 0, sizeof(float) * R, s));
    SSM_CUDA(cudaMemsetAsync(g->cW[i], 0, sizeof(float) * R, s));
    SSM_CUDA(cudaMemcpyAsync(g->cA[i], pl->coefA, sizeof(float) * r, cudaMemcpyDeviceToDevice, s));
    SSM_CUDA(cudaMemcpyAsync(g->cW[i], pl->coefW, sizeof(float) * r, cudaMemcpyDeviceToDevice, s));
    SSM_TRY(table_gather_factors(pl->Bp64, pl->alpha64, P, pl->n, r, R, g->B[i], s));
    TableProblem& t = tp[i];
    t.Z[0] = pl->Z[0];
    t.Z[1] = pl->Z[1];
    t.D[0] = pl->Dl[0];
    t.D[1] = pl->Dl[1];
    t.U[0] = g->U0[i];
    t.U[1] = g->U1[i];
    t.S = g->S[i];
    t.V = g->V[i];
    t.coefA = g->cA[i];
    t.coefW = g->cW[i];
    t.labels = nullptr;
    t.g = pl->g;
    t.Q = Q;
    t.nseg = g->nseg[i];
    t.ndict = 1;
    t.beta = (float)pl->p.beta;
    t.inv_beta = (float)(1.0 / pl->p.beta);
    t.xi = (float)pl->xi;
    t.lam_s = (float)pl->lam_s;
    t.inv_xb = (float)(1.0 / (pl->xi + pl->p.beta));
  }
  if (entries > INT32_MAX) {
    set_error("group too large for one launch");
    return SSM_EUNSUPPORTED;
  }
  g->table_cap = entries;
  SSM_TRY(galloc(g, &g->probs, (size_t)np, s));
  SSM_TRY(galloc(g, &g->table, (size_t)entries, s));
  SSM_TRY(galloc(g, &g->ranges, (size_t)2 * np, s));
  SSM_TRY(galloc(g, &g->red, (size_t)entries * 4, s));
  SSM_TRY(galloc(g, &g->sums, (size_t)3 * np, s));
  g->sums_host.assign((size_t)3 * np, 0.0);
  SSM_CUDA(cudaMemcpyAsync(g->probs, tp.data(), sizeof(TableProblem) * np,
                           cudaMemcpyHostToDevice, s));
  SSM_CUDA(cudaStreamSynchronize(s));   // `tp` is a host temporary
  return SSM_OK;
}

struct ProbRun {
  bool active = false, use_tol = false;
  int iters = 0, cur = 0;
  double rp = -1, rc = -1;
  ssm_status status = SSM_OK;
};

// iteration j of a problem forms its residual sums (it ends on a test or is its last)
bool is_check(const ssm_params& p, int j) {
  if (j >= p.max_iter) return false;
  const bool use_tol = p.tol_primal > 0 || p.tol_change > 0;
  const bool at = p.check_every > 0 && ((j + 1) % p.check_every == 0);
  return (use_tol && at) || j + 1 == p.max_iter;
}

ssm_status solve_impl(ssm_group_s* g, const float* const* M, const int64_t* ldm,
                      float* const* F, const int64_t* ldf, ssm_info* infos, cudaStream_t s) {
  const int np = (int)g->plans.size();
  std::vector<ProbRun> run(np);
  for (int i = 0; i < np; ++i) {
    ssm_plan_s* pl = g->plans[i];
    const size_t QN = (size_t)pl->Q * pl->g.ld;
    pl->has_state = false;   // the group's partial u is not the plan's: nothing to resume
    // step 4: projections (FP64 accumulation); step 2: z = d = 0, u = 0
    SSM_TRY(table_project(g->B[i], pl->P, g->R, nullptr, M[i], ldm[i], pl->g.N, g->S[i],
                          pl->g.ld, s));
    SSM_CUDA(cudaMemsetAsync(pl->Z[0], 0, sizeof(float) * QN, s));
    SSM_CUDA(cudaMemsetAsync(pl->Dl[0], 0, sizeof(float) * QN, s));
    SSM_CUDA(cudaMemsetAsync(
        g->U0[i], 0, sizeof(float) * (size_t)table_state_floats(pl->g.N, g->nseg[i], g->R), s));
    run[i].active = pl->p.max_iter > 0;
    run[i].use_tol = pl->p.tol_primal > 0 || pl->p.tol_change > 0;
  }
  std::vector<int> act;           // active problems, in problem order
  std::vector<int4> entries;
  std::vector<int64_t> ranges;
  auto rebuild = [&]() -> ssm_status {
    act.clear();
    entries.clear();
    ranges.clear();
    for (int i = 0; i < np; ++i)
      if (run[i].active) {
        act.push_back(i);
        ranges.push_back((int64_t)entries.size());
        table_entries(i, g->ntiles[i], g->nseg[i], &entries);
        ranges.push_back((int64_t)entries.size() - ranges.back());
      }
    if (act.empty()) return SSM_OK;
    // pageable sources: the copies are staged before the calls return
    SSM_CUDA(cudaMemcpyAsync(g->table, entries.data(), sizeof(int4) * entries.size(),
                             cudaMemcpyHostToDevice, s));
    SSM_CUDA(cudaMemcpyAsync(g->ranges, ranges.data(), sizeof(int64_t) * ranges.size(),
                             cudaMemcpyHostToDevice, s));
    return SSM_OK;
  };
  SSM_TRY(rebuild());
  int k = 0, cur = 0;
  while (!act.empty()) {
    bool check = false, write_d = false;
    for (int i : act) {
      check = check || is_check(g->plans[i]->p, k);
      write_d = write_d || is_check(g->plans[i]->p, k + 1);
    }
    SSM_TRY(table_iteration(g->probs, g->table, (int64_t)entries.size(), g->R, cur, check,
                            write_d, g->red, s));
    cur ^= 1;
    ++k;
    if (!check) continue;
    group_finish_kernel<<<(unsigned)act.size(), FT, 0, s>>>(g->red, g->ranges, g->sums);
    SSM_LAUNCHED();
    SSM_CUDA(cudaMemcpyAsync(g->sums_host.data(), g->sums, sizeof(double) * 3 * act.size(),
                             cudaMemcpyDeviceToHost, s));
    SSM_CUDA(cudaStreamSynchronize(s));
    bool changed = false;
    for (size_t j = 0; j < act.size(); ++j) {
      const int i = act[j];
      const ssm_params& p = g->plans[i]->p;
      if (!is_check(p, k - 1)) continue;
      ProbRun& pr = run[i];
      const double* h = g->sums_host.data() + 3 * j;
      bool done = k == p.max_iter;
      if (!std::isfinite(h[0]) || !std::isfinite(h[1]) || !std::isfinite(h[2])) {
        pr.status = SSM_ENAN;
        done = true;
      } else {
        const double zn = std::max(h[2], 1e-300);
        pr.rp = std::sqrt(h[0] / zn);
        pr.rc = std::sqrt(h[1] / zn);
        const bool at = p.check_every > 0 && (k % p.check_every == 0);
        if (pr.use_tol && at) {
          const bool ok_p = p.tol_primal <= 0 || pr.rp <= p.tol_primal;
          const bool ok_c = p.tol_change <= 0 || pr.rc <= p.tol_change;
          if (ok_p && ok_c) done = true;
          else if (k == p.max_iter) pr.status = SSM_ENOTCONVERGED;
        } else if (pr.use_tol && k == p.max_iter) {
          pr.status = SSM_ENOTCONVERGED;
        }
      }
      if (done) {
        pr.active = false;
        pr.iters = k;
        pr.cur = cur;
        changed = true;
      }
    }
    if (changed) SSM_TRY(rebuild());
  }
  ssm_status result = SSM_OK;
  for (int i = 0; i < np; ++i) {
    ssm_plan_s* pl = g->plans[i];
    // F = z (a problem with max_iter = 0 returns the zero start)
    SSM_CUDA(cudaMemcpy2DAsync(F[i], sizeof(float) * ldf[i], pl->Z[run[i].cur],
                               sizeof(float) * pl->g.ld, sizeof(float) * pl->g.N, pl->Q,
                               cudaMemcpyDeviceToDevice, s));
    if (run[i].status != SSM_OK && run[i].status != SSM_ENOTCONVERGED && result == SSM_OK)
      result = run[i].status;
  }
  if (result == SSM_OK)
    for (int i = 0; i < np; ++i)
      if (run[i].status == SSM_ENOTCONVERGED) result = SSM_ENOTCONVERGED;
  if (infos) {
    SSM_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < np; ++i) {
      const ssm_plan_s* pl = g->plans[i];
      ssm_info& in = infos[i];
      std::memset(&in, 0, sizeof(in));
      in.status = run[i].status;
      in.iterations = run[i].iters;
      in.rank = pl->r;
      in.gram_side = pl->gram_side;
      in.xi_p = pl->xi;
      in.dtd_norm = pl->dtd_norm;
      in.sigma1 = pl->sigma1;
      in.res_primal = run[i].rp;
      in.res_change = run[i].rc;
      in.plan_ms = pl->plan_ms;
      in.hess_norm = pl->hess_power;
      in.kk_norm = pl->kk_power;
      in.dtd_norm_power = pl->dtd_power;
      in.power_iters = pl->power_iters;
      in.power_converged = pl->power_conv;
    }
  }
  return result;
}

}  // namespace
}  // namespace ssm

using namespace ssm;

extern "C" {

ssm_status ssm_group_create(ssm_group_t* out, int nplans, const ssm_plan_t* plans,
                            void* stream) {
  if (!out || !plans || nplans < 1) {
    set_error("NULL argument or nplans < 1");
    return SSM_EINVAL;
  }
  *out = nullptr;
  const int device = plans[0] ? plans[0]->device : 0;
  for (int i = 0; i < nplans; ++i) SSM_TRY(check_plan(plans[i], device));
  SSM_CUDA(cudaSetDevice(device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* g = new ssm_group_s();
  g->device = device;
  g->stream = s;
  g->plans.assign(plans, plans + nplans);
  const ssm_status st = create_impl(g, s);
  if (st != SSM_OK) {
    cudaStreamSynchronize(s);
    group_release(g);
    return st;
  }
  *out = g;
  return SSM_OK;
}

ssm_status ssm_group_solve(ssm_group_t group, const float* const* M_devs, const int64_t* ldms,
                           float* const* F_devs, const int64_t* ldfs, ssm_info* infos,
                           void* stream) {
  if (!group || !M_devs || !ldms || !F_devs || !ldfs) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  for (size_t i = 0; i < group->plans.size(); ++i) {
    if (!M_devs[i] || !F_devs[i]) {
      set_error("NULL buffer for problem " + std::to_string(i));
      return SSM_EINVAL;
    }
    if (ldms[i] < group->plans[i]->g.N || ldfs[i] < group->plans[i]->g.N) {
      set_error("leading dimension smaller than N for problem " + std::to_string(i));
      return SSM_EINVAL;
    }
  }
  SSM_CUDA(cudaSetDevice(group->device));
  group->stream = static_cast<cudaStream_t>(stream);
  return solve_impl(group, M_devs, ldms, F_devs, ldfs, infos, group->stream);
}

ssm_status ssm_group_device_bytes(ssm_group_t group, int64_t* bytes) {
  if (!group || !bytes) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  *bytes = group->bytes;
  return SSM_OK;
}

ssm_status ssm_group_destroy(ssm_group_t group) {
  group_release(group);
  return SSM_OK;
}

}  // extern "C"
