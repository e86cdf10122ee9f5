// C ABI of the solver (include/ssm.h): parameter checks, the plan (Algorithm 2,
// steps 1-3), the solve loop (steps 4-12 with the stopping rule) and the objective.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include <cudaTypedefs.h>

#include "ssm_internal.cuh"
#include "ssm_tma.cuh"

namespace ssm {

std::atomic<int64_t> g_launches{0};
thread_local int64_t t_launches = 0;
static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    int a = 0;
    if (cudaDeviceGetAttribute(&a, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || a <= 0)
      a = 148;
    v = a;
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

std::mutex& attr_mutex() {
  static std::mutex m;
  return m;
}

cudaError_t encode_2d(CUtensorMap* map, CUtensorMapDataType dtype, size_t elem, const void* base,
                      uint64_t cols, uint64_t rows, uint64_t ld, unsigned box_cols,
                      unsigned box_rows, CUtensorMapSwizzle swizzle) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * elem};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

namespace {

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// ||D^T D|| for the free-boundary box grid: D^T D = s L and the grid Laplacian's
// largest eigenvalue is sum over axes of 2 - 2 cos(pi (n_d - 1)/n_d) (path graphs).
double dtd_norm_closed(const int64_t* dims, int ndim, int pairs) {
  const double s = pairs == 2 ? 2.0 : 1.0;
  double t = 0.0;
  for (int d = 0; d < ndim; ++d)
    if (dims[d] >= 2) t += 2.0 - 2.0 * std::cos(M_PI * (double)(dims[d] - 1) / (double)dims[d]);
  return s * t;
}

// floats of one partial-u buffer of the low-rank forms
int64_t lowrank_state_floats(const ssm_plan_s* pl, int64_t grid) {
  if (pl->ndict > 0) return table_state_floats(pl->g.N, pl->mseg, pl->R);
  return pl->p.precision == SSM_TF32X3 ? lrtc_partial_floats(pl, grid)
                                       : lowrank_partial_floats(pl, grid);
}

int padded_rank(int r) {
  static const int opts[] = {4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64};
  for (int o : opts)
    if (r <= o) return o;
  return -1;
}

template <typename T>
ssm_status dalloc(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) return SSM_OK;
  SSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(T) * count, s));
  return SSM_OK;
}

// an allocation the plan owns: counted in pl->bytes
template <typename T>
ssm_status palloc(ssm_plan_s* pl, T** p, size_t count, cudaStream_t s) {
  SSM_TRY(dalloc(p, count, s));
  pl->bytes += (int64_t)(sizeof(T) * count);
  return SSM_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

ssm_status validate(const ssm_params* p) {
  if (!p) {
    set_error("params is NULL");
    return SSM_EINVAL;
  }
  if (p->ndim < 1 || p->ndim > 3) {
    set_error("ndim must be 1, 2 or 3");
    return SSM_EINVAL;
  }
  int64_t N = 1;
  for (int d = 0; d < p->ndim; ++d) {
    if (p->dims[d] < 1 || p->dims[d] > (int64_t)1 << 31) {
      set_error("grid dimensions must be >= 1");
      return SSM_EINVAL;
    }
    N *= p->dims[d];
  }
  if (N > ((int64_t)1 << 31) - 4096) {
    set_error("too many voxels (at most 2^31 - 4096: TMA coordinates are 32-bit)");
    return SSM_EINVAL;
  }
  if (p->P < 1 || p->Q < 1 || p->P > 65536 || p->Q > 65536) {
    set_error("P and Q must be in [1, 65536]");
    return SSM_EINVAL;
  }
  if (!(p->beta > 0.0) || !std::isfinite(p->beta)) {
    set_error("beta must be > 0");
    return SSM_EINVAL;
  }
  if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) {
    set_error("lambda must be >= 0");
    return SSM_EINVAL;
  }
  if (p->form != SSM_FORM_LOWRANK && p->form != SSM_FORM_DENSE && p->form != SSM_FORM_ADMM) {
    set_error("unknown form");
    return SSM_EINVAL;
  }
  if (p->precision != SSM_FP32 && p->precision != SSM_BF16X3 && p->precision != SSM_TF32X3) {
    set_error("unknown precision");
    return SSM_EINVAL;
  }
  if (p->stencil_pairs != 1 && p->stencil_pairs != 2) {
    set_error("stencil_pairs must be 1 or 2");
    return SSM_EINVAL;
  }
  if (p->max_iter < 0 || p->check_every < 0 || p->rank < 0) {
    set_error("max_iter, check_every and rank must be >= 0");
    return SSM_EINVAL;
  }
  return SSM_OK;
}

void release(ssm_plan_s* pl) {
  if (!pl) return;
  tc_release(pl);
  dfree(pl->K64);
  dfree(pl->Bp64);
  dfree(pl->Kt64);
  dfree(pl->sig64);
  dfree(pl->alpha64);
  dfree(pl->K32);
  dfree(pl->Kr32);
  dfree(pl->V32);
  dfree(pl->V1h);
  dfree(pl->V1l);
  dfree(pl->V2h);
  dfree(pl->V2l);
  dfree(pl->coefA);
  dfree(pl->coefW);
  dfree(pl->Mq32);
  dfree(pl->Mhi);
  dfree(pl->Mlo);
  dfree(pl->Gq32);
  for (int i = 0; i < 2; ++i) {
    dfree(pl->Z[i]);
    dfree(pl->Dl[i]);
    dfree(pl->U[i]);
    dfree(pl->Whi[i]);
    dfree(pl->Wlo[i]);
  }
  for (float** v : {&pl->adm.x, &pl->adm.y, &pl->adm.z, &pl->adm.dx, &pl->adm.dy, &pl->adm.dz,
                    &pl->adm.f, &pl->adm.w, &pl->adm.r, &pl->adm.t, &pl->adm_D})
    dfree(*v);
  for (auto& tt : pl->adm_T)
    for (float*& v : tt) dfree(v);
  dfree(pl->mask);
  dfree(pl->labels);
  dfree(pl->B_multi);
  dfree(pl->tprob);
  dfree(pl->ttable);
  dfree(pl->C32);
  dfree(pl->S);
  dfree(pl->H);
  dfree(pl->Wf);
  dfree(pl->Acc);
  dfree(pl->Res);
  dfree(pl->Mstage);
  dfree(pl->Fstage);
  dfree(pl->red);
  dfree(pl->red_out);
  dfree(pl->dev_err);
  if (pl->red_host) cudaFreeHost(pl->red_host);
  if (pl->ev0) cudaEventDestroy(pl->ev0);
  if (pl->ev1) cudaEventDestroy(pl->ev1);
  for (cudaEvent_t e : pl->prof_ev) cudaEventDestroy(e);
  for (GraphBlock& b : pl->graphs)
    if (b.exec) cudaGraphExecDestroy(b.exec);
  delete pl;
}

// grid, xi_p (Eq. 32) and the stencil weight of a plan from its parameters
void setup_grid(ssm_plan_s* pl) {
  const ssm_params& p = pl->p;
  pl->P = p.P;
  pl->Q = p.Q;
  pl->g.nx = (int)p.dims[0];
  pl->g.ny = p.ndim >= 2 ? (int)p.dims[1] : 1;
  pl->g.nz = p.ndim >= 3 ? (int)p.dims[2] : 1;
  pl->g.N = (int64_t)pl->g.nx * pl->g.ny * pl->g.nz;
  pl->g.ld = round_up(pl->g.N, 128);
  // a slice stack (z not linked) has the smoothness of one slice: the x and y axes only
  pl->dtd_norm = dtd_norm_closed(p.dims, pl->g.zlink ? p.ndim : 2, p.stencil_pairs);
  pl->xi = p.xi_p > 0.0 ? p.xi_p : 0.75 * p.lambda * pl->dtd_norm + 1e-10;  // Eq. 32
  pl->lam_s = p.lambda * (p.stencil_pairs == 2 ? 2.0 : 1.0);
}

ssm_status plan_impl(ssm_plan_s* pl, const double* K_host, cudaStream_t s) {
  const ssm_params& p = pl->p;
  SSM_CUDA(cudaEventCreate(&pl->ev0));
  SSM_CUDA(cudaEventCreate(&pl->ev1));
  SSM_CUDA(cudaEventRecord(pl->ev0, s));
  const int P = p.P, Q = p.Q;
  setup_grid(pl);
  pl->n = std::min(P, Q);
  pl->gram_side = P <= Q ? 0 : 1;
  const int n = pl->n;

  // dictionary and its Gram eigendecomposition (FP64)
  SSM_TRY(palloc(pl, &pl->K64, (size_t)P * Q, s));
  SSM_CUDA(cudaMemcpyAsync(pl->K64, K_host, sizeof(double) * P * Q, cudaMemcpyHostToDevice, s));
  double *A = nullptr, *E = nullptr, *scratch = nullptr;
  SSM_TRY(dalloc(&A, (size_t)n * n, s));
  SSM_TRY(dalloc(&E, (size_t)n * n, s));
  SSM_TRY(dalloc(&scratch, (size_t)n * n + 2, s));
  SSM_TRY(gram_fp64(pl->K64, P, Q, pl->gram_side, A, s));
  // lambda_max of the Hessian of Eq. 7 by FP64 power iteration (reads A before Jacobi
  // overwrites it)
  ssm_status st = hessian_power(pl, A, n, s);
  if (st != SSM_OK) {
    cudaFreeAsync(A, s);
    cudaFreeAsync(E, s);
    cudaFreeAsync(scratch, s);
    return st;
  }
  std::vector<double> evals;
  st = jacobi_eigen(A, n, E, scratch, evals, s);
  if (st != SSM_OK) {
    cudaFreeAsync(A, s);
    cudaFreeAsync(E, s);
    cudaFreeAsync(scratch, s);
    return st;
  }
  pl->perm.resize(n);
  std::iota(pl->perm.begin(), pl->perm.end(), 0);
  std::stable_sort(pl->perm.begin(), pl->perm.end(),
                   [&](int a, int b) { return evals[a] > evals[b]; });
  pl->sigma.resize(n);
  for (int i = 0; i < n; ++i) pl->sigma[i] = std::sqrt(std::max(0.0, evals[pl->perm[i]]));
  pl->sigma1 = pl->sigma[0];

  // rank (Sec. III-E): smallest r with ||K - K_r||_F < tol ||K||_F
  if (p.form == SSM_FORM_LOWRANK) {
    if (p.rank > 0) {
      pl->r = std::min(p.rank, n);
    } else {
      const double tol = p.rank_tol > 0 ? p.rank_tol : 5e-5;
      double total = 0.0;
      for (double v : pl->sigma) total += v * v;
      int r = n;
      for (int c = 0; c <= n; ++c) {
        double tail = 0.0;
        for (int i = c; i < n; ++i) tail += pl->sigma[i] * pl->sigma[i];
        if (total > 0 && std::sqrt(tail / total) < tol) {
          r = c;
          break;
        }
      }
      pl->r = std::max(r, 1);
    }
    pl->R = padded_rank(pl->r);
    if (pl->R < 0) {
      cudaFreeAsync(A, s);
      cudaFreeAsync(E, s);
      cudaFreeAsync(scratch, s);
      set_error("low-rank form supports r <= 64; use the dense form for higher ranks");
      return SSM_EUNSUPPORTED;
    }
    if (p.precision == SSM_TF32X3) {
      // the tensor-core form pads the rank to its MMA shapes (32 or 64; the padding
      // ranks carry zero weights, basis vectors and projections)
      pl->R = lrtc_padded_rank(pl->r, pl->g.nz > 1 && pl->g.zlink);
      if (pl->R == 0) {
        cudaFreeAsync(A, s);
        cudaFreeAsync(E, s);
        cudaFreeAsync(scratch, s);
        set_error("the TF32x3 low-rank form supports r <= 64 (r <= 32 on 3D grids)");
        return SSM_EUNSUPPORTED;
      }
    }
  } else {
    pl->r = n;
    pl->R = 0;
  }
  if (p.form == SSM_FORM_ADMM && p.precision != SSM_FP32) {
    cudaFreeAsync(A, s);
    cudaFreeAsync(E, s);
    cudaFreeAsync(scratch, s);
    set_error("the ADMM form runs in FP32 only");
    return SSM_EUNSUPPORTED;
  }
  if (p.form == SSM_FORM_DENSE && p.precision == SSM_TF32X3) {
    cudaFreeAsync(A, s);
    cudaFreeAsync(E, s);
    cudaFreeAsync(scratch, s);
    set_error("TF32x3 is a precision of the low-rank form (the dense form offers BF16x3)");
    return SSM_EUNSUPPORTED;
  }
  pl->Qp = (int)round_up(Q, 64);

  SSM_TRY(palloc(pl, &pl->Bp64, (size_t)P * n, s));
  SSM_TRY(palloc(pl, &pl->Kt64, (size_t)Q * n, s));
  SSM_TRY(palloc(pl, &pl->sig64, (size_t)n, s));
  SSM_TRY(palloc(pl, &pl->alpha64, (size_t)n, s));
  SSM_TRY(palloc(pl, &pl->K32, (size_t)P * Q, s));
  SSM_TRY(palloc(pl, &pl->Kr32, (size_t)P * Q, s));
  if (p.form == SSM_FORM_LOWRANK) {
    SSM_TRY(palloc(pl, &pl->V32, (size_t)Q * pl->R, s));
    SSM_TRY(palloc(pl, &pl->coefA, (size_t)pl->R, s));
    SSM_TRY(palloc(pl, &pl->coefW, (size_t)pl->R, s));
    if (p.precision == SSM_TF32X3) {
      pl->lrtc_qs = (int)round_up(Q, 32);
      SSM_TRY(palloc(pl, &pl->V1h, (size_t)Q * pl->R, s));
      SSM_TRY(palloc(pl, &pl->V1l, (size_t)Q * pl->R, s));
      SSM_TRY(palloc(pl, &pl->V2h, (size_t)pl->R * pl->lrtc_qs, s));
      SSM_TRY(palloc(pl, &pl->V2l, (size_t)pl->R * pl->lrtc_qs, s));
    }
  } else {
    SSM_TRY(palloc(pl, &pl->Gq32, (size_t)Q * n, s));
    SSM_TRY(palloc(pl, &pl->Mq32, (size_t)Q * pl->Qp, s));
    if (p.precision == SSM_BF16X3) {
      SSM_TRY(palloc(pl, &pl->Mhi, (size_t)Q * pl->Qp, s));
      SSM_TRY(palloc(pl, &pl->Mlo, (size_t)Q * pl->Qp, s));
    }
  }
  st = factors_fp64(pl, E, s);
  cudaFreeAsync(A, s);
  cudaFreeAsync(E, s);
  cudaFreeAsync(scratch, s);
  if (st != SSM_OK) return st;
  if (p.form != SSM_FORM_LOWRANK) SSM_TRY(form_dense_inverse(pl, s));

  // the device error word first: the tuning launches below report into it
  SSM_TRY(palloc(pl, &pl->dev_err, 1, s));
  SSM_CUDA(cudaMemsetAsync(pl->dev_err, 0, sizeof(int), s));

  // per-voxel state
  const size_t QN = (size_t)Q * pl->g.ld;
  if (p.form != SSM_FORM_ADMM)
    for (int i = 0; i < 2; ++i) {
      SSM_TRY(palloc(pl, &pl->Z[i], QN, s));
      SSM_TRY(palloc(pl, &pl->Dl[i], QN, s));
    }
  int maxparts = 1;
  if (p.form == SSM_FORM_ADMM) {
    AdmmState& a = pl->adm;
    for (float** v : {&a.x, &a.y, &a.z, &a.dx, &a.dy, &a.dz, &a.f, &a.w, &a.r, &a.t})
      SSM_TRY(palloc(pl, v, QN, s));
    SSM_TRY(palloc(pl, &pl->C32, (size_t)n * pl->g.ld, s));
    SSM_TRY(palloc(pl, &pl->H, QN, s));
    SSM_TRY(palloc(pl, &pl->Acc, QN, s));
    std::vector<std::pair<float**, std::vector<float>>> tables;
    SSM_TRY(admm_tables(pl, &tables));
    for (auto& t : tables) {
      SSM_TRY(palloc(pl, t.first, t.second.size(), s));
      SSM_CUDA(cudaMemcpyAsync(*t.first, t.second.data(), sizeof(float) * t.second.size(),
                               cudaMemcpyHostToDevice, s));
    }
    SSM_CUDA(cudaStreamSynchronize(s));   // the host tables are temporaries
    SSM_TRY(admm_prepare());
    maxparts = std::max(admm_partial_rows(pl), dense_max_partials(pl));
  } else if (p.form == SSM_FORM_LOWRANK) {
    SSM_TRY(palloc(pl, &pl->S, (size_t)pl->R * pl->g.ld, s));
    if (p.precision == SSM_TF32X3) {
      SSM_TRY(lrtc_prepare());
      pl->lr_grid = lrtc_grid(pl);
      maxparts = (int)pl->lr_grid;
    } else {
      pl->lr_grid = lowrank_grid(pl);
      maxparts = lowrank_max_partials(pl);
    }
    const size_t pf = (size_t)lowrank_state_floats(pl, pl->lr_grid);
    for (int i = 0; i < 2; ++i) SSM_TRY(palloc(pl, &pl->U[i], pf, s));
  } else {
    SSM_TRY(palloc(pl, &pl->C32, (size_t)n * pl->g.ld, s));
    SSM_TRY(palloc(pl, &pl->H, QN, s));
    if (p.precision == SSM_FP32) {
      SSM_TRY(palloc(pl, &pl->Wf, QN, s));
      SSM_TRY(palloc(pl, &pl->Acc, QN, s));
      maxparts = dense_max_partials(pl);
    } else {
      // w for the tensor-core operand: voxel-major rows of Qp compartments
      const size_t WN = (size_t)pl->g.ld * pl->Qp;
      SSM_TRY(palloc(pl, &pl->Acc, QN, s));
      for (int i = 0; i < 2; ++i) {
        SSM_TRY(palloc(pl, &pl->Whi[i], WN, s));
        SSM_TRY(palloc(pl, &pl->Wlo[i], WN, s));
      }
      SSM_TRY(tc_prepare(pl, s));
      maxparts = std::max(tc_max_partials(pl), dense_max_partials(pl));
    }
  }
  maxparts = std::max(maxparts, (int)((pl->g.N + 255) / 256));  // objective partials
  pl->red_cap = maxparts;
  SSM_TRY(palloc(pl, &pl->red, (size_t)maxparts * 4, s));
  SSM_TRY(palloc(pl, &pl->red_out, 8, s));
  SSM_CUDA(cudaMallocHost(&pl->red_host, 8 * sizeof(double)));
  SSM_CUDA(cudaEventRecord(pl->ev1, s));
  SSM_CUDA(cudaEventSynchronize(pl->ev1));
  SSM_CUDA(cudaEventElapsedTime(&pl->plan_ms, pl->ev0, pl->ev1));
  return SSM_OK;
}

// A plan with one dictionary per voxel label (ssm_plan_multi). Each dictionary is
// factorised by an ordinary plan on a one-voxel grid (FP64 Gram matrix, power
// iteration, Jacobi, the rank rule), one at a time; its basis V_r, weights and scaled
// left factors sigma_i u_i are copied out at the largest padded stride, then repacked
// to the common padded rank R.
ssm_status multi_plan_impl(ssm_plan_s* pl, int ndict, const double* K_host,
                           const int32_t* labels_host, cudaStream_t s) {
  const ssm_params& p = pl->p;
  SSM_CUDA(cudaEventCreate(&pl->ev0));
  SSM_CUDA(cudaEventCreate(&pl->ev1));
  SSM_CUDA(cudaEventRecord(pl->ev0, s));
  setup_grid(pl);
  const int P = p.P, Q = p.Q;
  const int RM = kMaxTableRank;
  pl->n = std::min(P, Q);
  pl->ndict = ndict;
  pl->ranks.assign(ndict, 0);
  // staging at stride RM: V [q][c][i], weights [c][i], sigma_i u_i [c][p][i]
  float *Vs = nullptr, *As = nullptr, *Ws = nullptr;
  double* Bs = nullptr;
  auto free_staging = [&]() {
    cudaFreeAsync(Vs, s);
    cudaFreeAsync(As, s);
    cudaFreeAsync(Ws, s);
    cudaFreeAsync(Bs, s);
  };
  SSM_TRY(dalloc(&Vs, (size_t)ndict * Q * RM, s));
  SSM_TRY(dalloc(&As, (size_t)ndict * RM, s));
  SSM_TRY(dalloc(&Ws, (size_t)ndict * RM, s));
  SSM_TRY(dalloc(&Bs, (size_t)ndict * P * RM, s));
  SSM_CUDA(cudaMemsetAsync(Vs, 0, sizeof(float) * ndict * Q * RM, s));
  ssm_params sp = p;
  sp.ndim = 1;
  sp.dims[0] = sp.dims[1] = sp.dims[2] = 1;
  sp.xi_p = 0.0;
  int rmax = 0;
  for (int c = 0; c < ndict; ++c) {
    ssm_plan_t sub = nullptr;
    ssm_status st = plan_create(&sub, &sp, K_host + (size_t)c * P * Q, pl->device, s, 1);
    if (st == SSM_OK && sub->r > RM) {
      set_error("spatially varying dictionaries: each dictionary's rank must be <= 32");
      st = SSM_EUNSUPPORTED;
    }
    if (st == SSM_OK) {
      const int r = sub->r;
      pl->ranks[c] = r;
      rmax = std::max(rmax, r);
      pl->sigma1 = std::max(pl->sigma1, sub->sigma1);
      pl->kk_power = std::max(pl->kk_power, sub->kk_power);
      pl->power_iters = std::max(pl->power_iters, sub->power_iters);
      pl->power_conv = c == 0 ? sub->power_conv : std::min(pl->power_conv, sub->power_conv);
      // V at [q][c][i]: row q of dictionary c at (q ndict + c) RM
      cudaError_t e = cudaMemcpy2DAsync(Vs + (size_t)c * RM, sizeof(float) * RM * ndict,
                                        sub->V32, sizeof(float) * sub->R, sizeof(float) * r, Q,
                                        cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(As + (size_t)c * RM, 0, sizeof(float) * RM, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(Ws + (size_t)c * RM, 0, sizeof(float) * RM, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(As + (size_t)c * RM, sub->coefA, sizeof(float) * r,
                            cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(Ws + (size_t)c * RM, sub->coefW, sizeof(float) * r,
                            cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) {
        set_error(std::string("copying a dictionary's factors: ") + cudaGetErrorString(e));
        st = SSM_ECUDA;
      }
      if (st == SSM_OK)
        st = table_gather_factors(sub->Bp64, sub->alpha64, P, sub->n, r, RM,
                                  Bs + (size_t)c * P * RM, s);
      // the copies read the sub-plan's buffers: finish them before it is freed
      if (cudaStreamSynchronize(s) != cudaSuccess && st == SSM_OK) st = SSM_ECUDA;
    }
    if (sub) release(sub);
    if (st != SSM_OK) {
      free_staging();
      return st;
    }
  }
  pl->r = rmax;
  pl->R = table_padded_rank(rmax);
  // the common padded rank: repack the staged factors at stride R
  ssm_status st = SSM_OK;
  auto repack = [&]() -> ssm_status {
    const int R = pl->R;
    SSM_TRY(palloc(pl, &pl->V32, (size_t)ndict * Q * R, s));
    SSM_TRY(palloc(pl, &pl->coefA, (size_t)ndict * R, s));
    SSM_TRY(palloc(pl, &pl->coefW, (size_t)ndict * R, s));
    SSM_TRY(palloc(pl, &pl->B_multi, (size_t)ndict * P * R, s));
    SSM_CUDA(cudaMemcpy2DAsync(pl->V32, sizeof(float) * R, Vs, sizeof(float) * RM,
                               sizeof(float) * R, (size_t)ndict * Q, cudaMemcpyDeviceToDevice, s));
    SSM_CUDA(cudaMemcpy2DAsync(pl->coefA, sizeof(float) * R, As, sizeof(float) * RM,
                               sizeof(float) * R, ndict, cudaMemcpyDeviceToDevice, s));
    SSM_CUDA(cudaMemcpy2DAsync(pl->coefW, sizeof(float) * R, Ws, sizeof(float) * RM,
                               sizeof(float) * R, ndict, cudaMemcpyDeviceToDevice, s));
    SSM_CUDA(cudaMemcpy2DAsync(pl->B_multi, sizeof(double) * R, Bs, sizeof(double) * RM,
                               sizeof(double) * R, (size_t)ndict * P, cudaMemcpyDeviceToDevice,
                               s));
    return SSM_OK;
  };
  st = repack();
  free_staging();
  if (st != SSM_OK) return st;

  SSM_TRY(palloc(pl, &pl->labels, (size_t)pl->g.N, s));
  SSM_CUDA(cudaMemcpyAsync(pl->labels, labels_host, sizeof(int32_t) * pl->g.N,
                           cudaMemcpyHostToDevice, s));
  SSM_TRY(palloc(pl, &pl->dev_err, 1, s));
  SSM_CUDA(cudaMemsetAsync(pl->dev_err, 0, sizeof(int), s));
  const size_t QN = (size_t)Q * pl->g.ld;
  for (int i = 0; i < 2; ++i) {
    SSM_TRY(palloc(pl, &pl->Z[i], QN, s));
    SSM_TRY(palloc(pl, &pl->Dl[i], QN, s));
  }
  SSM_TRY(palloc(pl, &pl->S, (size_t)pl->R * pl->g.ld, s));
  const int64_t ntiles = (pl->g.N + kTableTile - 1) / kTableTile;
  pl->mseg = table_segments(ntiles, Q, pl->R);
  const size_t pf = (size_t)table_state_floats(pl->g.N, pl->mseg, pl->R);
  for (int i = 0; i < 2; ++i) SSM_TRY(palloc(pl, &pl->U[i], pf, s));
  // the iteration's problem descriptor and (tile, segment) table
  std::vector<int4> entries;
  table_entries(0, ntiles, pl->mseg, &entries);
  pl->tblocks = (int64_t)entries.size();
  pl->lr_grid = pl->tblocks;
  TableProblem tp{};
  for (int i = 0; i < 2; ++i) {
    tp.Z[i] = pl->Z[i];
    tp.D[i] = pl->Dl[i];
    tp.U[i] = pl->U[i];
  }
  tp.S = pl->S;
  tp.V = pl->V32;
  tp.coefA = pl->coefA;
  tp.coefW = pl->coefW;
  tp.labels = pl->labels;
  tp.g = pl->g;
  tp.Q = Q;
  tp.nseg = pl->mseg;
  tp.ndict = ndict;
  tp.beta = (float)p.beta;
  tp.inv_beta = (float)(1.0 / p.beta);
  tp.xi = (float)pl->xi;
  tp.lam_s = (float)pl->lam_s;
  tp.inv_xb = (float)(1.0 / (pl->xi + p.beta));
  SSM_TRY(palloc(pl, &pl->tprob, 1, s));
  SSM_TRY(palloc(pl, &pl->ttable, entries.size(), s));
  SSM_CUDA(cudaMemcpyAsync(pl->tprob, &tp, sizeof(tp), cudaMemcpyHostToDevice, s));
  SSM_CUDA(cudaMemcpyAsync(pl->ttable, entries.data(), sizeof(int4) * entries.size(),
                           cudaMemcpyHostToDevice, s));
  SSM_CUDA(cudaStreamSynchronize(s));   // the host copies are temporaries
  const int maxparts = (int)std::max<int64_t>(pl->lr_grid, (pl->g.N + 255) / 256);
  pl->red_cap = maxparts;
  SSM_TRY(palloc(pl, &pl->red, (size_t)maxparts * 4, s));
  SSM_TRY(palloc(pl, &pl->red_out, 8, s));
  SSM_CUDA(cudaMallocHost(&pl->red_host, 8 * sizeof(double)));
  SSM_CUDA(cudaEventRecord(pl->ev1, s));
  SSM_CUDA(cudaEventSynchronize(pl->ev1));
  SSM_CUDA(cudaEventElapsedTime(&pl->plan_ms, pl->ev0, pl->ev1));
  return SSM_OK;
}

// Device bytes a plan for `p` takes, following plan_impl allocation by allocation:
// `persistent` = what the plan holds between calls (with the staging buffers of
// ssm_solve_host when `staging`), `peak` = persistent plus planning's temporaries
// (Gram matrix, eigenvectors, Jacobi scratch, K_r and the FP64 inverse). The low-rank
// rank is known only after the eigendecomposition: without a fixed rank the bound
// takes r = min(P, Q, 64), the largest the low-rank kernel supports.
ssm_status footprint_impl(const ssm_params& p, bool staging, int waves, int64_t* persistent,
                          int64_t* peak, bool zlink = true) {
  ssm_plan_s t;
  t.p = p;
  t.g.zlink = zlink ? 1 : 0;
  t.waves = std::max(1, waves);
  t.P = p.P;
  t.Q = p.Q;
  t.g.nx = (int)p.dims[0];
  t.g.ny = p.ndim >= 2 ? (int)p.dims[1] : 1;
  t.g.nz = p.ndim >= 3 ? (int)p.dims[2] : 1;
  t.g.N = (int64_t)t.g.nx * t.g.ny * t.g.nz;
  t.g.ld = round_up(t.g.N, 128);
  t.n = std::min(p.P, p.Q);
  const int64_t P = p.P, Q = p.Q, n = t.n, ld = t.g.ld;
  t.Qp = (int)round_up(Q, 64);
  if (p.form == SSM_FORM_LOWRANK) {
    t.r = p.rank > 0 ? std::min(p.rank, t.n) : std::min(t.n, kMaxRank);
    t.R = padded_rank(t.r);
    if (t.R < 0) {
      set_error("low-rank form supports r <= 64; use the dense form for higher ranks");
      return SSM_EUNSUPPORTED;
    }
    if (p.precision == SSM_TF32X3) {
      // without a fixed rank the bound takes the largest padding the grid allows
      const bool three_d = t.g.nz > 1 && zlink;
      t.R = lrtc_padded_rank(p.rank > 0 ? t.r : (three_d ? 32 : 64), three_d);
      if (t.R == 0) {
        set_error("the TF32x3 low-rank form supports r <= 64 (r <= 32 on 3D grids)");
        return SSM_EUNSUPPORTED;
      }
      t.lrtc_qs = (int)round_up(p.Q, 32);
    }
  }
  int64_t b = 0;
  auto add = [&](int64_t elem, int64_t count) { b += elem * count; };
  add(8, P * Q);                              // K64
  add(8, P * n);                              // Bp64
  add(8, Q * n);                              // Kt64
  add(8, n);                                  // sig64
  add(8, n);                                  // alpha64
  add(4, P * Q);                              // K32
  add(4, P * Q);                              // Kr32
  if (p.form == SSM_FORM_LOWRANK) {
    add(4, Q * t.R);                          // V32
    add(4, 2 * (int64_t)t.R);                 // coefA, coefW
    if (p.precision == SSM_TF32X3) add(4, 2 * (Q + t.lrtc_qs) * t.R);  // V1h/l, V2h/l
  } else {
    add(4, Q * n);                            // Gq32
    add(4, Q * t.Qp);                         // Mq32
    if (p.precision == SSM_BF16X3) add(2, 2 * Q * t.Qp);  // Mhi, Mlo
  }
  const int64_t QN = Q * ld;
  if (p.form != SSM_FORM_ADMM) add(4, 4 * QN);  // Z[2], Dl[2]
  int64_t maxparts = 1;
  if (p.form == SSM_FORM_ADMM) {
    add(4, 10 * QN);                          // x, y, z, d_x, d_y, d_z, f, w, r, t
    add(4, n * ld);                           // C32
    add(4, 2 * QN);                           // H, Acc
    const int64_t dd[3] = {t.g.nx, t.g.ny, t.g.nz};
    for (int d = 0; d < 3; ++d)
      if (dd[d] > 1 && (d < 2 || zlink))
        add(4, 2 * dd[d] * 64 * ((dd[d] + 63) / 64));  // DCT tables
    add(4, t.g.N);                            // spectral scaling
    maxparts = std::max<int64_t>(admm_partial_rows(&t), dense_max_partials(&t));
  } else if (p.form == SSM_FORM_LOWRANK) {
    add(4, (int64_t)t.R * ld);                // S
    if (p.precision == SSM_TF32X3) {
      t.lr_grid = lrtc_grid(&t);
      maxparts = t.lr_grid;
    } else {
      t.lr_grid = lowrank_grid(&t);
      maxparts = lowrank_max_partials(&t);
    }
    add(4, 2 * lowrank_state_floats(&t, t.lr_grid));  // U[2]
  } else {
    add(4, n * ld);                           // C32
    add(4, QN);                               // H
    if (p.precision == SSM_FP32) {
      add(4, 2 * QN);                         // Wf, Acc
      maxparts = dense_max_partials(&t);
    } else {
      add(4, QN);                             // Acc
      add(2, 4 * ld * t.Qp);                  // Whi[2], Wlo[2]
      maxparts = std::max(tc_max_partials(&t), dense_max_partials(&t));
    }
  }
  maxparts = std::max<int64_t>(maxparts, (t.g.N + 255) / 256);
  add(8, maxparts * 4);                       // red
  add(8, 8);                                  // red_out
  add(4, 1);                                  // dev_err
  if (staging) add(4, (P + Q) * ld);          // Mstage, Fstage
  *persistent = b;
  int64_t tmp = 8 * (3 * n * n + 2) + 4 * n + 8 * P * Q;  // A, E, scratch, perm, K_r
  if (p.form != SSM_FORM_LOWRANK) tmp += 8 * (n + Q * Q);   // inverse weights, FP64 inverse
  *peak = b + tmp;
  return SSM_OK;
}

// residual test: returns (rp, rc) from the three FP64 sums
// a kernel's bounded wait gave up: report it once and clear the word
ssm_status check_device_error(ssm_plan_s* pl, int host_err) {
  if (host_err != 0) {
    set_error("a device-side wait timed out (bounded mbarrier wait)");
    return (ssm_status)host_err;
  }
  return SSM_OK;
}

ssm_status read_residuals(ssm_plan_s* pl, int nparts, cudaStream_t s, double* rp, double* rc) {
  const bool admm = pl->p.form == SSM_FORM_ADMM;
  int nsum = 3;
  if (admm) {
    // rows [0, nparts): ||f-y||^2, ||dy||^2, ||y||^2; rows [nparts, 2 nparts): ||f-x||^2, ||f-z||^2
    SSM_TRY(finish_partials(pl->red, nparts, 3, pl->red_out, s));
    SSM_TRY(finish_partials(pl->red + (int64_t)nparts * 4, nparts, 2, pl->red_out + 3, s));
    nsum = 5;
  } else {
    SSM_TRY(finish_partials(pl->red, nparts, 3, pl->red_out, s));
  }
  SSM_CUDA(cudaMemcpyAsync(pl->red_host, pl->red_out, nsum * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  int* herr = reinterpret_cast<int*>(pl->red_host + 7);
  SSM_CUDA(cudaMemcpyAsync(herr, pl->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SSM_CUDA(cudaStreamSynchronize(s));
  if (*herr != 0) {
    const int e = *herr;
    *herr = 0;
    SSM_CUDA(cudaMemsetAsync(pl->dev_err, 0, sizeof(int), s));
    return check_device_error(pl, e);
  }
  const double* h = pl->red_host;
  for (int i = 0; i < nsum; ++i)
    if (!std::isfinite(h[i])) {
      set_error("residual is not finite");
      return SSM_ENAN;
    }
  if (admm) {
    const double yn = std::max(h[2], 1e-300);
    *rp = std::sqrt((h[0] + h[3] + h[4]) / yn);
    *rc = std::sqrt(h[1] / yn);
  } else {
    const double zn = std::max(h[2], 1e-300);
    *rp = std::sqrt(h[0] / zn);
    *rc = std::sqrt(h[1] / zn);
  }
  return SSM_OK;
}

// event pair around the dominant kernel of an iteration (profiling mode only)
ssm_status prof_mark(ssm_plan_s* pl, bool start, cudaStream_t s) {
  if (!pl->prof_enabled) return SSM_OK;
  const size_t idx = 2 * pl->prof_used + (start ? 0 : 1);
  while (pl->prof_ev.size() <= idx) {
    cudaEvent_t e;
    SSM_CUDA(cudaEventCreate(&e));
    pl->prof_ev.push_back(e);
  }
  SSM_CUDA(cudaEventRecord(pl->prof_ev[idx], s));
  if (!start) ++pl->prof_used;
  return SSM_OK;
}

ssm_status one_iteration(ssm_plan_s* pl, int cur, bool check, bool check_next, int* nparts,
                         cudaStream_t s) {
  const ssm_params& p = pl->p;
  if (p.form == SSM_FORM_ADMM) {
    // the event pair brackets the whole iteration (elementwise steps, the x-step
    // product, the z-step transforms)
    SSM_TRY(prof_mark(pl, true, s));
    SSM_TRY(admm_iteration(pl, check, pl->red, nparts, s));
    return prof_mark(pl, false, s);
  }
  SSM_TRY(prof_mark(pl, true, s));
  if (pl->ndict > 0) {
    SSM_TRY(table_iteration(pl->tprob, pl->ttable, pl->tblocks, pl->R, cur, check, check_next,
                            pl->red, s));
    *nparts = (int)pl->tblocks;
    return prof_mark(pl, false, s);
  }
  if (p.form == SSM_FORM_LOWRANK) {
    if (p.precision == SSM_TF32X3)
      SSM_TRY(lrtc_iteration(pl, cur, check, check_next, pl->red, nparts, s));
    else
      SSM_TRY(lowrank_iteration(pl, cur, check, check_next, pl->red, nparts, s));
    return prof_mark(pl, false, s);
  }
  if (p.precision == SSM_FP32) {
    // acc = M w (w^0 = 0, so the first product is 0)
    SSM_TRY(sgemm(pl->Q, (int)pl->g.N, pl->Q, 1.f, pl->Mq32, pl->Qp, pl->Wf, pl->g.ld, 0.f,
                  pl->Acc, pl->g.ld, s));
    SSM_TRY(prof_mark(pl, false, s));
    return dense_update(pl, cur, pl->Acc, check, true, false, pl->red, nparts, s);
  }
  if (pl->tc_fused) {
    // one kernel: the product M w with the element-wise steps in its epilogue
    SSM_TRY(tc_iteration(pl, cur, check, pl->red, nparts, s));
    return prof_mark(pl, false, s);
  }
  // two kernels; the dominant one is the product M w
  SSM_TRY(tc_gemm(pl, cur, s));
  SSM_TRY(prof_mark(pl, false, s));
  return tc_update(pl, cur, check, pl->red, nparts, s);
}

// iterations per block when no residual test ends it earlier
constexpr int kBlockMax = 64;

// a stream that can be captured: not the legacy default stream, not already capturing
bool capturable(cudaStream_t s) {
  if (s == nullptr || s == cudaStreamLegacy) return false;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st == cudaStreamCaptureStatusNone;
}

// iterations k .. k+L-1 as direct launches; *nparts = partial rows of the last test
template <typename IsCheck>
ssm_status run_block(ssm_plan_s* pl, int cur, int k, int L, const IsCheck& is_check, int* nparts,
                     cudaStream_t s) {
  for (int j = k; j < k + L; ++j) {
    int np = 0;
    SSM_TRY(one_iteration(pl, cur, is_check(j), is_check(j + 1), &np, s));
    if (is_check(j)) *nparts = np;
    cur ^= 1;
  }
  return SSM_OK;
}

// the same block replayed from a graph captured on its first use; the graph bakes in
// the plan's buffers and the block's pattern of residual tests, both fixed for a plan
template <typename IsCheck>
ssm_status run_block_graph(ssm_plan_s* pl, int cur, int k, int L, const IsCheck& is_check,
                           int* nparts, cudaStream_t s) {
  std::string key;
  key.reserve(2 * L + 8);
  key += (char)cur;
  key += std::to_string(L);
  key += ':';
  for (int j = k; j < k + L; ++j) key += (char)('0' + (is_check(j) ? 1 : 0) + (is_check(j + 1) ? 2 : 0));
  GraphBlock* blk = nullptr;
  for (GraphBlock& b : pl->graphs)
    if (b.key == key) blk = &b;
  if (!blk) {
    SSM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const int64_t t0 = t_launches;
    int np = 0;
    const ssm_status st = run_block(pl, cur, k, L, is_check, &np, s);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    const int64_t captured = t_launches - t0;
    g_launches.fetch_sub(captured, std::memory_order_relaxed);  // counted when replayed
    t_launches -= captured;
    if (st != SSM_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (st != SSM_OK) return st;
      SSM_CUDA(e);
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    SSM_CUDA(ei);
    GraphBlock b;
    b.key = key;
    b.exec = exec;
    b.kernels = captured;
    b.nparts = np;
    pl->graphs.push_back(std::move(b));
    blk = &pl->graphs.back();
  }
  SSM_CUDA(cudaGraphLaunch(blk->exec, s));
  g_launches.fetch_add(blk->kernels, std::memory_order_relaxed);
  t_launches += blk->kernels;
  *nparts = blk->nparts;
  return SSM_OK;
}

void fill_power_info(const ssm_plan_s* pl, ssm_info* info) {
  info->hess_norm = pl->hess_power;
  info->kk_norm = pl->kk_power;
  info->dtd_norm_power = pl->dtd_power;
  info->power_iters = pl->power_iters;
  info->power_converged = pl->power_conv;
}

// resume: continue from the state the plan's last solve left (z, d, the tensor-core
// operand w, the low-rank form's partial u) instead of the zero start
ssm_status solve_impl(ssm_plan_s* pl, const float* M, int64_t ldm, float* F, int64_t ldf,
                      ssm_info* info, cudaStream_t s, bool resume = false) {
  const ssm_params& p = pl->p;
  const int64_t ld = pl->g.ld;
  const size_t QN = (size_t)pl->Q * ld;
  if (resume && !pl->has_state) {
    set_error("nothing to resume: the plan has no iteration state (solve first)");
    return SSM_EINVAL;
  }
  pl->has_state = false;   // set again when this solve completes
  // step 4: projections of the data on the singular vectors (FP64 accumulation)
  if (pl->ndict > 0) {
    // each voxel's projections on its own dictionary's factors (zero past its rank)
    SSM_TRY(table_project(pl->B_multi, pl->P, pl->R, pl->labels, M, ldm, pl->g.N, pl->S,
                          pl->g.ld, s));
    if (!resume)
      SSM_CUDA(cudaMemsetAsync(
          pl->U[0], 0, sizeof(float) * (size_t)lowrank_state_floats(pl, pl->lr_grid), s));
  } else if (p.form == SSM_FORM_LOWRANK) {
    SSM_TRY(project_data(pl, M, ldm, pl->r, s));
    if (pl->R > pl->r)
      SSM_CUDA(cudaMemsetAsync(pl->S + (size_t)pl->r * ld, 0,
                               sizeof(float) * (size_t)(pl->R - pl->r) * ld, s));
    if (!resume)
      SSM_CUDA(cudaMemsetAsync(
          pl->U[0], 0, sizeof(float) * (size_t)lowrank_state_floats(pl, pl->lr_grid), s));
  } else {
    SSM_TRY(project_data(pl, M, ldm, pl->n, s));
    // h = M g = sum_i Gq_i c_i
    SSM_TRY(sgemm(pl->Q, (int)pl->g.N, pl->n, 1.f, pl->Gq32, pl->n, pl->C32, ld, 0.f, pl->H, ld,
                  s));
    if (pl->Wf && !resume) SSM_CUDA(cudaMemsetAsync(pl->Wf, 0, sizeof(float) * QN, s));
    if (pl->Whi[0] && !resume) {
      const size_t WN = (size_t)pl->g.ld * pl->Qp;
      SSM_CUDA(cudaMemsetAsync(pl->Whi[0], 0, sizeof(__nv_bfloat16) * WN, s));
      SSM_CUDA(cudaMemsetAsync(pl->Wlo[0], 0, sizeof(__nv_bfloat16) * WN, s));
    }
  }
  // step 2: z = d = 0 (Algorithm 1: x = y = z = d_x = d_y = d_z = 0)
  if (resume) {
    // the state stays as the last solve left it
  } else if (p.form == SSM_FORM_ADMM) {
    const AdmmState& a = pl->adm;
    for (float* v : {a.x, a.y, a.z, a.dx, a.dy, a.dz})
      SSM_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * QN, s));
  } else {
    // with a mask, voxels outside the object are never written: both ping-pong halves
    // (and both tensor-core operands) must hold zeros there
    const int nbuf = pl->mask ? 2 : 1;
    for (int i = 0; i < nbuf; ++i) {
      SSM_CUDA(cudaMemsetAsync(pl->Z[i], 0, sizeof(float) * QN, s));
      SSM_CUDA(cudaMemsetAsync(pl->Dl[i], 0, sizeof(float) * QN, s));
    }
    if (pl->mask && pl->Whi[1]) {
      const size_t WN = (size_t)pl->g.ld * pl->Qp;
      SSM_CUDA(cudaMemsetAsync(pl->Whi[1], 0, sizeof(__nv_bfloat16) * WN, s));
      SSM_CUDA(cudaMemsetAsync(pl->Wlo[1], 0, sizeof(__nv_bfloat16) * WN, s));
    }
  }

  const bool use_tol = p.tol_primal > 0 || p.tol_change > 0;
  int cur = resume ? pl->cur_state : 0, k = 0;
  double rp = -1, rc = -1;
  ssm_status result = SSM_OK;
  bool converged = false;
  // iteration j forms the residual sums when it ends on a test boundary or is the last;
  // "iteration max_iter" counts as a test, so the last iteration also stores d (the
  // low-rank forms keep d only around tests), which a resumed solve's first test reads
  auto is_check = [&](int j) {
    if (j >= p.max_iter) return j == p.max_iter;
    const bool at = p.check_every > 0 && ((j + 1) % p.check_every == 0);
    return (use_tol && at) || j + 1 == p.max_iter;
  };
  const bool graphs = pl->use_graphs && !pl->prof_enabled && capturable(s);
  // blocks of iterations end at each residual test (the host reads the sums there) or
  // after kBlockMax iterations; a block runs as direct launches or as one graph replay
  while (k < p.max_iter) {
    int L = 0;
    while (k + L < p.max_iter && L < kBlockMax) {
      ++L;
      if (is_check(k + L - 1)) break;
    }
    int nparts = 0;
    if (graphs)
      SSM_TRY(run_block_graph(pl, cur, k, L, is_check, &nparts, s));
    else
      SSM_TRY(run_block(pl, cur, k, L, is_check, &nparts, s));
    cur ^= (L & 1);
    k += L;
    if (is_check(k - 1)) {
      SSM_TRY(read_residuals(pl, nparts, s, &rp, &rc));
      const bool at_check = p.check_every > 0 && (k % p.check_every == 0);
      if (use_tol && at_check) {
        const bool ok_p = p.tol_primal <= 0 || rp <= p.tol_primal;
        const bool ok_c = p.tol_change <= 0 || rc <= p.tol_change;
        if (ok_p && ok_c) {
          converged = true;
          break;
        }
      }
    }
  }
  if (use_tol && !converged) result = SSM_ENOTCONVERGED;
  pl->cur_state = cur;
  pl->has_state = true;
  // F = z (the feasible iterate; y for Algorithm 1)
  const float* Fsrc = p.form == SSM_FORM_ADMM ? pl->adm.y : pl->Z[cur];
  SSM_CUDA(cudaMemcpy2DAsync(F, sizeof(float) * ldf, Fsrc, sizeof(float) * ld,
                             sizeof(float) * pl->g.N, pl->Q, cudaMemcpyDeviceToDevice, s));
  if (info) {
    SSM_CUDA(cudaStreamSynchronize(s));
    info->status = result;
    info->iterations = k;
    info->rank = pl->r;
    info->gram_side = pl->gram_side;
    info->xi_p = pl->xi;
    info->dtd_norm = pl->dtd_norm;
    info->sigma1 = pl->sigma1;
    info->res_primal = rp;
    info->res_change = rc;
    info->plan_ms = pl->plan_ms;
    fill_power_info(pl, info);
  }
  return result;
}

}  // namespace

ssm_status plan_footprint(const ssm_params& p, bool staging, int waves, int64_t* persistent,
                          int64_t* peak) {
  return footprint_impl(p, staging, waves, persistent, peak);
}

ssm_status validate_params(const ssm_params* p) { return validate(p); }

ssm_status plan_create(ssm_plan_t* out, const ssm_params* p, const double* K_host, int device,
                       cudaStream_t s, int waves, bool zlink) {
  if (!out) {
    set_error("out is NULL");
    return SSM_EINVAL;
  }
  *out = nullptr;
  SSM_TRY(validate(p));
  if (!K_host) {
    set_error("K_host is NULL");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(device));
  auto* pl = new ssm_plan_s();
  pl->p = *p;
  pl->device = device;
  pl->waves = std::max(1, waves);
  pl->g.zlink = zlink ? 1 : 0;
  ssm_status st = plan_impl(pl, K_host, s);
  if (st != SSM_OK) {
    cudaStreamSynchronize(s);
    release(pl);
    return st;
  }
  *out = pl;
  return SSM_OK;
}

}  // namespace ssm

using namespace ssm;

extern "C" {

ssm_status ssm_default_params(ssm_params* p) {
  if (!p) return SSM_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->ndim = 2;
  p->dims[0] = p->dims[1] = p->dims[2] = 1;
  p->lambda = 0.0;
  p->beta = 1.0;
  p->xi_p = 0.0;
  p->form = SSM_FORM_LOWRANK;
  p->rank = 0;
  p->rank_tol = 5e-5;
  p->precision = SSM_FP32;
  p->stencil_pairs = 2;
  p->max_iter = 300;
  p->check_every = 10;
  return SSM_OK;
}

ssm_status ssm_plan(ssm_plan_t* out, const ssm_params* p, const double* K_host, int device,
                    void* stream) {
  return plan_create(out, p, K_host, device, static_cast<cudaStream_t>(stream), 1);
}

ssm_status ssm_plan_ex(ssm_plan_t* out, const ssm_params* p, const double* K_host, int device,
                       void* stream, int launch_waves) {
  if (launch_waves < 1 || launch_waves > 64) {
    set_error("launch_waves must be in [1, 64]");
    return SSM_EINVAL;
  }
  return plan_create(out, p, K_host, device, static_cast<cudaStream_t>(stream), launch_waves);
}

ssm_status ssm_plan_batched(ssm_plan_t* out, const ssm_params* p, int64_t nbatch,
                            const double* K_host, int device, void* stream, int launch_waves) {
  if (!out || !p) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  *out = nullptr;
  if (p->ndim < 1 || p->ndim > 2) {
    set_error("a batched plan stacks 1D or 2D slices (ndim 1 or 2)");
    return SSM_EINVAL;
  }
  if (nbatch < 1 || nbatch > (int64_t)1 << 31 || launch_waves < 1 || launch_waves > 64) {
    set_error("nbatch must be >= 1 and launch_waves in [1, 64]");
    return SSM_EINVAL;
  }
  ssm_params q = *p;
  if (q.ndim == 1) q.dims[1] = 1;
  q.ndim = 3;
  q.dims[2] = nbatch;
  return plan_create(out, &q, K_host, device, static_cast<cudaStream_t>(stream), launch_waves,
                     false);
}

ssm_status ssm_plan_multi(ssm_plan_t* out, const ssm_params* p, int ndict,
                          const double* K_host, const int32_t* labels_host, int device,
                          void* stream) {
  if (!out) {
    set_error("out is NULL");
    return SSM_EINVAL;
  }
  *out = nullptr;
  SSM_TRY(validate(p));
  if (!K_host || !labels_host) {
    set_error("K_host or labels_host is NULL");
    return SSM_EINVAL;
  }
  if (ndict < 1 || ndict > 65536) {
    set_error("ndict must be in [1, 65536]");
    return SSM_EINVAL;
  }
  if (p->form != SSM_FORM_LOWRANK || p->precision != SSM_FP32) {
    set_error("spatially varying dictionaries run the low-rank form in FP32");
    return SSM_EUNSUPPORTED;
  }
  int64_t N = 1;
  for (int d = 0; d < p->ndim; ++d) N *= p->dims[d];
  for (int64_t i = 0; i < N; ++i)
    if (labels_host[i] < 0 || labels_host[i] >= ndict) {
      set_error("label " + std::to_string(labels_host[i]) + " of voxel " + std::to_string(i) +
                " is outside [0, ndict)");
      return SSM_EINVAL;
    }
  SSM_CUDA(cudaSetDevice(device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* pl = new ssm_plan_s();
  pl->p = *p;
  pl->device = device;
  pl->waves = 1;
  pl->g.zlink = 1;
  ssm_status st = multi_plan_impl(pl, ndict, K_host, labels_host, s);
  if (st != SSM_OK) {
    cudaStreamSynchronize(s);
    release(pl);
    return st;
  }
  *out = pl;
  return SSM_OK;
}

ssm_status ssm_solve(ssm_plan_t plan, const float* M_dev, int64_t ldm, float* F_dev, int64_t ldf,
                     ssm_info* info, void* stream) {
  if (!plan || !M_dev || !F_dev) {
    set_error("NULL plan or buffer");
    return SSM_EINVAL;
  }
  if (ldm < plan->g.N || ldf < plan->g.N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  return solve_impl(plan, M_dev, ldm, F_dev, ldf, info, static_cast<cudaStream_t>(stream));
}

ssm_status ssm_solve_resume(ssm_plan_t plan, const float* M_dev, int64_t ldm, float* F_dev,
                            int64_t ldf, ssm_info* info, void* stream) {
  if (!plan || !M_dev || !F_dev) {
    set_error("NULL plan or buffer");
    return SSM_EINVAL;
  }
  if (ldm < plan->g.N || ldf < plan->g.N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  return solve_impl(plan, M_dev, ldm, F_dev, ldf, info, static_cast<cudaStream_t>(stream), true);
}

ssm_status ssm_solve_host(ssm_plan_t plan, const float* M_host, int64_t ldm, float* F_host,
                          int64_t ldf, ssm_info* info, void* stream) {
  if (!plan || !M_host || !F_host) {
    set_error("NULL plan or buffer");
    return SSM_EINVAL;
  }
  if (ldm < plan->g.N || ldf < plan->g.N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ld = plan->g.ld;
  if (!plan->Mstage) SSM_TRY(palloc(plan, &plan->Mstage, (size_t)plan->P * ld, s));
  if (!plan->Fstage) SSM_TRY(palloc(plan, &plan->Fstage, (size_t)plan->Q * ld, s));
  SSM_CUDA(cudaMemcpy2DAsync(plan->Mstage, sizeof(float) * ld, M_host, sizeof(float) * ldm,
                             sizeof(float) * plan->g.N, plan->P, cudaMemcpyHostToDevice, s));
  ssm_status st = solve_impl(plan, plan->Mstage, ld, plan->Fstage, ld, info, s);
  if (st != SSM_OK && st != SSM_ENOTCONVERGED) return st;
  SSM_CUDA(cudaMemcpy2DAsync(F_host, sizeof(float) * ldf, plan->Fstage, sizeof(float) * ld,
                             sizeof(float) * plan->g.N, plan->Q, cudaMemcpyDeviceToHost, s));
  SSM_CUDA(cudaStreamSynchronize(s));
  return st;
}

ssm_status ssm_objective(ssm_plan_t plan, const float* M_dev, int64_t ldm, const float* F_dev,
                         int64_t ldf, int use_full_k, double* J_host, void* stream) {
  if (!plan || !M_dev || !F_dev || !J_host) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  if (plan->ndict > 0) {
    set_error("the objective is not available for a plan with spatially varying dictionaries");
    return SSM_EUNSUPPORTED;
  }
  if (ldm < plan->g.N || ldf < plan->g.N) {
    set_error("leading dimension smaller than N");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ld = plan->g.ld;
  if (!plan->Res) SSM_TRY(palloc(plan, &plan->Res, (size_t)plan->P * ld, s));
  SSM_CUDA(cudaMemcpy2DAsync(plan->Res, sizeof(float) * ld, M_dev, sizeof(float) * ldm,
                             sizeof(float) * plan->g.N, plan->P, cudaMemcpyDeviceToDevice, s));
  const float* Kd = (use_full_k || plan->p.form != SSM_FORM_LOWRANK) ? plan->K32 : plan->Kr32;
  // Res = M - K' F
  SSM_TRY(sgemm(plan->P, (int)plan->g.N, plan->Q, -1.f, Kd, plan->Q, F_dev, ldf, 1.f, plan->Res,
                ld, s));
  int nparts = 0;
  SSM_TRY(objective_terms(plan, plan->Res, plan->P, F_dev, ldf, plan->red, &nparts, s));
  SSM_TRY(finish_partials(plan->red, nparts, 2, plan->red_out, s));
  SSM_CUDA(cudaMemcpyAsync(plan->red_host, plan->red_out, 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  SSM_CUDA(cudaStreamSynchronize(s));
  // 1/2 ||R||^2 + lambda * 1/2 ||D F||^2, with 1/2 ||D F||^2 = (s/2) sum_edges (F_n - F_m)^2
  const double sfac = plan->p.stencil_pairs == 2 ? 1.0 : 0.5;
  *J_host = 0.5 * plan->red_host[0] + plan->p.lambda * sfac * plan->red_host[1];
  return SSM_OK;
}

ssm_status ssm_plan_factors(ssm_plan_t plan, double* sigma_host, double* vr_host, int* rank_out) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  if (plan->ndict > 0) {
    set_error("ssm_plan_factors is not available for a plan with spatially varying dictionaries");
    return SSM_EUNSUPPORTED;
  }
  if (sigma_host) std::memcpy(sigma_host, plan->sigma.data(), sizeof(double) * plan->n);
  if (rank_out) *rank_out = plan->r;
  if (vr_host) {
    // V_r from Kt: K K^T side holds sigma_i v_i, K^T K side holds v_i
    SSM_CUDA(cudaSetDevice(plan->device));
    std::vector<double> kt((size_t)plan->Q * plan->n);
    SSM_CUDA(cudaMemcpy(kt.data(), plan->Kt64, sizeof(double) * kt.size(), cudaMemcpyDeviceToHost));
    for (int q = 0; q < plan->Q; ++q)
      for (int i = 0; i < plan->r; ++i) {
        double v = kt[(size_t)q * plan->n + i];
        if (plan->gram_side == 0) v = plan->sigma[i] > 0 ? v / plan->sigma[i] : 0.0;
        vr_host[(size_t)q * plan->r + i] = v;
      }
  }
  return SSM_OK;
}

ssm_status ssm_plan_info(ssm_plan_t plan, ssm_info* info) {
  if (!plan || !info) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  std::memset(info, 0, sizeof(*info));
  info->status = SSM_OK;
  info->rank = plan->r;
  info->gram_side = plan->gram_side;
  info->xi_p = plan->xi;
  info->dtd_norm = plan->dtd_norm;
  info->sigma1 = plan->sigma1;
  info->res_primal = -1.0;
  info->res_change = -1.0;
  info->plan_ms = plan->plan_ms;
  fill_power_info(plan, info);
  return SSM_OK;
}

ssm_status ssm_plan_set_graphs(ssm_plan_t plan, int enable) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  plan->use_graphs = enable != 0;
  return SSM_OK;
}

ssm_status ssm_plan_set_mask(ssm_plan_t plan, const uint8_t* mask_host, void* stream) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  if (plan->ndict > 0) {
    set_error("a mask is not available for a plan with spatially varying dictionaries");
    return SSM_EUNSUPPORTED;
  }
  if (plan->p.form == SSM_FORM_ADMM) {
    set_error("the ADMM form's z-step needs the whole box grid: masks are not supported");
    return SSM_EUNSUPPORTED;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  plan->has_state = false;   // another problem: nothing to resume
  // captured graphs hold the old mask pointer (or none) in their kernel arguments
  for (GraphBlock& b : plan->graphs)
    if (b.exec) cudaGraphExecDestroy(b.exec);
  plan->graphs.clear();
  if (!mask_host) {
    if (plan->mask) {
      SSM_CUDA(cudaStreamSynchronize(s));
      dfree(plan->mask);
      plan->bytes -= plan->g.N;
    }
    return SSM_OK;
  }
  if (!plan->mask) SSM_TRY(palloc(plan, &plan->mask, (size_t)plan->g.N, s));
  SSM_CUDA(cudaMemcpyAsync(plan->mask, mask_host, (size_t)plan->g.N, cudaMemcpyHostToDevice, s));
  SSM_CUDA(cudaStreamSynchronize(s));   // the caller may free its buffer on return
  return SSM_OK;
}

ssm_status ssm_plan_set_stopping(ssm_plan_t plan, int max_iter, int check_every,
                                 double tol_primal, double tol_change) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  if (max_iter < 0 || check_every < 0 || !(tol_primal == tol_primal) ||
      !(tol_change == tol_change)) {
    set_error("max_iter and check_every must be >= 0, tolerances not NaN");
    return SSM_EINVAL;
  }
  plan->p.max_iter = max_iter;
  plan->p.check_every = check_every;
  plan->p.tol_primal = tol_primal;
  plan->p.tol_change = tol_change;
  // captured iteration blocks stay valid: a block is keyed by its length, start parity
  // and test pattern, none of which a kernel argument depends on
  return SSM_OK;
}

ssm_status ssm_plan_set_beta(ssm_plan_t plan, double beta, void* stream) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  if (plan->ndict > 0) {
    set_error("changing beta is not available for a plan with spatially varying dictionaries");
    return SSM_EUNSUPPORTED;
  }
  if (!(beta > 0.0) || !std::isfinite(beta)) {
    set_error("beta must be > 0");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  plan->p.beta = beta;
  plan->has_state = false;   // another iteration: nothing to resume
  // captured graphs hold the old beta in their kernel arguments
  for (GraphBlock& b : plan->graphs)
    if (b.exec) cudaGraphExecDestroy(b.exec);
  plan->graphs.clear();
  SSM_TRY(beta_weights(plan, s));
  if (plan->p.form != SSM_FORM_LOWRANK) SSM_TRY(form_dense_inverse(plan, s));
  if (plan->p.form == SSM_FORM_ADMM) {
    // the z-step's spectral scaling 1 / (lambda s mu + beta) depends on beta
    std::vector<std::pair<float**, std::vector<float>>> tables;
    SSM_TRY(admm_tables(plan, &tables));
    for (auto& t : tables)
      if (t.first == &plan->adm_D)
        SSM_CUDA(cudaMemcpyAsync(plan->adm_D, t.second.data(), sizeof(float) * t.second.size(),
                                 cudaMemcpyHostToDevice, s));
    SSM_CUDA(cudaStreamSynchronize(s));   // the host tables are temporaries
  }
  return SSM_OK;
}

ssm_status ssm_plan_footprint(const ssm_params* p, int device, int64_t* persistent_bytes,
                              int64_t* peak_bytes) {
  SSM_TRY(validate(p));
  if (!persistent_bytes || !peak_bytes) {
    set_error("NULL output");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(device));
  return footprint_impl(*p, true, 1, persistent_bytes, peak_bytes);
}

ssm_status ssm_plan_launch_info(ssm_plan_t plan, ssm_launch_info* out) {
  if (!plan || !out) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  std::memset(out, 0, sizeof(*out));
  out->launch_waves = plan->waves;
  out->sm_count = sm_count();
  if (plan->p.form == SSM_FORM_LOWRANK) {
    out->lowrank_grid = (int)plan->lr_grid;
  } else if (plan->Whi[0]) {
    out->gemm_tile_n = tc_tile_width(plan);
    out->gemm_grid = tc_gemm_grid(plan);
    out->update_grid = tc_update_grid(plan);
    out->tc_fused = plan->tc_fused ? (plan->tc_fused_reg ? 2 : 1) : 0;
  }
  return SSM_OK;
}

ssm_status ssm_plan_device_bytes(ssm_plan_t plan, int64_t* bytes) {
  if (!plan || !bytes) {
    set_error("NULL argument");
    return SSM_EINVAL;
  }
  *bytes = plan->bytes;
  return SSM_OK;
}

ssm_status ssm_profile_enable(ssm_plan_t plan, int enable) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  plan->prof_enabled = enable != 0;
  return SSM_OK;
}

ssm_status ssm_profile_read(ssm_plan_t plan, double* main_kernel_ms, int64_t* launches) {
  if (!plan) {
    set_error("NULL plan");
    return SSM_EINVAL;
  }
  SSM_CUDA(cudaSetDevice(plan->device));
  double total = 0.0;
  for (size_t i = 0; i < plan->prof_used; ++i) {
    SSM_CUDA(cudaEventSynchronize(plan->prof_ev[2 * i + 1]));
    float ms = 0.f;
    SSM_CUDA(cudaEventElapsedTime(&ms, plan->prof_ev[2 * i], plan->prof_ev[2 * i + 1]));
    total += ms;
  }
  if (main_kernel_ms) *main_kernel_ms = total;
  if (launches) *launches = (int64_t)plan->prof_used;
  plan->prof_used = 0;
  return SSM_OK;
}

ssm_status ssm_destroy(ssm_plan_t plan) {
  if (!plan) return SSM_OK;
  cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  release(plan);
  return SSM_OK;
}

const char* ssm_status_string(int status) {
  switch (status) {
    case SSM_OK: return "ok";
    case SSM_EINVAL: return "invalid argument";
    case SSM_ENOMEM: return "out of device memory";
    case SSM_ECUDA: return "CUDA error";
    case SSM_ENAN: return "non-finite residual";
    case SSM_ETIMEOUT: return "device wait timed out";
    case SSM_EUNSUPPORTED: return "unsupported configuration";
    case SSM_ENOTCONVERGED: return "tolerance not reached within max_iter";
    case SSM_EPENDING: return "request not finished";
    default: return "unknown status";
  }
}

const char* ssm_last_error(void) { return t_last_error.c_str(); }

int64_t ssm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
