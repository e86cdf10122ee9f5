// Internal declarations shared by the CUDA translation units of the solver library.
// Nothing here is part of the public ABI (include/ssm.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "ssm.h"

namespace ssm {

// ------------------------------------------------------------------------------------
// error handling: every CUDA call is checked; failures become a status + message
// ------------------------------------------------------------------------------------
void set_error(const std::string& msg);
extern std::atomic<int64_t> g_launches;
// kernels launched (or captured into a graph) by the calling thread
extern thread_local int64_t t_launches;

// SM count of the current device (queried once per device; safe from any thread)
int sm_count();
// serialises the one-time kernel attribute / occupancy set-up across host threads
std::mutex& attr_mutex();

#define SSM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ::ssm::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));              \
      return e_ == cudaErrorMemoryAllocation ? SSM_ENOMEM : SSM_ECUDA;                   \
    }                                                                                    \
  } while (0)

#define SSM_LAUNCHED()                                                                   \
  do {                                                                                   \
    ::ssm::g_launches.fetch_add(1, std::memory_order_relaxed);                           \
    ++::ssm::t_launches;                                                                 \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess) {                                                             \
      ::ssm::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));         \
      return SSM_ECUDA;                                                                  \
    }                                                                                    \
  } while (0)

#define SSM_TRY(expr)                                                                    \
  do {                                                                                   \
    ssm_status s_ = (expr);                                                              \
    if (s_ != SSM_OK) return s_;                                                         \
  } while (0)

// ------------------------------------------------------------------------------------
// grid description used by every stencil kernel (Eq. 8, free boundary)
// ------------------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;     // nz = 1 for 2D, ny = nz = 1 for 1D
  int64_t N;          // nx*ny*nz
  int64_t ld;         // leading dimension of every map-major Q x N array (elements)
  int zlink = 1;      // 0: the z axis stacks independent slices (no smoothness across it)
};

// One element of the full-rank iteration's z-step (Eq. 31, with D^T D z = s (deg z -
// sum_nbr z)) and dual step (step 11), given f = h + M w:
//     z' = max(0, (xi z - lambda s (deg z - nb) + beta f + d) / (xi + beta))
//     d' = d - beta (z' - f),   w' = beta z' - d'
// Every rounding is explicit (fmaf / __fmul_rn), so each kernel that applies the step
// produces the same bits whatever the compiler would otherwise contract.
struct DenseStep {
  float xi, lam_s, beta, inv_xb;   // inv_xb = 1 / (xi + beta)
  __device__ __forceinline__ float apply(float z, float d, float f, float deg, float nb, float& dn,
                                         float& w) const {
    const float lap = fmaf(deg, z, -nb);                                  // deg z - nb
    const float num = fmaf(xi, z, fmaf(-lam_s, lap, fmaf(beta, f, d)));
    const float zn = fmaxf(0.f, __fmul_rn(num, inv_xb));
    dn = fmaf(-beta, __fsub_rn(zn, f), d);
    w = fmaf(beta, zn, -dn);
    return zn;
  }
};

// the largest padded rank the fused low-rank kernel is instantiated for
constexpr int kMaxRank = 64;

// One problem of the work-table iteration (ssm_table.cu): the low-rank d-free recurrence
// on its own grid, with its own basis and state. The iteration kernel reads a table of
// (problem, voxel tile, compartment segment) entries, one per block, so one launch can
// run the iterations of several problems of differing N, P, Q.
struct TableProblem {
  float* Z[2];                      // z ping-pong (Q x ld)
  float* D[2];                      // d ping-pong (Q x ld; read/written around tests)
  float* U[2];                      // partial u per (tile, segment) [tile][seg][R][32]
  const float* S;                   // R x ld: S_i = sigma_i u_i^T m per voxel
  const float* V;                   // Q x ndict x R  [q][c][i]: a compartment's rows of
                                    // every dictionary side by side
  const float* coefA;               // ndict x R: 1/(beta + sigma^2)
  const float* coefW;               // ndict x R: sigma^2/(beta^2 + beta sigma^2)
  const int32_t* labels;            // dictionary of each voxel (nullptr: dictionary 0)
  Grid g;
  int Q;
  int nseg;                         // compartment segments per tile
  int ndict;                        // dictionaries (labels in [0, ndict))
  float beta, inv_beta, xi, lam_s, inv_xb;
};

// the device state of Algorithm 1 (map-major Q x ld arrays)
struct AdmmState {
  float *x, *y, *z, *dx, *dy, *dz;   // splits and duals
  float *f, *w, *r, *t;              // f, w = beta f - d_x, r = beta f - d_z, transform scratch
};

// a block of iterations captured once and replayed as a CUDA graph; `key` holds the
// start parity, the block length and each iteration's (test, next test) flags
struct GraphBlock {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;   // kernel launches one replay performs
  int nparts = 0;        // residual partial rows written by the block's last iteration
};

// ------------------------------------------------------------------------------------
// the plan (opaque ssm_plan_t)
// ------------------------------------------------------------------------------------
}  // namespace ssm

struct ssm_plan_s {
  ssm_params p;
  int device = 0;
  ssm::Grid g{};
  int P = 0, Q = 0, n = 0;     // n = min(P, Q): size of the Gram eigenproblem
  int gram_side = 0;           // 0: K K^T, 1: K^T K
  int r = 0, R = 0;            // rank used, padded rank (multiple of 4)
  double xi = 0, dtd_norm = 0, sigma1 = 0, lam_s = 0;
  // largest eigenvalues by FP64 power iteration (ssm_power.cu): K^T K, D^T D, the Hessian
  double kk_power = 0, dtd_power = 0, hess_power = 0;
  int power_iters = 0, power_conv = 0;
  std::vector<double> sigma;   // n singular values, descending
  std::vector<int> perm;       // eigen order (descending) into the Jacobi output
  float plan_ms = 0.f;

  // FP64 plan data
  double* K64 = nullptr;       // P x Q
  double* Bp64 = nullptr;      // P x n  : c = Bp^T m (u_i, or K v_i)
  double* Kt64 = nullptr;      // Q x n  : k_i = K^T u_i (KK^T side) or v_i (K^TK side)
  double* sig64 = nullptr;     // n      : sigma_i (descending)

  // FP32 operands
  float* K32 = nullptr;        // P x Q (objective with the full K)
  float* Kr32 = nullptr;       // P x Q (objective with K_r)
  float* V32 = nullptr;        // Q x R  [q][i]  low-rank right singular vectors
                               // (multi plans: Q x ndict x R, [q][c][i])
  // TF32x3 low-rank form: V (Q x R) and V^T (R x lrtc_qs), split into TF32 hi/lo parts
  float* V1h = nullptr;
  float* V1l = nullptr;
  float* V2h = nullptr;
  float* V2l = nullptr;
  int lrtc_qs = 0;             // row stride of V^T: Q rounded up to 32
  float* coefA = nullptr;      // R      1/(beta + sigma_i^2)
  float* coefW = nullptr;      // R      sigma_i^2/(beta^2 + beta sigma_i^2)
  double* alpha64 = nullptr;   // n      S_i = alpha_i c_i
  float* Mq32 = nullptr;       // Q x Q  (K^T K + beta I)^{-1}, row stride Qp
  __nv_bfloat16* Mhi = nullptr;  // Q x Qp (bf16 split of Mq: hi + lo)
  __nv_bfloat16* Mlo = nullptr;
  float* Gq32 = nullptr;       // Q x n  : h = Gq c
  int Qp = 0;                  // padded row stride of Q x Q operands

  // per-voxel state (map-major, leading dimension g.ld)
  float* Z[2] = {nullptr, nullptr};  // z ping-pong            (Q x ld)
  float* Dl[2] = {nullptr, nullptr}; // dual d ping-pong       (Q x ld)
  float* C32 = nullptr;              // projections c          (n x ld)
  float* S = nullptr;                // S_i = sigma_i u_i^T m  (R x ld)
  float* U[2] = {nullptr, nullptr};  // partial u = V^T (beta z - d) per (tile, segment)
  int64_t lr_grid = 0;               // persistent grid of the low-rank kernel
  float* H = nullptr;                // h = M g                (Q x ld)     dense
  float* Wf = nullptr;               // w = beta z - d (FP32)  (Q x ld)     dense fp32
  float* Acc = nullptr;              // M w                    (Q x ld)     dense fp32
  __nv_bfloat16* Whi[2] = {nullptr, nullptr};  // w split, ping-pong (Q x ld) dense bf16
  __nv_bfloat16* Wlo[2] = {nullptr, nullptr};
  float* Res = nullptr;              // P x ld residual buffer for the objective (lazy)
  float* Mstage = nullptr;           // P x ld device staging for ssm_solve_host (lazy)
  float* Fstage = nullptr;           // Q x ld
  double* red = nullptr;             // reduction partials
  double* red_out = nullptr;         // finished sums (device)
  double* red_host = nullptr;        // pinned host copy
  int* dev_err = nullptr;            // device error word (a kernel's bounded wait gave up)
  int red_cap = 0;                   // capacity (rows of 4 doubles)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  void* tc_state = nullptr;          // tensor-core path descriptors (ssm_tc.cu)
  // optional timing of the dominant kernel of each iteration (ssm_profile_*)
  bool prof_enabled = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs (start, stop)
  size_t prof_used = 0;              // pairs recorded since the last read
  // device bytes the plan holds (every allocation it owns)
  int64_t bytes = 0;
  // persistent grids are launched with `waves` times the resident CTAs (1 = one CTA per
  // resident slot; more = shorter-lived CTAs, so other streams get SMs sooner)
  int waves = 1;
  // compartment-tile width of the tensor-core GEMM (chosen by its autotuner)
  int tc_bn = 256;
  int tc_bn_fused = 0;          // tile width of the fused iteration kernel (0: none fits)
  bool tc_fused = false;        // tensor-core form: one fused GEMM + update kernel per iteration
  bool tc_fused_reg = false;    // ... with the register epilogue (else the staged one)
  // Algorithm 1 (SSM_FORM_ADMM): state, per-axis DCT matrices (forward, inverse), scaling
  ssm::AdmmState adm{};
  float* adm_T[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  float* adm_D = nullptr;
  // voxels inside the object (N bytes, 1 = inside), nullptr = every voxel
  uint8_t* mask = nullptr;
  // the iteration state left by the last completed solve (ssm_solve_resume continues it)
  bool has_state = false;
  int cur_state = 0;           // ping-pong half holding z^k (and w^k, partial u)
  // spatially varying dictionaries (ssm_plan_multi): ndict > 0. V32, coefA and coefW
  // then hold every dictionary's factors ([q][c][i], [c][i]), padded to the common R
  int ndict = 0;
  int32_t* labels = nullptr;         // N dictionary labels
  double* B_multi = nullptr;         // ndict x P x R: sigma_{c,i} u_{c,i} (S = B^T m per voxel)
  int mseg = 1;                      // compartment segments per voxel tile
  std::vector<int> ranks;            // r_c per dictionary
  ssm::TableProblem* tprob = nullptr;  // the iteration's problem descriptor (device)
  int4* ttable = nullptr;            // its (problem, tile, segment) table (device)
  int64_t tblocks = 0;               // entries of the table
  // iteration blocks replayed as CUDA graphs (ssm_plan_set_graphs)
  bool use_graphs = false;
  std::vector<ssm::GraphBlock> graphs;
};

namespace ssm {

// parameter checks of ssm_plan; device bytes of a plan for p (see ssm_plan_footprint)
ssm_status validate_params(const ssm_params* p);
ssm_status plan_footprint(const ssm_params& p, bool staging, int waves, int64_t* persistent,
                          int64_t* peak);
// ssm_plan with the launch-waves setting
ssm_status plan_create(ssm_plan_t* out, const ssm_params* p, const double* K_host, int device,
                       cudaStream_t s, int waves, bool zlink = true);

// ------------------------------------------------------------------------------------
// launchers (each returns a status; the stream is the caller's)
// ------------------------------------------------------------------------------------
// plan stage (ssm_plan_kernels.cu)
ssm_status gram_fp64(const double* K, int P, int Q, int side, double* A, cudaStream_t s);
ssm_status jacobi_eigen(double* A, int n, double* E, double* scratch, std::vector<double>& evals,
                        cudaStream_t s);
ssm_status factors_fp64(ssm_plan_s* pl, const double* E, cudaStream_t s);
// power iterations for lambda_max of K^T K (Gram A, n x n) and D^T D (ssm_power.cu)
ssm_status hessian_power(ssm_plan_s* pl, const double* A, int n, cudaStream_t s);
ssm_status form_dense_inverse(ssm_plan_s* pl, cudaStream_t s);
ssm_status beta_weights(ssm_plan_s* pl, cudaStream_t s);
ssm_status project_data(const ssm_plan_s* pl, const float* M, int64_t ldm, int ncomp,
                        cudaStream_t s);
ssm_status split_bf16(const float* X, int rows, int cols, int64_t ldx,
                      __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo, cudaStream_t s);

// low-rank iteration (ssm_lowrank.cu)
// low-rank iteration k -> k+1 with state (z, per-voxel u); `check` forms the residual
// sums (and reads d^k), `write_d` stores d^{k+1} for the next iteration's test
ssm_status lowrank_iteration(ssm_plan_s* pl, int cur, bool check, bool write_d, double* partial,
                             int* nparts, cudaStream_t s);
int lowrank_max_partials(const ssm_plan_s* pl);
int64_t lowrank_grid(const ssm_plan_s* pl);
int64_t lowrank_partial_floats(const ssm_plan_s* pl, int64_t grid);

// low-rank iteration with both rank-r products on the tensor cores (ssm_lowrank_tc.cu)
int lrtc_padded_rank(int r, bool three_d);
int64_t lrtc_grid(const ssm_plan_s* pl);
int64_t lrtc_partial_floats(const ssm_plan_s* pl, int64_t grid);
ssm_status lrtc_prepare();
ssm_status lrtc_split_basis(ssm_plan_s* pl, cudaStream_t s);
ssm_status lrtc_iteration(ssm_plan_s* pl, int cur, bool check, bool write_d, double* partial,
                          int* nparts, cudaStream_t s);

// work-table iteration (ssm_table.cu): a tile is 32 voxels; padded ranks 4, 8, .., 32
constexpr int kTableTile = 32;
constexpr int kMaxTableRank = 32;
int table_padded_rank(int r);
int table_blocks_per_sm(int R);
// compartment segments per tile for a problem of ntiles tiles and Q compartments
int table_segments(int64_t ntiles, int Q, int R);
int64_t table_state_floats(int64_t N, int nseg, int R);   // one partial-u buffer
// (problem, tile, segment) entries of one problem, segment-major, appended to `out`
void table_entries(int problem, int64_t ntiles, int nseg, std::vector<int4>* out);
// B [P][R] = alpha_i Bp[p][i] for i < r (sigma_i u_i), zero for r <= i < R
ssm_status table_gather_factors(const double* Bp, const double* alpha, int P, int n, int r, int R,
                                double* out, cudaStream_t s);
// S [R][ld] = B[c(n)]^T m_n per voxel (FP64 accumulation); labels nullptr: dictionary 0
ssm_status table_project(const double* B, int P, int R, const int32_t* labels, const float* M,
                         int64_t ldm, int64_t N, float* S, int64_t ld, cudaStream_t s);
// one iteration of every problem of the table (blocks = entries); z^k in Z[cur]
ssm_status table_iteration(const TableProblem* probs, const int4* table, int64_t nblocks, int R,
                           int cur, bool check, bool write_d, double* partial, cudaStream_t s);


// dense iteration and shared kernels (ssm_dense.cu)
ssm_status sgemm(int M, int N, int K, float alpha, const float* A, int64_t lda,
                 const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                 cudaStream_t s);
ssm_status dense_update(ssm_plan_s* pl, int cur, const float* acc, bool check,
                        bool write_fp32_w, bool write_bf16_w, double* partial, int* nparts,
                        cudaStream_t s);
int dense_max_partials(const ssm_plan_s* pl);
ssm_status finish_partials(const double* partial, int nparts, int width, double* out,
                           cudaStream_t s);
ssm_status objective_terms(const ssm_plan_s* pl, const float* Res, int P, const float* F,
                           int64_t ldf, double* partial, int* nparts, cudaStream_t s);

// Algorithm 1 (ssm_admm.cu)
ssm_status admm_tables(ssm_plan_s* pl, std::vector<std::pair<float**, std::vector<float>>>* out);
int admm_partial_rows(const ssm_plan_s* pl);
ssm_status admm_prepare();
ssm_status admm_iteration(ssm_plan_s* pl, bool check, double* partial, int* nparts,
                          cudaStream_t s);

// tensor-core dense iteration (ssm_tc.cu)
ssm_status tc_prepare(ssm_plan_s* pl, cudaStream_t s);
ssm_status tc_iteration(ssm_plan_s* pl, int cur, bool check, double* partial, int* nparts,
                        cudaStream_t s);
ssm_status tc_gemm(ssm_plan_s* pl, int cur, cudaStream_t s);
ssm_status tc_update_prepare(ssm_plan_s* pl);
int tc_update_grid(const ssm_plan_s* pl);
ssm_status tc_update(ssm_plan_s* pl, int cur, bool check, double* partial, int* nparts,
                     cudaStream_t s);
void tc_release(ssm_plan_s* pl);
int tc_max_partials(const ssm_plan_s* pl);
int tc_gemm_grid(const ssm_plan_s* pl);
int tc_tile_width(const ssm_plan_s* pl);

}  // namespace ssm
