/*
 * ssm.h -- C ABI of the GB300 LADMM solver for spatial-spectral compartment mapping.
 *
 * The library estimates nonnegative compartment maps F (Q x N) from multi-contrast
 * data M (P x N) and a dictionary K (P x Q) by solving
 *
 *     min_{F >= 0}  1/2 ||M - K F||_F^2 + lambda * 1/2 ||D F||^2            (Eq. 7, Eq. 8)
 *
 * with the linearized ADMM iteration of Algorithm 2 (Sec. III-F). D is the spatial
 * finite-difference operator of Eq. 8 on an axis-aligned 1D/2D/3D voxel grid with a
 * free (maskless) boundary: 2 neighbours per axis, fewer at the image edge.
 *
 * Two forms of the per-voxel f-step are offered:
 *   SSM_FORM_LOWRANK  the rank-r form of Eq. 27/28, exactly as Algorithm 2 (the paper's
 *                     proposed method); HBM-bandwidth bound.
 *   SSM_FORM_DENSE    the full-rank form of Eq. 26, f_n = (K^T K + beta I)^{-1} c_n, a
 *                     Q x Q by Q x N contraction every iteration (FP32 SIMT, or BF16 split
 *                     hi+lo products on the tcgen05 tensor cores with FP32 accumulation).
 *
 * Conventions for every entry point:
 *   - Layouts are row-major. K is P x Q (row p = one contrast encoding). M is P x N and
 *     F is Q x N, "map-major": row p (or q) is one image over the N voxels, with the
 *     voxel index n = x + nx*(y + ny*z) (x fastest). Leading dimensions are in elements.
 *   - Device pointers must be CUDA device memory on the plan's device; host pointers
 *     are ordinary host memory (pinned memory makes the copies asynchronous).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     All GPU work is enqueued on it; calls that return host values synchronise it.
 *   - Errors are reported only by the returned status (never by a device trap);
 *     ssm_last_error() gives a human-readable message for the calling thread.
 *   - Ownership: the caller owns K, M, F and `info`; the plan owns every device buffer
 *     it allocates (factors, state, workspace) and ssm_destroy releases them.
 */
#ifndef SSM_H
#define SSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssm_plan_s* ssm_plan_t;

typedef enum {
  SSM_OK = 0,
  SSM_EINVAL = 1,          /* invalid argument (sizes, pointers, parameters)        */
  SSM_ENOMEM = 2,          /* device allocation failed                              */
  SSM_ECUDA = 3,           /* a CUDA runtime/driver call failed                     */
  SSM_ENAN = 4,            /* a residual became NaN or Inf                          */
  SSM_ETIMEOUT = 5,        /* a bounded device-side wait gave up                    */
  SSM_EUNSUPPORTED = 6,    /* valid request outside what this build implements      */
  SSM_ENOTCONVERGED = 7,   /* tolerance set but not reached within max_iter (info)  */
  SSM_EPENDING = 8         /* a served request has not finished yet                 */
} ssm_status;

typedef enum {
  SSM_FORM_LOWRANK = 0,    /* Algorithm 2 with the rank-r f-step of Eq. 28          */
  SSM_FORM_DENSE = 1,      /* full-rank f-step of Eq. 26                            */
  SSM_FORM_ADMM = 2        /* Algorithm 1, the three-split ADMM the paper compares
                              against (Sec. II-C): full-rank x-step, exact z-step by
                              DCT-II diagonalisation of lambda D^T D + beta I (grid
                              axes up to 256); FP32 only; F = y (the nonnegative
                              split); residuals: ||f-x||^2+||f-y||^2+||f-z||^2 and
                              ||y^{k+1}-y^k||^2, each relative to ||y||^2           */
} ssm_form;

typedef enum {
  SSM_FP32 = 0,            /* FP32 arithmetic, FP32 state                           */
  SSM_BF16X3 = 1,          /* dense form: BF16 hi/lo split products (3 tcgen05 MMAs
                              per tile, FP32 accumulation), FP32 state              */
  SSM_TF32X3 = 2           /* low-rank form: both rank-r products of an iteration
                              (V a and V^T w, Eq. 28) on the tcgen05 tensor cores,
                              kind::tf32 with TF32 hi/lo split operands (3 MMAs per K
                              step), FP32 accumulation; z and u FP32. The rank is
                              padded to 32 or 64 (r <= 64; r <= 32 on 3D grids)     */
} ssm_precision;

typedef struct {
  int ndim;                /* 1, 2 or 3                                             */
  int64_t dims[3];         /* grid (nx, ny, nz); unused trailing dims ignored       */
  int P, Q;                /* dictionary size                                       */
  double lambda;           /* regularisation weight of Eq. 7, >= 0                  */
  double beta;             /* ADMM penalty, > 0 (the paper tunes it, Sec. III-E)    */
  double xi_p;             /* z-step proximal weight; <= 0 selects Eq. 32:
                              0.75 * lambda * ||D^T D|| + 1e-10                     */
  int form;                /* ssm_form                                              */
  int rank;                /* low-rank form: 0 = smallest r with
                              ||K - K_r||_F < rank_tol ||K||_F (Sec. III-E), > 0 = r */
  double rank_tol;         /* <= 0 selects 5e-5 (the paper's 0.005 %)               */
  int precision;           /* ssm_precision: dense form FP32 or BF16X3; low-rank form
                              FP32 or TF32X3 (BF16X3 there runs FP32); ADMM FP32     */
  int stencil_pairs;       /* 2 = literal Eq. 8 (each neighbour pair counted from
                              both ends, D^T D = 2 L); 1 = once per pair (D^T D = L) */
  int max_iter;            /* iteration budget (>= 0)                               */
  int check_every;         /* residual test period; 0 = never test                  */
  double tol_primal;       /* stop when ||z-f|| <= tol_primal ||z|| ...            */
  double tol_change;       /* ... and ||z^{k+1}-z^k|| <= tol_change ||z^{k+1}||;
                              a tolerance <= 0 is not used; none used = fixed budget */
} ssm_params;

typedef struct {
  int status;              /* ssm_status of the solve                               */
  int iterations;          /* iterations run                                        */
  int rank;                /* r used by the low-rank form (min(P,Q) for dense)      */
  int gram_side;           /* 0: eigenpairs from K K^T (P x P); 1: from K^T K       */
  double xi_p;             /* xi_p used                                             */
  double dtd_norm;         /* ||D^T D|| (closed form for the box grid)              */
  double sigma1;           /* largest singular value of K                           */
  double res_primal;       /* ||z - f|| / ||z|| at the last test (-1: none)          */
  double res_change;       /* ||z^{k+1} - z^k|| / ||z^{k+1}|| at the last test      */
  double plan_ms;          /* device time of ssm_plan                               */
  /* The largest eigenvalue of the Hessian of Eq. 7, H = I (x) K^T K + lambda D^T D (x) I,
   * which bounds the step of a gradient method on Eq. 7; xi_p of Eq. 32 is to exceed
   * 0.75 lambda ||D^T D|| (the convergence condition the paper cites, Sec. III-C). H is
   * a Kronecker sum, so lambda_max(H) = lambda_max(K^T K) + lambda lambda_max(D^T D),
   * and D^T D on the box grid is a Kronecker sum of path-graph Laplacians; ssm_plan runs
   * one FP64 iteration on the device per factor: power iteration on the Gram matrix of
   * the smaller side for K^T K, and power iteration on (4 s I - s L)^{-1} (inverse
   * iteration) for each grid axis of 2 .. 2^22 voxels. With a mask the grid values are
   * the box grid's (an upper bound of the masked operator's).                          */
  double hess_norm;        /* lambda_max(K^T K) + lambda lambda_max(D^T D)           */
  double kk_norm;          /* lambda_max(K^T K) by power iteration (sigma_1^2)       */
  double dtd_norm_power;   /* lambda_max(D^T D) by power iteration                   */
  int power_iters;         /* most steps any of the iterations took                 */
  int power_converged;     /* 1: every iteration met its stopping rule (its Rayleigh
                              quotient rose by at most 1e-15 relative over 32 steps
                              for K^T K, over one step for an axis); 0: one hit its
                              cap (its value is a lower bound) or an axis longer
                              than 2^22 voxels was left out                          */
} ssm_info;

/* Fill `p` with defaults: 2D, lambda 0, beta 1, xi_p rule, low-rank auto rank,
 * literal stencil, FP32, max_iter 300, check_every 10, no tolerance. */
ssm_status ssm_default_params(ssm_params* p);

/*
 * Plan a solver for one dictionary and one grid (Algorithm 2, steps 1-3).
 *   K_host : P x Q row-major doubles on the host, read during the call only.
 * Work done (on `stream`, device `device`): K is copied to the device; the Gram
 * matrix of the smaller side (K K^T if P <= Q, else K^T K) is formed in FP64 and
 * eigendecomposed by cyclic Jacobi in FP64, giving sigma_i, u_i, v_i of Eq. 27; the
 * rank rule of Sec. III-E picks r; the weights sigma_i^2 / (beta^2 + beta sigma_i^2)
 * of Eq. 28 (low-rank) or the matrix (K^T K + beta I)^{-1} of Eq. 26 (dense) are
 * formed in FP64; xi_p follows Eq. 32 unless given. The per-voxel state (z, d and
 * per-voxel projections) is allocated for N = prod(dims) voxels.
 * Returns SSM_EINVAL for bad sizes/parameters, SSM_ENOMEM if the state does not fit.
 * On success *out owns every allocation; on failure *out is NULL.
 */
ssm_status ssm_plan(ssm_plan_t* out, const ssm_params* p, const double* K_host,
                    int device, void* stream);

/*
 * ssm_plan with a launch setting (no counterpart in the paper): the solver's persistent
 * kernels are launched with launch_waves (1..64) times as many CTAs as fit on the device
 * at once, each doing 1/launch_waves of the work. 1 (what ssm_plan uses) gives the
 * highest throughput; more waves make CTAs shorter-lived, so kernels on other streams,
 * higher-priority ones first, get SMs within a fraction of a kernel's duration. Results
 * are the same within rounding: the low-rank form sums its per-voxel partial products
 * over a grid-dependent number of segments.
 */
ssm_status ssm_plan_ex(ssm_plan_t* out, const ssm_params* p, const double* K_host,
                       int device, void* stream, int launch_waves);

/*
 * A batch of nbatch independent problems that share the dictionary, the grid (p: one 1D
 * or 2D slice), lambda, beta and the stopping rule -- e.g. the slices of one subject -- as
 * one plan whose kernels solve them all at once (batching, no counterpart in the paper).
 * The plan's grid is (nx, ny, nbatch) with no smoothness across the batch axis: each
 * slice's problem is exactly Eq. 7 on its own grid, and xi_p (Eq. 32) is the slice's.
 * M and F hold the slices one after another: P x (N nbatch), slice b in columns
 * [b N, (b + 1) N). The residual test is over the whole batch (the batch stops when the
 * stacked residuals meet the tolerance). Masks apply (N nbatch bytes). launch_waves as
 * in ssm_plan_ex.
 */
ssm_status ssm_plan_batched(ssm_plan_t* out, const ssm_params* p, int64_t nbatch,
                            const double* K_host, int device, void* stream, int launch_waves);

/*
 * Spatially varying dictionaries (Sec. IV-D: the fingerprinting experiment's dictionary
 * per quantised B1 level): voxel n is modelled with dictionary c(n), so Eq. 7 becomes
 *     min_{F >= 0} sum_n 1/2 ||m_n - K_{c(n)} f_n||^2 + lambda/2 ||D F||^2
 * and Algorithm 2 runs unchanged but for the f-step, which takes the voxel's own
 * dictionary's rank-r factors (Eq. 27, Eq. 28; each dictionary's rank by the rule of
 * Sec. III-E with p->rank_tol, or p->rank for all). The z-step, the dual step, xi_p
 * (Eq. 32) and the stopping rule are those of one dictionary.
 *   p           : as for ssm_plan; form must be SSM_FORM_LOWRANK and precision SSM_FP32
 *                 (else SSM_EUNSUPPORTED). P and Q are every dictionary's shape.
 *   ndict       : number of dictionaries, 1..65536.
 *   K_host      : ndict x P x Q doubles on the host, dictionary c at offset c P Q,
 *                 each row-major P x Q; read during the call only.
 *   labels_host : N int32 labels on the host (voxel order of M's columns), each in
 *                 [0, ndict) (else SSM_EINVAL, nothing allocated); read during the call.
 * Each dictionary's rank must be <= 32 (else SSM_EUNSUPPORTED). ssm_solve,
 * ssm_solve_host, ssm_solve_resume, ssm_plan_set_stopping, graphs, profiling and
 * ssm_plan_info apply (info->rank and sigma1 are the largest over the dictionaries,
 * kk_norm the largest lambda_max(K_c^T K_c); hess_norm is not formed, 0). ssm_objective,
 * ssm_plan_factors, ssm_plan_set_mask and ssm_plan_set_beta return SSM_EUNSUPPORTED.
 * Planning synchronises `stream`.
 */
ssm_status ssm_plan_multi(ssm_plan_t* out, const ssm_params* p, int ndict,
                          const double* K_host, const int32_t* labels_host, int device,
                          void* stream);

/*
 * Groups: independent low-rank problems of differing N, P and Q solved together, one
 * launch per iteration for all of them (the work-table kernel: a table of (problem,
 * voxel tile, compartment segment) entries, one per block). For many small solves (the
 * serving path's smallest requests) this replaces one launch per problem per iteration.
 * No counterpart in the paper: each problem runs Algorithm 2 exactly as ssm_solve does,
 * with its own stopping rule, and leaves the group when it stops.
 *   plans : nplans plans on one device, each SSM_FORM_LOWRANK / SSM_FP32, rank <= 32,
 *           one dictionary (not ssm_plan_multi), no mask (else SSM_EUNSUPPORTED). The
 *           group borrows them: they must outlive it. It copies their factors (V_r, the
 *           weights, sigma_i u_i) at creation, so a later ssm_plan_set_beta needs a new
 *           group, and it runs in their state buffers (z, d), so a plan must not be
 *           solved on its own while a group solve that holds it runs.
 * A problem's iterates do not depend on the other problems of the group (nor on their
 * ranks): a problem solved in any group gives the same bits. They are not the bits of
 * ssm_solve (another kernel, another summation order), within rounding of them.
 */
typedef struct ssm_group_s* ssm_group_t;

ssm_status ssm_group_create(ssm_group_t* out, int nplans, const ssm_plan_t* plans,
                            void* stream);

/*
 * Solve every problem of the group. M_devs[i] (P_i x N_i, leading dimension ldms[i]) and
 * F_devs[i] (Q_i x N_i, ldfs[i]) are device buffers; infos (nplans entries, may be NULL)
 * receive each problem's status, iterations and residuals as ssm_solve's info. Each
 * problem uses its plan's max_iter, check_every and tolerances. Returns SSM_OK when
 * every problem ended SSM_OK, else the first error status among the problems (then
 * SSM_ENOTCONVERGED if only some ran out of iterations); every F is written. Synchronises
 * `stream` at each residual test.
 */
ssm_status ssm_group_solve(ssm_group_t group, const float* const* M_devs, const int64_t* ldms,
                           float* const* F_devs, const int64_t* ldfs, ssm_info* infos,
                           void* stream);

/* Device bytes the group holds (its own buffers, not the plans'). */
ssm_status ssm_group_device_bytes(ssm_group_t group, int64_t* bytes);

/* Free the group (not its plans). NULL is accepted. */
ssm_status ssm_group_destroy(ssm_group_t group);

/*
 * Run the LADMM iteration (Algorithm 2, steps 4-12) on data M and write F = z.
 *   M_dev : P x N floats on the device, leading dimension ldm >= N; read only.
 *   F_dev : Q x N floats on the device, leading dimension ldf >= N; written.
 *   info  : host struct, may be NULL; filled after the solve (synchronises `stream`).
 * z, f and d start at 0 (Algorithm 2, step 2). The projections of M on the singular
 * vectors (g_n of step 4) are formed once with FP64 accumulation. The returned F is
 * the feasible iterate z (F >= 0 elementwise). With a tolerance set, residuals are
 * tested every check_every iterations (a host read of three FP64 sums); the status
 * is SSM_ENOTCONVERGED when the budget ran out first (F is still written).
 * Calls on one plan must not overlap (the plan holds the iteration state).
 */
ssm_status ssm_solve(ssm_plan_t plan, const float* M_dev, int64_t ldm, float* F_dev,
                     int64_t ldf, ssm_info* info, void* stream);

/*
 * Continue the iteration (checkpoint/resume within a plan, no counterpart in the paper):
 * run max_iter more iterations from the state the plan's last completed ssm_solve /
 * ssm_solve_resume left (z, d and the form's internal operands stay on the device
 * between calls), with the same stopping rule, and write F = z. M must be the data of
 * that solve (its projections are formed again). The iterates are exactly those of one
 * solve running the iterations of both calls. info->iterations counts this call's
 * iterations. SSM_EINVAL when the plan holds no state: before the first solve, after a
 * failed one, or after ssm_plan_set_beta / ssm_plan_set_mask.
 */
ssm_status ssm_solve_resume(ssm_plan_t plan, const float* M_dev, int64_t ldm, float* F_dev,
                            int64_t ldf, ssm_info* info, void* stream);

/*
 * Same as ssm_solve with HOST buffers: M_host (P x N, ldm) is copied in, the solve
 * runs, F_host (Q x N, ldf) is copied out; returns after the copy-out completes.
 * Staging buffers are the plan's own (allocated at plan time).
 */
ssm_status ssm_solve_host(ssm_plan_t plan, const float* M_host, int64_t ldm,
                          float* F_host, int64_t ldf, ssm_info* info, void* stream);

/*
 * Objective of Eq. 7 / Eq. 8 for given F (device, Q x N, ldf) and M (device, P x N):
 *   1/2 ||M - K' F||_F^2 + lambda * 1/2 ||D F||^2,
 * with K' the dictionary the plan iterates with (K for the dense form, the truncated
 * K_r of Eq. 27 for the low-rank form) unless use_full_k != 0 (then K). The product
 * K' F is FP32 with FP32 accumulation; both sums are accumulated in FP64.
 * Writes *J_host and synchronises `stream`.
 */
ssm_status ssm_objective(ssm_plan_t plan, const float* M_dev, int64_t ldm,
                         const float* F_dev, int64_t ldf, int use_full_k,
                         double* J_host, void* stream);

/*
 * Objective of Eq. 7 / Eq. 8 without allocating any device memory and without a plan
 * (the paper has no counterpart: this serves callers that cannot allocate -- e.g. a
 * pipeline that forbids allocation once it runs, a process whose device memory is
 * held by another allocator, or work on a busy device where cudaMalloc/cudaFree would
 * synchronise it). Computes 1/2 ||M - K F||_F^2 + lambda * 1/2 ||D F||^2 from device
 * buffers K (P x Q row-major floats), M (P x N, ldm) and F (Q x N, ldf) on the grid
 * `dims` (ndim 1..3), with the stencil convention `stencil_pairs` (as in ssm_params);
 * K F is FP32 with FP32 accumulation, both sums FP64. Writes *J_host and synchronises
 * `stream`.
 * Scratch: a fixed device array inside the library (256 KB per device, kept until
 * the process exits) caps N at 4,194,304 voxels; larger grids get SSM_EINVAL. The
 * first call on a device looks up that array's device address (with the device
 * current), so make the first call before any stream capture. All calls share the
 * array: calls that overlap on the GPU race. Nothing needs clearing between calls.
 */
ssm_status ssm_objective_noalloc(const float* K_dev, int P, int Q, const float* M_dev,
                                 int64_t ldm, const float* F_dev, int64_t ldf, int ndim,
                                 const int64_t* dims, double lambda, int stencil_pairs,
                                 double* J_host, void* stream);

/*
 * The plan-level fields of ssm_info (rank, gram_side, xi_p, dtd_norm, sigma1, plan_ms and
 * the power-iteration results) without solving; status SSM_OK, iterations 0, residuals
 * -1. Host only (no device work).
 */
ssm_status ssm_plan_info(ssm_plan_t plan, ssm_info* info);

/*
 * Read back the plan's factors (for tests): sigma (min(P,Q) doubles, descending) and,
 * when non-NULL, V_r (Q x r row-major doubles, the first r right singular vectors).
 */
ssm_status ssm_plan_factors(ssm_plan_t plan, double* sigma_host, double* vr_host,
                            int* rank_out);

/*
 * Kernel timing (measurement support, no counterpart in the paper). When enabled,
 * each solve records a CUDA event pair on `stream` around every launch of the
 * iteration's dominant kernel (the fused low-rank kernel, the FP32 matrix product,
 * or the tensor-core kernel) and ssm_profile_read returns the summed device time
 * (ms) and launch count since the last read (then resets them; synchronises the
 * plan's device). Disabled by default; enabling costs two event records per
 * iteration.
 */
ssm_status ssm_profile_enable(ssm_plan_t plan, int enable);
ssm_status ssm_profile_read(ssm_plan_t plan, double* main_kernel_ms,
                            int64_t* main_kernel_launches);

/*
 * Replay the solve loop's iteration blocks as CUDA graphs (launch-overhead support, no
 * counterpart in the paper). A block is the run of iterations up to the next residual
 * test, or 64 iterations when no test comes sooner; each distinct block (start parity,
 * length, test pattern) is captured once on the plan and replayed by later blocks and
 * later solves. Results are bitwise the same as with direct launches. Graphs are used
 * only on a stream other than the legacy default stream, when the stream is not already
 * being captured, and when profiling is off; otherwise launches are issued directly.
 */
ssm_status ssm_plan_set_graphs(ssm_plan_t plan, int enable);

/*
 * Restrict the problem to the voxels inside an object: mask_host holds N bytes (voxel
 * order as M's columns), nonzero = inside; NULL removes the mask. This is the paper's
 * maskless form (footnote to Algorithm 1): only voxels inside the object are estimated
 * and no smoothness is imposed across the object boundary, i.e. D of Eq. 8 has the
 * pairs of the grid graph the mask induces (an inside voxel's neighbours outside the
 * object do not count). Later solves return F = 0 outside the object, and ssm_objective
 * sums the data term over the inside voxels and the roughness over the induced pairs.
 * xi_p (Eq. 32) keeps the box grid's ||D^T D||, an upper bound of the masked operator's
 * norm (removing edges cannot raise a graph Laplacian's eigenvalues). The plan copies the
 * mask to the device (N more bytes, not in ssm_plan_footprint) and drops its captured
 * graphs; synchronises `stream`. The ADMM form does not support masks
 * (SSM_EUNSUPPORTED).
 */
ssm_status ssm_plan_set_mask(ssm_plan_t plan, const uint8_t* mask_host, void* stream);

/*
 * Change the plan's stopping rule for later solves (max_iter >= 0, check_every >= 0,
 * tolerances as in ssm_params); the factors, state and beta are kept, so a resumed solve
 * (ssm_solve_resume) can run with a new budget. Host only; must not overlap a solve on
 * the same plan.
 */
ssm_status ssm_plan_set_stopping(ssm_plan_t plan, int max_iter, int check_every,
                                 double tol_primal, double tol_change);

/*
 * Change the plan's beta without refactorising K (the spectral factors of Sec. III-D do
 * not depend on beta): re-forms the weights of Eq. 28 (low-rank) or the inverse of
 * Eq. 26 (dense) on `stream` and drops the plan's captured graphs. The next solve uses
 * the new beta; xi_p (Eq. 32) does not depend on beta and is kept.
 */
ssm_status ssm_plan_set_beta(ssm_plan_t plan, double beta, void* stream);

/*
 * The beta heuristic of Sec. III-E: beta is tuned on the centre patch of the image
 * (3 voxels per axis, starting at dims/2 - 1) and reused on the whole image. Each
 * candidate beta_k = sigma_1^2 * 10^(grid_lo + (grid_hi - grid_lo) k / (n_grid - 1)),
 * k = 0 .. n_grid-1, runs `iters` iterations of the low-rank form (rank and lambda as in
 * `p`; the patch's own xi_p rule) from the zero start; the candidate with the lowest
 * objective J(z) (Eq. 7 with K_r) wins, the smaller beta on a tie. The paper asks for
 * the fastest convergence without fixing a measure: the lowest J after a fixed budget
 * is the reading taken here.
 *   p      : grid, P, Q, lambda, rank, rank_tol, stencil_pairs (beta, form, precision
 *            and the stopping rule are ignored)
 *   M_host : P x N floats (ldm >= N), host memory; only the patch's columns are read
 *   betas, J : n_grid doubles each, may be NULL (the candidates and their objectives)
 * One plan is made on the patch (one eigendecomposition); candidates differ only in
 * their beta-dependent weights (ssm_plan_set_beta). Synchronises `stream`.
 */
ssm_status ssm_tune_beta(const ssm_params* p, const double* K_host, const float* M_host,
                         int64_t ldm, int iters, int n_grid, double grid_lo, double grid_hi,
                         int device, void* stream, double* beta_out, double* betas,
                         double* J);

/*
 * Device memory a plan for `p` would take on `device`, from the same sizes ssm_plan
 * allocates: *persistent_bytes = what the plan holds between calls, including the
 * staging buffers of ssm_solve_host; *peak_bytes = that plus the temporaries of
 * planning. For the low-rank form without a fixed rank the bound assumes the largest
 * supported rank, min(P, Q, 64). Allocates nothing.
 */
ssm_status ssm_plan_footprint(const ssm_params* p, int device, int64_t* persistent_bytes,
                              int64_t* peak_bytes);

/* Launch configuration a plan uses (measurement support, no counterpart in the paper). */
typedef struct {
  int launch_waves;        /* see ssm_plan_ex                                        */
  int gemm_tile_n;         /* tensor-core GEMM compartment-tile width (autotuned), 0
                              when the plan has no tensor-core product              */
  int gemm_grid;           /* CTAs of the tensor-core GEMM                           */
  int update_grid;         /* CTAs of the tensor-core form's update kernel (two-kernel
                              iteration only)                                       */
  int lowrank_grid;        /* CTAs of the fused low-rank kernel                      */
  int sm_count;            /* SMs of the plan's device                               */
  int tc_fused;            /* tensor-core iteration: 0 = GEMM + update kernel; 1 = one
                              kernel, the update in the GEMM's epilogue with its reads
                              staged in shared memory by TMA; 2 = one kernel, reads
                              pipelined in registers. Chosen at plan time by timing
                              the candidates; results are identical                 */
} ssm_launch_info;

ssm_status ssm_plan_launch_info(ssm_plan_t plan, ssm_launch_info* out);

/* Device bytes the plan currently holds (every allocation it owns). */
ssm_status ssm_plan_device_bytes(ssm_plan_t plan, int64_t* bytes);

/* Free everything the plan owns. NULL is accepted. Synchronises the plan's device. */
ssm_status ssm_destroy(ssm_plan_t plan);

/*
 * ------------------------------------------------------------------------------------
 * Serving: continuous batching of independent solves on one device (no counterpart in
 * the paper, which fits one data set at a time).
 *
 * A server owns `max_active` workers, each a host thread with its own CUDA stream.
 * Requests are admitted while a worker is free and the request's device footprint
 * (ssm_plan_footprint, peak) fits in what remains of the HBM budget. Admission is
 * first-come first-served; a later request may pass a waiting one that does not fit
 * yet ("backfill"), but at most `max_bypass` times, after which admission waits for
 * memory to free up. Admitted solves run concurrently on their streams, so their
 * kernels overlap on the GPU. Requests are ranked by footprint (the iteration is
 * HBM-bound, so the footprint stands for the cost of an iteration): up to `small_bytes`
 * is class 0, each factor of 4 above is one class more, up to the device's number of
 * stream priorities, and a class-c request runs on a stream of the c-th highest
 * priority. `reserved_small` workers take class-0 requests only, so a small request is
 * admitted even while large ones hold every other worker. Requests above class 0 have
 * their plans made by ssm_plan_ex(...,
 * large_waves), so smaller solves get SMs within a fraction of a larger solve's
 * kernel. With `cache_plans`, a finished solve's plan (factors and
 * state) stays resident; a later request with the same K, grid and plan parameters
 * (all of ssm_params except max_iter, check_every, tol_primal and tol_change) reuses
 * it without planning again. Idle plans are evicted least recently used first when a
 * new request needs their memory. Each request's result is exactly what ssm_solve_host
 * (or ssm_solve) gives for it alone on a plan made with the same launch waves: the
 * kernels and launch shapes do not depend on what else runs. With `group_small`, small
 * low-rank requests are solved in groups (one launch per iteration for a whole group);
 * their results are exactly those of a group of one, whatever else is in the group.
 * ------------------------------------------------------------------------------------
 */
typedef struct ssm_server_s* ssm_server_t;

typedef struct {
  int device;              /* CUDA device the server runs on                        */
  int max_active;          /* solves in flight at once, >= 1                         */
  int64_t hbm_budget;      /* device bytes the server may hold in plans; <= 0 selects
                              90 % of the device's free memory at creation          */
  int use_graphs;          /* replay iteration blocks as CUDA graphs                 */
  int cache_plans;         /* keep idle plans resident for reuse                     */
  int max_bypass;          /* passes of a waiting request by later ones; < 0 selects
                              2 * max_active                                        */
  int64_t simulate_us;     /* > 0: scheduler test mode. Nothing is planned and no GPU
                              work is issued; an admitted request holds its slot and
                              its footprint for max_iter * simulate_us microseconds,
                              leaves F untouched and finishes with SSM_OK and 0
                              iterations. 0 = normal operation                      */
  int64_t small_bytes;     /* footprint bound of the highest-priority class         */
  int large_waves;         /* launch waves of the plans of larger requests, 1..64    */
  int reserved_small;      /* workers that admit class-0 requests only (so a small
                              request never queues behind large ones holding every
                              worker); < 0 selects 1 when max_active >= 2; at most
                              max_active - 1                                         */
  int group_small;         /* > 1: a worker that admits a class-0 low-rank FP32 request
                              with device buffers also admits up to group_small - 1
                              more such requests waiting behind it, and solves them
                              as one group (ssm_group_*: one launch per iteration for
                              all); such a request then always runs in a group, alone
                              or not, so its result does not depend on the others.
                              0 or 1: off (the default)                             */
} ssm_server_config;

typedef struct {
  int status;              /* ssm_status of the solve                               */
  int iterations;          /* iterations run                                        */
  double res_primal;       /* residuals at the last test (-1: none)                 */
  double res_change;
  double queue_ms;         /* submit -> admitted                                    */
  double plan_ms;          /* host time spent planning (0 when a plan was reused)   */
  double solve_ms;         /* admitted -> F_host written (planning included)        */
  double latency_ms;       /* submit -> F_host written                              */
  int64_t footprint;       /* device bytes reserved at admission (peak estimate)    */
  int64_t order;           /* admission sequence number, from 0                     */
  int slot;                /* worker that ran the solve                             */
  int plan_reused;         /* 1 if a resident plan was reused                       */
  int group_size;          /* requests solved together with it in one group (itself
                              included); 0 when it ran on its own (ssm_solve)       */
} ssm_request_info;

typedef struct {
  int64_t submitted, completed, failed, rejected;
  int64_t plans_created, plans_reused, plans_evicted;
  int64_t bytes_held;      /* reserved now: running requests and resident plans     */
  int64_t peak_bytes_held; /* largest reservation seen (never above hbm_budget)     */
  int64_t budget;          /* the HBM budget in force                               */
  int active, pending;     /* requests running / waiting now                        */
} ssm_server_stats;

/* Defaults: device 0, 4 workers, 90 % of free memory, graphs on, plan cache on,
 * max_bypass 2 * max_active, normal operation, small_bytes 64 MiB, large_waves 8,
 * one worker reserved for class-0 requests. */
ssm_status ssm_server_default_config(ssm_server_config* c);

/* Create a server (threads and streams start here). */
ssm_status ssm_server_create(ssm_server_t* out, const ssm_server_config* c);

/*
 * Queue one solve. K_host (P x Q doubles), M_host (P x N floats, ldm) and F_host
 * (Q x N floats, ldf) are the caller's and must stay valid until ssm_server_wait or
 * ssm_server_poll reports the request finished: K and M are read after admission, F
 * is written at the end. *ticket identifies the request. Returns SSM_EINVAL for bad
 * parameters and SSM_ENOMEM (nothing queued) when the request's footprint exceeds the
 * whole budget.
 */
ssm_status ssm_server_submit(ssm_server_t s, const ssm_params* p, const double* K_host,
                             const float* M_host, int64_t ldm, float* F_host, int64_t ldf,
                             int64_t* ticket);

/* As ssm_server_submit with M and F in device memory on the server's device (the result
 * stays on the device; no host copies). The reservation is the same. */
ssm_status ssm_server_submit_device(ssm_server_t s, const ssm_params* p, const double* K_host,
                                    const float* M_dev, int64_t ldm, float* F_dev,
                                    int64_t ldf, int64_t* ticket);

/* SSM_OK and *info filled (the solve's own status in info->status) once the request
 * has finished, after which the ticket is released; SSM_EPENDING while it has not;
 * SSM_EINVAL for an unknown ticket. */
ssm_status ssm_server_poll(ssm_server_t s, int64_t ticket, ssm_request_info* info);

/* As ssm_server_poll, blocking up to timeout_ms (< 0: no limit). */
ssm_status ssm_server_wait(ssm_server_t s, int64_t ticket, double timeout_ms,
                           ssm_request_info* info);

ssm_status ssm_server_stats_read(ssm_server_t s, ssm_server_stats* out);

/* Wait for every submitted request to finish, stop the workers and free every plan.
 * Tickets not yet collected become invalid. NULL is accepted. */
ssm_status ssm_server_destroy(ssm_server_t s);

/*
 * Self-test of failure detection (no counterpart in the paper): every mbarrier wait in
 * the solver's kernels is bounded and reports SSM_ETIMEOUT instead of hanging. This runs
 * one small kernel whose wait can never succeed (an mbarrier nobody arrives at), polled
 * `polls` times (1 .. 2^20) by the same wait routine, and returns the status the host
 * reads back: SSM_ETIMEOUT when the mechanism works. The device stays usable afterwards.
 * Synchronises `stream`.
 */
ssm_status ssm_selftest_wait_timeout(unsigned polls, void* stream);

/* Static description of a status code. */
const char* ssm_status_string(int status);

/* Last error message recorded on the calling thread ("" if none). */
const char* ssm_last_error(void);

/* Number of kernel launches the library has issued on this process (all plans). */
int64_t ssm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SSM_H */
