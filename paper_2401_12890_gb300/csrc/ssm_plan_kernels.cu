// Plan-stage kernels (Algorithm 2, steps 3-4): FP64 Gram matrix, parallel cyclic
// Jacobi eigendecomposition, the singular factors of Eq. 27, the weights of Eq. 28,
// the full-rank inverse of Eq. 26, and the data projections g_n (step 4).
//
// All of this runs once per plan (factors) or once per solve (projections) and is
// FP64 where the paper's conditioning needs it. GB300's FP64 rate is low, so the
// kernels spread FP64 work over every SM rather than one CTA.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "ssm_internal.cuh"

namespace ssm {
namespace {

// ---------------------------------------------------------------------------
// generic FP64 matrix product  C (m x n) = alpha * op(A) op(B) + diag_shift * I
//   op(A)[i][k] = transA ? A[k*lda + i] : A[i*lda + k]
//   op(B)[k][j] = transB ? B[j*ldb + k] : B[k*ldb + j]
// 32x32 output tile per block, k streamed through shared memory.
// ---------------------------------------------------------------------------
constexpr int TD = 32;

__global__ void __launch_bounds__(TD * 8) dgemm_naive(int m, int n, int kdim, const double* __restrict__ A,
                                             int64_t lda, int transA, const double* __restrict__ B,
                                             int64_t ldb, int transB, double* __restrict__ C,
                                             int64_t ldc, const double* __restrict__ colw,
                                             double diag) {
  // optional column weights on the k index: C = sum_k op(A)[i][k] * w[k] * op(B)[k][j]
  __shared__ double As[TD][TD + 1];
  __shared__ double Bs[TD][TD + 1];
  const int tx = threadIdx.x;          // 0..31  -> column j
  const int ty = threadIdx.y;          // 0..7   -> rows i = ty + 8*t
  const int i0 = blockIdx.y * TD, j0 = blockIdx.x * TD;
  double acc[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < kdim; k0 += TD) {
    for (int t = 0; t < 4; ++t) {
      int ii = ty + 8 * t;
      int i = i0 + ii, k = k0 + tx;
      double a = 0.0;
      if (i < m && k < kdim) a = transA ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k];
      if (colw && k < kdim) a *= colw[k];
      As[ii][tx] = a;
      int kk = k0 + ii, j = j0 + tx;
      double b = 0.0;
      if (kk < kdim && j < n) b = transB ? B[(int64_t)j * ldb + kk] : B[(int64_t)kk * ldb + j];
      Bs[ii][tx] = b;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TD; ++kk) {
      double b = Bs[kk][tx];
      for (int t = 0; t < 4; ++t) acc[t] = fma(As[ty + 8 * t][kk], b, acc[t]);
    }
    __syncthreads();
  }
  for (int t = 0; t < 4; ++t) {
    int i = i0 + ty + 8 * t, j = j0 + tx;
    if (i < m && j < n) C[(int64_t)i * ldc + j] = acc[t] + (i == j ? diag : 0.0);
  }
}

ssm_status dgemm(int m, int n, int k, const double* A, int64_t lda, bool tA, const double* B,
                 int64_t ldb, bool tB, double* C, int64_t ldc, cudaStream_t s,
                 const double* colw = nullptr, double diag = 0.0) {
  if (m <= 0 || n <= 0) return SSM_OK;
  dim3 block(TD, 8), grid((n + TD - 1) / TD, (m + TD - 1) / TD);
  dgemm_naive<<<grid, block, 0, s>>>(m, n, k, A, lda, tA ? 1 : 0, B, ldb, tB ? 1 : 0, C, ldc,
                                     colw, diag);
  SSM_LAUNCHED();
  return SSM_OK;
}

// ---------------------------------------------------------------------------
// parallel cyclic Jacobi (round-robin "circle" ordering)
// In round t of a sweep, the m/2 disjoint index pairs are
//   j = 0      : (m-1, t)
//   j = 1..m/2-1: ((t + j) mod (m-1), (t - j) mod (m-1))
// so every pair (p, q) is annihilated once per sweep. With n odd, m = n + 1 and the
// index n is a dummy (no rotation). Each round is one launch: block a owns rows
// (p_a, q_a) of A and of the eigenvector matrix E; it recomputes every pair's rotation
// from the previous A (double buffered), then writes its two rows of J^T A J and of E J.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void round_pair(int t, int j, int m, int& p, int& q) {
  int a, b;
  if (j == 0) {
    a = m - 1;
    b = t;
  } else {
    a = (t + j) % (m - 1);
    b = (t - j + (m - 1)) % (m - 1);
  }
  p = min(a, b);
  q = max(a, b);
}

// Golub & Van Loan's symmetric 2x2 Schur rotation: J = [[c, s], [-s, c]] on (p, q)
// makes (J^T A J)[p][q] = 0.
__device__ __forceinline__ void sym_schur(double app, double aqq, double apq, double& c,
                                          double& s) {
  if (fabs(apq) <= 1e-300 || fabs(apq) <= 1e-17 * sqrt(fabs(app * aqq))) {
    c = 1.0;
    s = 0.0;
    return;
  }
  double tau = (aqq - app) / (2.0 * apq);
  double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

__global__ void jacobi_round(const double* __restrict__ Ao, double* __restrict__ An,
                             double* __restrict__ E, int n, int m, int t) {
  extern __shared__ double sh[];
  double* rc = sh;                 // m/2 cosines
  double* rs = sh + m / 2;         // m/2 sines
  const int half = m / 2;
  for (int b = threadIdx.x; b < half; b += blockDim.x) {
    int p, q;
    round_pair(t, b, m, p, q);
    double c = 1.0, s = 0.0;
    if (q < n) sym_schur(Ao[(int64_t)p * n + p], Ao[(int64_t)q * n + q], Ao[(int64_t)p * n + q], c, s);
    rc[b] = c;
    rs[b] = s;
  }
  __syncthreads();
  const int a = blockIdx.x;
  int pa, qa;
  round_pair(t, a, m, pa, qa);
  const bool qa_ok = qa < n;
  const double ca = rc[a], sa = rs[a];
  for (int b = threadIdx.x; b < half; b += blockDim.x) {
    int pb, qb;
    round_pair(t, b, m, pb, qb);
    const bool qb_ok = qb < n;
    const double cb = rc[b], sb = rs[b];
    double x00 = Ao[(int64_t)pa * n + pb];
    double x01 = qb_ok ? Ao[(int64_t)pa * n + qb] : 0.0;
    double x10 = qa_ok ? Ao[(int64_t)qa * n + pb] : 0.0;
    double x11 = (qa_ok && qb_ok) ? Ao[(int64_t)qa * n + qb] : 0.0;
    // T = R_a^T X
    double t00 = ca * x00 - sa * x10, t01 = ca * x01 - sa * x11;
    double t10 = sa * x00 + ca * x10, t11 = sa * x01 + ca * x11;
    // Y = T R_b
    double y00 = cb * t00 - sb * t01, y01 = sb * t00 + cb * t01;
    double y10 = cb * t10 - sb * t11, y11 = sb * t10 + cb * t11;
    if (a == b && qa_ok) {
      y01 = 0.0;
      y10 = 0.0;
    }
    An[(int64_t)pa * n + pb] = y00;
    if (qb_ok) An[(int64_t)pa * n + qb] = y01;
    if (qa_ok) An[(int64_t)qa * n + pb] = y10;
    if (qa_ok && qb_ok) An[(int64_t)qa * n + qb] = y11;
    // E <- E J on rows pa, qa
    double e0 = E[(int64_t)pa * n + pb];
    double e1 = qb_ok ? E[(int64_t)pa * n + qb] : 0.0;
    E[(int64_t)pa * n + pb] = cb * e0 - sb * e1;
    if (qb_ok) E[(int64_t)pa * n + qb] = sb * e0 + cb * e1;
    if (qa_ok) {
      double f0 = E[(int64_t)qa * n + pb];
      double f1 = qb_ok ? E[(int64_t)qa * n + qb] : 0.0;
      E[(int64_t)qa * n + pb] = cb * f0 - sb * f1;
      if (qb_ok) E[(int64_t)qa * n + qb] = sb * f0 + cb * f1;
    }
  }
}

__global__ void eye_kernel(double* E, int n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)n * n) E[i] = (i / n == i % n) ? 1.0 : 0.0;
}

// off-diagonal and total squared Frobenius norms -> out[0], out[1]
__global__ void offdiag_norm(const double* __restrict__ A, int n, double* out) {
  double off = 0.0, tot = 0.0;
  for (int64_t i = threadIdx.x; i < (int64_t)n * n; i += blockDim.x) {
    double v = A[i];
    tot += v * v;
    if (i / n != i % n) off += v * v;
  }
  __shared__ double so[32], st[32];
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  if ((threadIdx.x & 31) == 0) {
    so[threadIdx.x >> 5] = off;
    st[threadIdx.x >> 5] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += so[w];
      b += st[w];
    }
    out[0] = a;
    out[1] = b;
  }
}

__global__ void diag_kernel(const double* A, int n, double* d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[(int64_t)i * n + i];
}

// gather eigenvector columns in descending order: out[row][i] = E[row][perm[i]], i < cnt
__global__ void gather_cols(const double* __restrict__ E, int rows, int ldE, const int* __restrict__ perm,
                            int cnt, double* __restrict__ out, int ldo) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * cnt) return;
  int row = (int)(idx / cnt), i = (int)(idx % cnt);
  out[(int64_t)row * ldo + i] = E[(int64_t)row * ldE + perm[i]];
}

// per-component constants and the FP32 low-rank basis
//   V32[q][i]  = v_i[q]   (i < r, zero for r <= i < R)
//   coefA[i]   = 1/(beta + sigma_i^2),  coefW[i] = sigma_i^2/(beta^2 + beta sigma_i^2)
__global__ void lowrank_basis(const double* __restrict__ Kt, int Q, int n, const double* __restrict__ sig,
                              int r, int R, int side, double beta, float* __restrict__ V32,
                              float* __restrict__ coefA, float* __restrict__ coefW, double sig_floor) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < (int64_t)Q * R) {
    int q = (int)(idx / R), i = (int)(idx % R);
    float v = 0.f;
    if (i < r) {
      double si = sig[i];
      double kv = Kt[(int64_t)q * n + i];
      // K K^T side: k_i = sigma_i v_i; K^T K side: Kt holds v_i itself
      if (side == 0) v = si > sig_floor ? (float)(kv / si) : 0.f;
      else v = (float)kv;
    }
    V32[idx] = v;
  }
  if (idx < R) {
    int i = (int)idx;
    if (i < r) {
      double s2 = sig[i] * sig[i];
      coefA[i] = (float)(1.0 / (beta + s2));
      coefW[i] = (float)(s2 / (beta * beta + beta * s2));
    } else {
      coefA[i] = 0.f;
      coefW[i] = 0.f;
    }
  }
}

// Gq[q][i] = Kt[q][i] / (sigma_i^2 + beta)   (h = M g = sum_i Gq_i c_i)
__global__ void gq_kernel(const double* __restrict__ Kt, int Q, int n, const double* __restrict__ sig,
                          double beta, float* __restrict__ Gq) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Q * n) return;
  int i = (int)(idx % n);
  Gq[idx] = (float)(Kt[idx] / (sig[i] * sig[i] + beta));
}

__global__ void to_f32(const double* __restrict__ X, int64_t count, float* __restrict__ Y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) Y[i] = (float)X[i];
}

// Eq. 26 assembled from the eigenpairs (exact Woodbury form, no division by sigma):
//   K K^T side: M = I/beta - sum_i k_i k_i^T / (beta (beta + sigma_i^2))
//   K^T K side: M = sum_i v_i v_i^T / (sigma_i^2 + beta)
// computed by dgemm with column weights w_i; then stored FP32 with row stride Qp.
__global__ void inv_weights(const double* __restrict__ sig, int n, int side, double beta,
                            double* __restrict__ w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s2 = sig[i] * sig[i];
  w[i] = side == 0 ? -1.0 / (beta * (beta + s2)) : 1.0 / (s2 + beta);
}

__global__ void store_square_f32(const double* __restrict__ X, int Q, float* __restrict__ Y, int Qp) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Q * Qp) return;
  int q = (int)(idx / Qp), k = (int)(idx % Qp);
  Y[idx] = k < Q ? (float)X[(int64_t)q * Q + k] : 0.f;
}

__global__ void split_bf16_kernel(const float* __restrict__ X, int rows, int cols, int64_t ldx,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                  int64_t ldo) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)rows * ldo) return;
  int64_t r = idx / ldo, c = idx % ldo;
  float x = c < cols ? X[r * ldx + c] : 0.f;
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi[idx] = h;
  lo[idx] = l;
}

// ---------------------------------------------------------------------------
// data projections (Algorithm 2, step 4):  out[i][n] = scale_i * sum_p Bp[p][i] m[p][n]
// FP64 accumulation; a block covers 128 voxels x 8 components; Bp staged in smem.
// ---------------------------------------------------------------------------
constexpr int PJ_VOX = 128, PJ_COMP = 8, PJ_PCH = 128;

__global__ void __launch_bounds__(PJ_VOX) project_kernel(const double* __restrict__ Bp, int P, int nB,
                                                 int ncomp, const float* __restrict__ M,
                                                 int64_t ldm, int64_t N,
                                                 const double* __restrict__ scale,
                                                 float* __restrict__ out, int64_t ldo) {
  __shared__ double bs[PJ_PCH][PJ_COMP];
  const int64_t nv = blockIdx.x * (int64_t)PJ_VOX + threadIdx.x;
  const int c0 = blockIdx.y * PJ_COMP;
  double acc[PJ_COMP];
#pragma unroll
  for (int j = 0; j < PJ_COMP; ++j) acc[j] = 0.0;
  for (int p0 = 0; p0 < P; p0 += PJ_PCH) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < PJ_PCH * PJ_COMP; idx += PJ_VOX) {
      int pp = idx / PJ_COMP, j = idx % PJ_COMP;
      int p = p0 + pp, c = c0 + j;
      bs[pp][j] = (p < P && c < ncomp) ? Bp[(int64_t)p * nB + c] : 0.0;
    }
    __syncthreads();
    if (nv < N) {
      int pend = min(PJ_PCH, P - p0);
      for (int pp = 0; pp < pend; ++pp) {
        double mv = (double)M[(int64_t)(p0 + pp) * ldm + nv];
#pragma unroll
        for (int j = 0; j < PJ_COMP; ++j) acc[j] = fma(bs[pp][j], mv, acc[j]);
      }
    }
  }
  if (nv < N) {
#pragma unroll
    for (int j = 0; j < PJ_COMP; ++j) {
      int c = c0 + j;
      if (c < ncomp) out[(int64_t)c * ldo + nv] = (float)(scale ? acc[j] * scale[c] : acc[j]);
    }
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// A = K K^T (side 0, P x P) or K^T K (side 1, Q x Q), FP64
ssm_status gram_fp64(const double* K, int P, int Q, int side, double* A, cudaStream_t s) {
  if (side == 0) return dgemm(P, P, Q, K, Q, false, K, Q, true, A, P, s);
  return dgemm(Q, Q, P, K, Q, true, K, Q, false, A, Q, s);
}

// Symmetric eigendecomposition A = E diag(evals) E^T by parallel cyclic Jacobi.
// A (n x n) is overwritten; scratch holds n*n + 2 doubles. E is n x n (column j =
// eigenvector j, in Jacobi's order; evals in the same order).
ssm_status jacobi_eigen(double* A, int n, double* E, double* scratch, std::vector<double>& evals,
                        cudaStream_t s) {
  evals.assign(n, 0.0);
  if (n == 1) {
    double a;
    SSM_CUDA(cudaMemcpyAsync(&a, A, sizeof(double), cudaMemcpyDeviceToHost, s));
    double one = 1.0;
    SSM_CUDA(cudaMemcpyAsync(E, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    SSM_CUDA(cudaStreamSynchronize(s));
    evals[0] = a;
    return SSM_OK;
  }
  const int m = n + (n & 1);
  const int half = m / 2;
  double* B = scratch;
  double* nrm = scratch + (int64_t)n * n;
  eye_kernel<<<nblk((int64_t)n * n, 256), 256, 0, s>>>(E, n);
  SSM_LAUNCHED();
  const int threads = std::min(256, ((half + 31) / 32) * 32);
  const size_t shm = sizeof(double) * m;
  double* cur = A;
  double* nxt = B;
  double hn[2];
  const int max_sweeps = 40;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int t = 0; t < m - 1; ++t) {
      jacobi_round<<<half, threads, shm, s>>>(cur, nxt, E, n, m, t);
      SSM_LAUNCHED();
      std::swap(cur, nxt);
    }
    offdiag_norm<<<1, 1024, 0, s>>>(cur, n, nrm);
    SSM_LAUNCHED();
    SSM_CUDA(cudaMemcpyAsync(hn, nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SSM_CUDA(cudaStreamSynchronize(s));
    if (!(hn[0] == hn[0])) {
      set_error("Jacobi eigensolver produced NaN");
      return SSM_ENAN;
    }
    if (hn[0] <= 1e-30 * hn[1] || hn[1] == 0.0) break;
  }
  double* dd = nxt;  // the idle half of the double buffer holds the diagonal
  diag_kernel<<<nblk(n, 256), 256, 0, s>>>(cur, n, dd);
  SSM_LAUNCHED();
  SSM_CUDA(cudaMemcpyAsync(evals.data(), dd, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  SSM_CUDA(cudaStreamSynchronize(s));
  return SSM_OK;
}

// Factors of Eq. 27 from the Gram eigenvectors E (n x n, Jacobi order), see header.
ssm_status factors_fp64(ssm_plan_s* pl, const double* E, cudaStream_t s) {
  const int P = pl->P, Q = pl->Q, n = pl->n;
  int* dperm = nullptr;
  SSM_CUDA(cudaMallocAsync(&dperm, sizeof(int) * n, s));
  SSM_CUDA(cudaMemcpyAsync(dperm, pl->perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  std::vector<double> sig(pl->sigma);
  SSM_CUDA(cudaMemcpyAsync(pl->sig64, sig.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  if (pl->gram_side == 0) {
    // E columns are u_i (P-vectors): Bp = U, Kt = K^T U (k_i = sigma_i v_i)
    gather_cols<<<nblk((int64_t)P * n, 256), 256, 0, s>>>(E, P, n, dperm, n, pl->Bp64, n);
    SSM_LAUNCHED();
    SSM_TRY(dgemm(Q, n, P, pl->K64, Q, true, pl->Bp64, n, false, pl->Kt64, n, s));
  } else {
    // E columns are v_i (Q-vectors): Kt = V, Bp = K V (= sigma_i u_i)
    gather_cols<<<nblk((int64_t)Q * n, 256), 256, 0, s>>>(E, Q, n, dperm, n, pl->Kt64, n);
    SSM_LAUNCHED();
    SSM_TRY(dgemm(P, n, Q, pl->K64, Q, false, pl->Kt64, n, false, pl->Bp64, n, s));
  }
  SSM_CUDA(cudaFreeAsync(dperm, s));
  // S_i = alpha_i c_i with c = Bp^T m: alpha = sigma (K K^T side) or 1 (K^T K side)
  std::vector<double> alpha(n);
  for (int i = 0; i < n; ++i) alpha[i] = pl->gram_side == 0 ? pl->sigma[i] : 1.0;
  SSM_CUDA(cudaMemcpyAsync(pl->alpha64, alpha.data(), sizeof(double) * n,
                           cudaMemcpyHostToDevice, s));
  SSM_CUDA(cudaStreamSynchronize(s));   // `alpha` is a host temporary
  SSM_TRY(beta_weights(pl, s));
  // dictionaries for the objective: K (FP32) and K_r = Bp_r Kt_r^T
  to_f32<<<nblk((int64_t)P * Q, 256), 256, 0, s>>>(pl->K64, (int64_t)P * Q, pl->K32);
  SSM_LAUNCHED();
  double* Kr64 = nullptr;
  SSM_CUDA(cudaMallocAsync(&Kr64, sizeof(double) * P * Q, s));
  SSM_TRY(dgemm(P, Q, pl->r, pl->Bp64, n, false, pl->Kt64, n, true, Kr64, Q, s));
  to_f32<<<nblk((int64_t)P * Q, 256), 256, 0, s>>>(Kr64, (int64_t)P * Q, pl->Kr32);
  SSM_LAUNCHED();
  SSM_CUDA(cudaFreeAsync(Kr64, s));
  return SSM_OK;
}

// The beta-dependent part of the plan (the factors above do not depend on beta):
// low-rank V_r and the weights of Eq. 28, or the dense form's h-map Gq; the dense
// inverse itself is form_dense_inverse.
ssm_status beta_weights(ssm_plan_s* pl, cudaStream_t s) {
  const int Q = pl->Q, n = pl->n;
  const double floor = pl->sigma1 * 1e-15;
  if (pl->p.form == SSM_FORM_LOWRANK) {
    lowrank_basis<<<nblk((int64_t)Q * pl->R, 256), 256, 0, s>>>(
        pl->Kt64, Q, n, pl->sig64, pl->r, pl->R, pl->gram_side, pl->p.beta, pl->V32, pl->coefA,
        pl->coefW, floor);
    SSM_LAUNCHED();
    if (pl->V1h) SSM_TRY(lrtc_split_basis(pl, s));
  } else {
    gq_kernel<<<nblk((int64_t)Q * n, 256), 256, 0, s>>>(pl->Kt64, Q, n, pl->sig64, pl->p.beta,
                                                        pl->Gq32);
    SSM_LAUNCHED();
  }
  return SSM_OK;
}

ssm_status form_dense_inverse(ssm_plan_s* pl, cudaStream_t s) {
  const int Q = pl->Q, n = pl->n;
  double* w = nullptr;
  double* M64 = nullptr;
  SSM_CUDA(cudaMallocAsync(&w, sizeof(double) * n, s));
  SSM_CUDA(cudaMallocAsync(&M64, sizeof(double) * (int64_t)Q * Q, s));
  inv_weights<<<nblk(n, 256), 256, 0, s>>>(pl->sig64, n, pl->gram_side, pl->p.beta, w);
  SSM_LAUNCHED();
  const double diag = pl->gram_side == 0 ? 1.0 / pl->p.beta : 0.0;
  SSM_TRY(dgemm(Q, Q, n, pl->Kt64, n, false, pl->Kt64, n, true, M64, Q, s, w, diag));
  store_square_f32<<<nblk((int64_t)Q * pl->Qp, 256), 256, 0, s>>>(M64, Q, pl->Mq32, pl->Qp);
  SSM_LAUNCHED();
  if (pl->Mhi) {
    SSM_TRY(split_bf16(pl->Mq32, Q, pl->Qp, pl->Qp, pl->Mhi, pl->Mlo, pl->Qp, s));
  }
  SSM_CUDA(cudaFreeAsync(M64, s));
  SSM_CUDA(cudaFreeAsync(w, s));
  return SSM_OK;
}

ssm_status split_bf16(const float* X, int rows, int cols, int64_t ldx, __nv_bfloat16* hi,
                      __nv_bfloat16* lo, int64_t ldo, cudaStream_t s) {
  split_bf16_kernel<<<nblk((int64_t)rows * ldo, 256), 256, 0, s>>>(X, rows, cols, ldx, hi, lo, ldo);
  SSM_LAUNCHED();
  return SSM_OK;
}

// c (ncomp x ld, FP32) = scale .* (Bp^T m), FP64 accumulation. The low-rank form
// writes S (scale = alpha), the dense form writes the raw coefficients.
ssm_status project_data(const ssm_plan_s* pl, const float* M, int64_t ldm, int ncomp,
                        cudaStream_t s) {
  const bool lowrank = pl->p.form == SSM_FORM_LOWRANK;
  float* out = lowrank ? pl->S : pl->C32;
  const double* scale = lowrank ? pl->alpha64 : nullptr;
  dim3 grid(nblk(pl->g.N, PJ_VOX), (unsigned)((ncomp + PJ_COMP - 1) / PJ_COMP));
  project_kernel<<<grid, PJ_VOX, 0, s>>>(pl->Bp64, pl->P, pl->n, ncomp, M, ldm, pl->g.N, scale,
                                         out, pl->g.ld);
  SSM_LAUNCHED();
  return SSM_OK;
}

}  // namespace ssm
