// FP64 steps of the IBMI hot path: blocked Cholesky of the diagonal blocks,
// the triangular solves that form A_I^{-1} and W = A_I^{-1} A_{I,I^c}
// (eq. IBMI invariants), the two sweep products (a3, a4), the residual
// ||I - A H||_F and the FP64 Newton-Schulz step (eq. newton).
#include <math.h>

#include "gemm_f64.cuh"
#include "plan.cuh"

namespace ibmi {

// ------------------------------------------------------------ Cholesky ----

// Factors the jb x jb diagonal tile T (lower part, row-major, ld) in place:
// T = L L^T, and writes L^{-1} (jb x jb, ld jb) to linv.  One CTA of 32 x 32
// threads.  A non-positive or non-finite pivot records NOT_SPD (set `blk`,
// global pivot `row0 + j`) and is replaced by 1 so the factorisation finishes.
__global__ void __launch_bounds__(1024) k_potrf_tile(double* T, int64_t ld, int jb, double* linv,
                                                     DevStatus* st, int blk, int64_t row0) {
  __shared__ double L[CHOL_NB][CHOL_NB + 1];
  __shared__ double X[CHOL_NB][CHOL_NB + 1];
  const int c = threadIdx.x, r = threadIdx.y;
  L[r][c] = (r < jb && c <= r) ? T[r * ld + c] : 0.0;
  __syncthreads();
  for (int j = 0; j < jb; ++j) {
    if (r == j && c == j) {
      double d = L[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (atomicCAS(&st->code, 0, (int)IBMI_ERR_NOT_SPD) == 0) {
          st->block = blk;
          st->pivot = row0 + j;
        }
        d = 1.0;
      }
      L[j][j] = sqrt(d);
    }
    __syncthreads();
    if (c == j && r > j && r < jb) L[r][j] /= L[j][j];
    __syncthreads();
    if (c > j && r >= c && r < jb) L[r][c] -= L[r][j] * L[c][j];
    __syncthreads();
  }
  // X = L^{-1} by forward substitution, one column per thread of warp 0..
  if (r == 0 && c < jb) {
    for (int i = 0; i < jb; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int t = c; t < i; ++t) s -= L[i][t] * X[t][c];
      X[i][c] = (i >= c) ? s / L[i][i] : 0.0;
    }
  }
  __syncthreads();
  if (r < jb && c < jb) {
    T[r * ld + c] = (c <= r) ? L[r][c] : 0.0;
    linv[r * jb + c] = X[r][c];
  }
}

// Right-hand side of the two solves: B = A[I, :] with B[:, I] = identity, so
// that L^{-T} L^{-1} B = [A_I^{-1} on columns I | A_I^{-1} A_{I,I^c} elsewhere].
__global__ void k_build_rhs(const double* A, int64_t lda, int64_t lo, int64_t m, int64_t p,
                            double* W) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * p) return;
  int64_t i = idx / p, c = idx - i * p;
  W[idx] = (c >= lo && c < lo + m) ? ((c - lo == i) ? 1.0 : 0.0) : A[(lo + i) * lda + c];
}

// A_I^{-1} = W[:, I]; then W[:, I] = 0 (the zero columns keep sweep tiles that
// straddle I harmless and let W be addressed with physical column indices).
__global__ void k_extract_ainv(double* W, int64_t lo, int64_t m, int64_t p, double* ainv) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  int64_t i = idx / m, j = idx - i * m;
  // symmetrise: A_I^{-1} is symmetric in exact arithmetic
  double v = 0.5 * (W[i * p + lo + j] + W[j * p + lo + i]);
  ainv[idx] = v;
}

__global__ void k_zero_cols(double* W, int64_t lo, int64_t m, int64_t p) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  int64_t i = idx / m, j = idx - i * m;
  W[i * p + lo + j] = 0.0;
}

__global__ void k_copy_block(const double* A, int64_t lda, int64_t lo, int64_t m, double* L) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  int64_t i = idx / m, j = idx - i * m;
  L[idx] = A[(lo + i) * lda + lo + j];
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

ibmi_status invariants_f64(ibmi_plan_s* P, int k, const double* A, int64_t lda, cudaStream_t st) {
  const int64_t p = P->d.p, lo = P->lo[k], m = P->hi[k] - P->lo[k];
  double* Lw = P->lwork;   // m x m, ld m
  double* W = P->w[k];     // m x p
  ProfScope ps(IBMI_K_INVARIANTS, st, m * m * m / 3.0 + 2.0 * m * m * p);
  note_launch();
  k_copy_block<<<nblk(m * m), 256, 0, st>>>(A, lda, lo, m, Lw);
  IBMI_CUDA_TRY(cudaGetLastError());
  const GapMap id{0, 0};
  // blocked right-looking Cholesky, nb = 32
  for (int64_t j0 = 0; j0 < m; j0 += CHOL_NB) {
    const int jb = (int)std::min<int64_t>(CHOL_NB, m - j0);
    double* Ljj = Lw + j0 * m + j0;
    double* Li = P->linv + j0 * CHOL_NB;  // jb x jb, ld jb
    note_launch();
    k_potrf_tile<<<1, dim3(32, 32), 0, st>>>(Ljj, m, jb, Li, P->dstatus, k, lo + j0);
    IBMI_CUDA_TRY(cudaGetLastError());
    const int64_t rest = m - j0 - jb;
    if (rest <= 0) break;
    // panel: L[j0+jb:, j0:j0+jb] = A[...] L_jj^{-T}   (in place; one CTA column owns each row)
    {
      F64Operands op{Lw + (j0 + jb) * m + j0, m, id, id, Li, jb, id, id, rest, jb, jb};
      IBMI_CUDA_TRY((launch_gemm_f64<true, false>(op, EpiStore{Lw + (j0 + jb) * m + j0, m, 1.0, 0.0}, st)));
    }
    // trailing: A22 -= L21 L21^T
    {
      F64Operands op{Lw + (j0 + jb) * m + j0, m, id, id, Lw + (j0 + jb) * m + j0, m, id, id, rest, rest, jb};
      IBMI_CUDA_TRY((launch_gemm_f64<true, false>(
          op, EpiStore{Lw + (j0 + jb) * m + (j0 + jb), m, -1.0, 1.0}, st)));
    }
  }
  // B = [A_{I,:} with identity on I];  W <- L^{-T} L^{-1} B  (forward, then backward)
  note_launch();
  k_build_rhs<<<nblk(m * p), 256, 0, st>>>(A, lda, lo, m, p, W);
  IBMI_CUDA_TRY(cudaGetLastError());
  for (int64_t j0 = 0; j0 < m; j0 += CHOL_NB) {
    const int jb = (int)std::min<int64_t>(CHOL_NB, m - j0);
    const double* Li = P->linv + j0 * CHOL_NB;
    {  // tmp = L_jj^{-1} W[j0:j0+jb, :]
      F64Operands op{Li, jb, id, id, W + j0 * p, p, id, id, jb, p, jb};
      IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStore{P->tmp, p, 1.0, 0.0}, st)));
    }
    IBMI_CUDA_TRY(cudaMemcpyAsync(W + j0 * p, P->tmp, sizeof(double) * jb * p, cudaMemcpyDeviceToDevice, st));
    const int64_t rest = m - j0 - jb;
    if (rest > 0) {  // W[j0+jb:, :] -= L[j0+jb:, j0:j0+jb] tmp
      F64Operands op{Lw + (j0 + jb) * m + j0, m, id, id, P->tmp, p, id, id, rest, p, jb};
      IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStore{W + (j0 + jb) * p, p, -1.0, 1.0}, st)));
    }
  }
  const int64_t nbk = (m + CHOL_NB - 1) / CHOL_NB;
  for (int64_t b = nbk - 1; b >= 0; --b) {
    const int64_t j0 = b * CHOL_NB;
    const int jb = (int)std::min<int64_t>(CHOL_NB, m - j0);
    const double* Li = P->linv + j0 * CHOL_NB;
    {  // tmp = L_jj^{-T} W[j0:j0+jb, :]   (A operand column-major view of L_jj^{-1})
      F64Operands op{Li, jb, id, id, W + j0 * p, p, id, id, jb, p, jb};
      IBMI_CUDA_TRY((launch_gemm_f64<false, true>(op, EpiStore{P->tmp, p, 1.0, 0.0}, st)));
    }
    IBMI_CUDA_TRY(cudaMemcpyAsync(W + j0 * p, P->tmp, sizeof(double) * jb * p, cudaMemcpyDeviceToDevice, st));
    if (j0 > 0) {  // W[0:j0, :] -= L[j0:j0+jb, 0:j0]^T tmp
      F64Operands op{Lw + j0 * m, m, id, id, P->tmp, p, id, id, j0, p, jb};
      IBMI_CUDA_TRY((launch_gemm_f64<false, true>(op, EpiStore{W, p, -1.0, 1.0}, st)));
    }
  }
  note_launch();
  k_extract_ainv<<<nblk(m * m), 256, 0, st>>>(W, lo, m, p, P->ainv[k]);
  IBMI_CUDA_TRY(cudaGetLastError());
  note_launch();
  k_zero_cols<<<nblk(m * m), 256, 0, st>>>(W, lo, m, p);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

// --------------------------------------------------------------- sweep ----

// H[lo+i, lo+j] = (S[i, j] + S[j, i]) / 2
__global__ void k_symmetrize_into(const double* S, int64_t m, double* H, int64_t ldh, int64_t lo) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  int64_t i = idx / m, j = idx - i * m;
  H[(lo + i) * ldh + lo + j] = 0.5 * (S[i * m + j] + S[j * m + i]);
}

ibmi_status sweep_step_f64(ibmi_plan_s* P, int k, double* H, int64_t ldh, cudaStream_t st) {
  const int64_t p = P->d.p, lo = P->lo[k], m = P->hi[k] - P->lo[k], n = p - m;
  if (n == 0) {  // K = 1: H = A^{-1} directly
    note_launch();
    k_symmetrize_into<<<nblk(m * m), 256, 0, st>>>(P->ainv[k], m, H, ldh, lo);
    IBMI_CUDA_TRY(cudaGetLastError());
    return IBMI_OK;
  }
  const GapMap gap{lo, m}, id{0, 0};
  // a3: X = -W T with T = H[I^c, I^c]; scatter X to H[I, I^c] and X^T to H[I^c, I]
  {
    ProfScope ps(IBMI_K_SWEEP_X, st, 2.0 * m * n * n);
    F64Operands op{P->w[k], p, id, gap, H, ldh, gap, gap, m, n, n};
    IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiSweepX{H, ldh, lo, gap}, st)));
  }
  // a4: S = A_I^{-1} - X W^T with X = H[I, I^c]
  {
    ProfScope ps(IBMI_K_SWEEP_S, st, 2.0 * m * m * n);
    F64Operands op{H + lo * ldh, ldh, id, gap, P->w[k], p, gap, id, m, m, n};
    IBMI_CUDA_TRY((launch_gemm_f64<true, false>(op, EpiSweepS{P->ainv[k], P->S, m}, st)));
  }
  note_launch();
  k_symmetrize_into<<<nblk(m * m), 256, 0, st>>>(P->S, m, H, ldh, lo);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

// ------------------------------------------------------------ residual ----

// Deterministic single-CTA sum of the partials; writes sqrt(sum)/sqrt(p) to
// out[0] and the raw sum to out[1].
__global__ void k_finish_residual(const double* partials, int64_t n, int64_t p, double* out) {
  __shared__ double red[1024 / 32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    out[0] = sqrt(t) / sqrt((double)p);
    out[1] = t;
  }
}

ibmi_status residual_f64_dev(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                             double* partials, int64_t n_partials, double* dout, cudaStream_t st) {
  const GapMap id{0, 0};
  if (gemm_f64_ctas(p, p) > n_partials) return IBMI_ERR_INVALID_ARG;
  ProfScope ps(IBMI_K_RESIDUAL, st, 2.0 * (double)p * p * p);
  F64Operands op{A, lda, id, id, H, ldh, id, id, p, p, p};
  IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiResidual{partials, 0.0}, st)));
  note_launch();
  k_finish_residual<<<1, 1024, 0, st>>>(partials, gemm_f64_ctas(p, p), p, dout);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

// ------------------------------------------------------- Newton-Schulz ----

__global__ void k_symmetrize_full(const double* Xn, int64_t p, double* X, int64_t ldx) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * p) return;
  int64_t i = idx / p, j = idx - i * p;
  X[i * ldx + j] = 0.5 * (Xn[i * p + j] + Xn[j * p + i]);
}

ibmi_status ns_step_f64(ibmi_plan_s* P, const double* A, int64_t lda, double* X, int64_t ldx,
                        cudaStream_t st) {
  const int64_t p = P->d.p;
  const GapMap id{0, 0};
  ProfScope ps(IBMI_K_NS, st, 4.0 * (double)p * p * p);
  {  // R = I - A X
    F64Operands op{A, lda, id, id, X, ldx, id, id, p, p, p};
    IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiIdentityMinus{P->nsR, p}, st)));
  }
  {  // Xn = X + X R
    F64Operands op{X, ldx, id, id, P->nsR, p, id, id, p, p, p};
    IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiAddTo{X, ldx, P->nsX, p}, st)));
  }
  note_launch();
  k_symmetrize_full<<<nblk(p * p), 256, 0, st>>>(P->nsX, p, X, ldx);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

__global__ void k_set_identity(double* H, int64_t ldh, int64_t p) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * p) return;
  int64_t i = idx / p, j = idx - i * p;
  H[i * ldh + j] = (i == j) ? 1.0 : 0.0;
}

ibmi_status set_identity(double* H, int64_t ldh, int64_t p, cudaStream_t st) {
  note_launch();
  k_set_identity<<<nblk(p * p), 256, 0, st>>>(H, ldh, p);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

}  // namespace ibmi
