// FP64 steps of the IBMI hot path: blocked Cholesky of the diagonal blocks,
// the triangular solves that form A_I^{-1} and W = A_I^{-1} A_{I,I^c}
// (eq. IBMI invariants), the two sweep products (a3, a4), the residual
// ||I - A H||_F and the FP64 Newton-Schulz step (eq. newton).
#include <math.h>

#include "gemm_f64.cuh"
#include "plan.cuh"
#include "refine.cuh"

namespace ibmi {

// ------------------------------------------------------------ Cholesky ----
//
// All K diagonal blocks are factorised together: block k is embedded in an
// mmax x mmax matrix [[A_{I_k}, 0], [0, I]] (its Cholesky factor and inverse
// are [[L, 0], [0, I]] and [[A_{I_k}^{-1}, 0], [0, I]]), so every launch below
// works on the whole batch with blockIdx.z = k.

// Factors the jb x jb diagonal tile T (lower part, row-major, ld) in place:
// T = L L^T, and writes L^{-1} (jb x jb, ld jb) to linv.  One CTA of 32 x 32
// threads per block of the batch.  FP64 latency is what bounds this kernel on
// GB300, so each pivot takes one rsqrt (sqrt(d) = d rsqrt(d); the column is
// scaled by rsqrt(d)), computed by the thread that finishes the pivot's update
// in the previous step, which leaves two barriers per step.  L^{-1} is built
// column by column, one warp per column (lane = row), by right-looking
// substitution.  A non-positive or non-finite pivot records NOT_SPD (set z,
// global pivot lo_z + row0 + j) and is replaced by 1 so the factorisation
// finishes.
__global__ void __launch_bounds__(1024) k_potrf_tile(double* T, int64_t ld, int64_t zT, int jb, double* linv,
                                                     int64_t zL, DevStatus* st, const int64_t* dlo, int64_t row0,
                                                     int status_per_block) {
  if (status_per_block) st += blockIdx.z;   // one status word per block (batched groups)
  __shared__ double L[CHOL_NB][CHOL_NB + 1];
  __shared__ double X[CHOL_NB][CHOL_NB + 1];
  __shared__ double rd[CHOL_NB];   // rsqrt of the pivots
  const int z = blockIdx.z;
  T += z * zT;
  linv += z * zL;
  const int c = threadIdx.x, r = threadIdx.y;
  auto pivot = [&](double d, int j) -> double {   // returns sqrt(d), sets rd[j]
    if (!(d > 0.0) || !isfinite(d)) {
      if (atomicCAS(&st->code, 0, (int)IBMI_ERR_NOT_SPD) == 0) {
        st->block = z;
        st->pivot = dlo[z] + row0 + j;
      }
      d = 1.0;
    }
    const double q = rsqrt(d);
    rd[j] = q;
    return d * q;
  };
  L[r][c] = (r < jb && c <= r) ? T[r * ld + c] : 0.0;
  if (r == 0 && c == 0) L[0][0] = pivot(T[0], 0);
  __syncthreads();
  for (int j = 0; j < jb; ++j) {
    if (c == j && r > j && r < jb) L[r][j] *= rd[j];
    __syncthreads();
    if (c > j && r >= c && r < jb) {
      double v = L[r][c] - L[r][j] * L[c][j];
      if (r == j + 1 && c == j + 1) v = pivot(v, j + 1);
      L[r][c] = v;
    }
    __syncthreads();
  }
  {  // X = L^{-1}: warp w owns column w; x_t = acc_t rd[t] once rows < t are done
    const int w = r, i = c;
    double acc = (i == w) ? 1.0 : 0.0, xi = 0.0;
    for (int t = w; t < jb; ++t) {
      const double xt = __shfl_sync(0xffffffffu, acc * rd[t], t);
      if (i == t) xi = xt;
      if (i > t) acc -= L[i][t] * xt;
    }
    if (i < jb && w < jb) X[i][w] = (i >= w) ? xi : 0.0;
  }
  __syncthreads();
  if (r < jb && c < jb) {
    T[r * ld + c] = (c <= r) ? L[r][c] : 0.0;
    linv[r * jb + c] = X[r][c];
  }
}

// Lw[z] = [[A[I_z, I_z], 0], [0, I]]  (mmax x mmax)
// doffA (optional): element offset of block z's matrix within A (blocks of
// several matrices stacked in one batch).
__global__ void k_bat_copy_block(const double* A, int64_t lda, const int64_t* dlo, const int64_t* dm, int64_t mmax,
                                 double* Lw, const int64_t* doffA) {
  const int z = blockIdx.z;
  if (doffA) A += doffA[z];
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mmax * mmax) return;
  int64_t i = idx / mmax, j = idx - i * mmax;
  const int64_t lo = dlo[z], m = dm[z];
  Lw[z * mmax * mmax + idx] = (i < m && j < m) ? A[(lo + i) * lda + lo + j] : (i == j ? 1.0 : 0.0);
}

// Right-hand sides R[z] (mmax x ncols).  full_w: rows i < m_z hold A[I_z, :]
// with the identity on the columns of I_z (so the solution is A_I^{-1} on the
// columns of I and A_I^{-1} A_{I,I^c} elsewhere); otherwise R[z] = identity.
__global__ void k_bat_rhs(const double* A, int64_t lda, const int64_t* dlo, const int64_t* dm, int64_t mmax,
                          int64_t ncols, int full_w, double* R, const int64_t* doffA) {
  const int z = blockIdx.z;
  if (doffA) A += doffA[z];
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= mmax * ncols) return;
  int64_t i = idx / ncols, c = idx - i * ncols;
  const int64_t lo = dlo[z], m = dm[z];
  double v;
  if (full_w) {
    if (i >= m) v = 0.0;
    else if (c >= lo && c < lo + m) v = (c - lo == i) ? 1.0 : 0.0;
    else v = A[(lo + i) * lda + c];
  } else {
    v = (i == c) ? 1.0 : 0.0;
  }
  R[z * mmax * ncols + idx] = v;
}

// Scatter of the solutions: A_I^{-1} (symmetrised) and, for full_w, W with
// zero columns on I.  Offsets of the per-set outputs come from doff_*.
// lower_only: R holds A_I^{-1} on and below the diagonal only; the upper
// triangle is mirrored from it.
__global__ void k_bat_extract(const double* R, const int64_t* dlo, const int64_t* dm, int64_t mmax, int64_t ncols,
                              int full_w, int lower_only, double* base, const int64_t* doff_ainv,
                              const int64_t* doff_w, int64_t p) {
  const int z = blockIdx.z;
  const int64_t lo = dlo[z], m = dm[z];
  const double* Rz = R + z * mmax * ncols;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < m * m) {
    int64_t i = idx / m, j = idx - i * m;
    const int64_t cj = full_w ? lo + j : j, ci = full_w ? lo + i : i;
    if (lower_only)
      base[doff_ainv[z] + idx] = i >= j ? Rz[i * ncols + j] : Rz[j * ncols + i];
    else
      base[doff_ainv[z] + idx] = 0.5 * (Rz[i * ncols + cj] + Rz[j * ncols + ci]);
  }
  if (full_w && idx < m * p) {
    int64_t i = idx / p, c = idx - i * p;
    base[doff_w[z] + idx] = (c >= lo && c < lo + m) ? 0.0 : Rz[i * ncols + c];
  }
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

ibmi_status invariants_all(ibmi_plan_s* P, const double* A, int64_t lda, bool full_w, cudaStream_t st,
                           bool leave_y, RefineState* tc) {
  const int64_t p = P->d.p, mmax = P->mmax;
  const int K = (int)P->lo.size();
  const int64_t ncols = full_w ? p : mmax;
  const int64_t zL = mmax * mmax, zLi = mmax * CHOL_NB, zR = mmax * ncols;
  double* Lw = P->bat_L;
  double* R = P->bat_R;
  double flops = 0.0;
  for (int k = 0; k < K; ++k) {   // Cholesky m^3/3; then the two solves for W (2 m^2 p), or L^{-1}
    const double m = (double)(P->hi[k] - P->lo[k]);   // (m^3/3) and, unless left to the caller, Y^T Y (m^3/3)
    flops += m * m * m / 3.0 + (full_w ? 2.0 * m * m * (double)p : m * m * m / 3.0 * (leave_y ? 1.0 : 2.0));
  }
  ProfScope ps(IBMI_K_INVARIANTS, st, flops);
  const GapMap id{0, 0};
  auto bat = [&](F64Operands op, int64_t za, int64_t zb) {
    op.zA = za;
    op.zB = zb;
    op.batch = K;
    op.tile_batch = P->tile_batch;
    return op;
  };
  note_launch();
  k_bat_copy_block<<<dim3(nblk(mmax * mmax), 1, K), 256, 0, st>>>(A, lda, P->dlo, P->dm, mmax, Lw, P->doffA);
  IBMI_CUDA_TRY(cudaGetLastError());
  // blocked right-looking Cholesky, nb = 32, by block columns [J0, J1): the
  // whole matrix as one block column, or (tc, large blocks) columns of
  // kTcCholPanel whose own steps run in FP64 while the update of everything
  // right of them, C -= L21 L21^T with K = J1 - J0, runs on the tensor cores
  const bool tc_chol = tc != nullptr && mmax >= kTcCholMinOrder;
  const int64_t ncol = tc_chol ? kTcCholPanel : mmax;
  for (int64_t J0 = 0; J0 < mmax; J0 += ncol) {
    const int64_t J1 = std::min(mmax, J0 + ncol);
    for (int64_t j0 = J0; j0 < J1; j0 += CHOL_NB) {
      const int jb = (int)std::min<int64_t>(CHOL_NB, J1 - j0);
      double* Li = P->bat_linv + j0 * CHOL_NB;
      note_launch();
      k_potrf_tile<<<dim3(1, 1, K), dim3(32, 32), 0, st>>>(Lw + j0 * mmax + j0, mmax, zL, jb, Li, zLi, P->dstatus,
                                                            P->dlo, j0, P->doffA ? 1 : 0);
      IBMI_CUDA_TRY(cudaGetLastError());
      const int64_t rest = mmax - j0 - jb;
      if (rest <= 0) break;
      double* panel = Lw + (j0 + jb) * mmax + j0;
      {  // panel = panel L_jj^{-T} (in place: one CTA column owns each row)
        F64Operands op = bat(F64Operands{panel, mmax, id, id, Li, jb, id, id, rest, jb, jb}, zL, zLi);
        IBMI_CUDA_TRY((launch_gemm_f64<true, false>(op, EpiStore{panel, mmax, 1.0, 0.0, zL}, st)));
      }
      // trailing -= panel panel^T on the columns up to J1, on the tiles that
      // touch the lower triangle (the factorisation and the solves read
      // nothing above the diagonal)
      const int64_t ncols = J1 - j0 - jb;
      if (ncols > 0) {
        F64Operands op = bat(F64Operands{panel, mmax, id, id, panel, mmax, id, id, rest, ncols, jb}, zL, zL);
        op.lower_tiles = true;
        IBMI_CUDA_TRY((launch_gemm_f64<true, false>(op, EpiStore{panel + jb, mmax, -1.0, 1.0, zL}, st)));
      }
    }
    if (J1 < mmax) {   // all K blocks at once
      IBMI_TRY(refine_syrk_sub(tc, Lw + J1 * mmax + J0, mmax, zL, mmax - J1, J1 - J0, Lw + J1 * mmax + J1, mmax, zL,
                               K, st));
      ps.flops -= (double)K * (mmax - J1) * (mmax - J1) * (J1 - J0);   // counted by its own (tensor) class
    }
  }
  // R <- L^{-T} L^{-1} R (full_w); A_I^{-1} = L^{-T} L^{-1} otherwise
  note_launch();
  k_bat_rhs<<<dim3(nblk(mmax * ncols), 1, K), 256, 0, st>>>(A, lda, P->dlo, P->dm, mmax, ncols, full_w ? 1 : 0, R,
                                                           P->doffA);
  IBMI_CUDA_TRY(cudaGetLastError());
  // Both triangular solves work in place: the diagonal-block product reads
  // rows j0..j0+jb of one column tile and writes the same tile (one CTA owns
  // all jb rows of it, jb <= 32 <= the tile height, and reads its whole K
  // before writing).
  static_assert(CHOL_NB <= 32, "in-place diagonal-block products need jb within one tile row");
  // By block rows [J0, J1) as the factorisation's block columns: with tc
  // (A_I^{-1} only, large blocks) the update of the rows below a block row,
  // R[J1:, :J1] -= L[J1:, J0:J1] R[J0:J1, :J1], runs on the tensor cores.
  const bool tc_fwd = tc_chol && !full_w;
  const int64_t nrow = tc_fwd ? kTcCholPanel : mmax;
  for (int64_t J0 = 0; J0 < mmax; J0 += nrow) {
    const int64_t J1 = std::min(mmax, J0 + nrow);
    for (int64_t j0 = J0; j0 < J1; j0 += CHOL_NB) {
      const int jb = (int)std::min<int64_t>(CHOL_NB, J1 - j0);
      const double* Li = P->bat_linv + j0 * CHOL_NB;
      // With R = I (A_I^{-1} only) the forward solve builds L^{-1}, which is
      // lower triangular: rows j0.. of R are still zero right of column j0 + jb.
      const int64_t nc = full_w ? ncols : std::min<int64_t>(ncols, j0 + jb);
      double* Rj = R + j0 * ncols;
      {  // R[j0:j0+jb, :nc] = L_jj^{-1} R[j0:j0+jb, :nc]
        F64Operands op = bat(F64Operands{Li, jb, id, id, Rj, ncols, id, id, jb, nc, jb}, zLi, zR);
        IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStore{Rj, ncols, 1.0, 0.0, zR}, st)));
      }
      const int64_t rest = J1 - j0 - jb;
      if (rest > 0) {  // R[j0+jb:J1, :nc] -= L[j0+jb:J1, j0:j0+jb] R[j0:j0+jb, :nc]
        F64Operands op = bat(F64Operands{Lw + (j0 + jb) * mmax + j0, mmax, id, id, Rj, ncols, id, id, rest, nc, jb},
                             zL, zR);
        IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStore{R + (j0 + jb) * ncols, ncols, -1.0, 1.0, zR}, st)));
      }
    }
    if (J1 < mmax) {   // all K blocks at once
      IBMI_TRY(refine_gemm_sub(tc, Lw + J1 * mmax + J0, mmax, zL, mmax - J1, J1 - J0, R + J0 * ncols, ncols, zR, J1,
                               R + J1 * ncols, ncols, zR, K, st));
      ps.flops -= 2.0 * (double)K * (mmax - J1) * J1 * (J1 - J0);   // counted by its own (tensor) class
    }
  }
  double* X = R;   // the solutions
  if (full_w) {
    const int64_t nbk = (mmax + CHOL_NB - 1) / CHOL_NB;
    for (int64_t b = nbk - 1; b >= 0; --b) {
      const int64_t j0 = b * CHOL_NB;
      const int jb = (int)std::min<int64_t>(CHOL_NB, mmax - j0);
      const double* Li = P->bat_linv + j0 * CHOL_NB;
      double* Rj = R + j0 * ncols;
      {  // R[j0:j0+jb, :] = L_jj^{-T} R[j0:j0+jb, :]
        F64Operands op = bat(F64Operands{Li, jb, id, id, Rj, ncols, id, id, jb, ncols, jb}, zLi, zR);
        IBMI_CUDA_TRY((launch_gemm_f64<false, true>(op, EpiStore{Rj, ncols, 1.0, 0.0, zR}, st)));
      }
      if (j0 > 0) {  // R[0:j0, :] -= L[j0:j0+jb, 0:j0]^T R[j0:j0+jb, :]
        F64Operands op = bat(F64Operands{Lw + j0 * mmax, mmax, id, id, Rj, ncols, id, id, j0, ncols, jb}, zL, zR);
        IBMI_CUDA_TRY((launch_gemm_f64<false, true>(op, EpiStore{R, ncols, -1.0, 1.0, zR}, st)));
      }
    }
  } else if (leave_y) {
    return IBMI_OK;   // the caller forms A_I^{-1} = Y^T Y from P->bat_R
  } else {
    // R holds Y = L^{-1}; A_I^{-1} = Y^T Y in one product (into the buffer of L,
    // no longer needed), each tile summing only k >= max(i, j).
    F64Operands op = bat(F64Operands{R, ncols, id, id, R, ncols, id, id, mmax, mmax, mmax}, zR, zR);
    op.tri_k = true;
    op.lower_tiles = true;
    IBMI_CUDA_TRY((launch_gemm_f64<false, true>(op, EpiStore{Lw, mmax, 1.0, 0.0, zL}, st)));
    X = Lw;
  }
  const int64_t nout = std::max(mmax * mmax, full_w ? mmax * p : 0);
  note_launch();
  k_bat_extract<<<dim3(nblk(nout), 1, K), 256, 0, st>>>(X, P->dlo, P->dm, mmax, ncols, full_w ? 1 : 0,
                                                         full_w ? 0 : 1, P->pool, P->doff_ainv, P->doff_w, p);
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
                             double* partials, int64_t n_partials, double* dout, cudaStream_t st, bool a_lower) {
  const GapMap id{0, 0};
  if (gemm_f64_ctas(p, p) > n_partials) return IBMI_ERR_INVALID_ARG;
  ProfScope ps(IBMI_K_RESIDUAL, st, 2.0 * (double)p * p * p);
  F64Operands op{A, lda, id, id, H, ldh, id, id, p, p, p};
  op.a_lower = a_lower;
  IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiResidual{partials, 0.0}, st)));
  note_launch();
  k_finish_residual<<<1, 1024, 0, st>>>(partials, gemm_f64_ctas(p, p), p, dout);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

// Residual rows: out[0] = ||(H A)[rows] - I[rows]||_F / sqrt(p) for the m
// rows H[row0 .. row0 + m) of an iterate, given as an m x p strip.
struct EpiResidualRows {
  double* partials; int64_t row0;
  double s;
  __device__ void begin() { s = 0.0; }
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    const double r = (i + row0 == j ? 1.0 : 0.0) - acc;
    s = fma(r, r, s);
  }
  __device__ void end() {
    __shared__ double red[F64_THREADS / 32];
    double v = s;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < F64_THREADS / 32; ++w) t += red[w];
      partials[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
};

ibmi_status residual_rows_f64_dev(const double* Hrows, int64_t ldh, int64_t m, int64_t row0, const double* A,
                                  int64_t lda, int64_t p, double* partials, int64_t n_partials, double* dout,
                                  cudaStream_t st) {
  const GapMap id{0, 0};
  if (gemm_f64_ctas(m, p) > n_partials) return IBMI_ERR_INVALID_ARG;
  ProfScope ps(IBMI_K_RESIDUAL, st, 2.0 * (double)m * p * p);
  F64Operands op{Hrows, ldh, id, id, A, lda, id, id, m, p, p};
  IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiResidualRows{partials, row0, 0.0}, st)));
  note_launch();
  k_finish_residual<<<1, 1024, 0, st>>>(partials, gemm_f64_ctas(m, p), p, dout);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status symmetrize_into(const double* S, int64_t m, double* H, int64_t ldh, int64_t lo, cudaStream_t st) {
  note_launch();
  k_symmetrize_into<<<nblk(m * m), 256, 0, st>>>(S, m, H, ldh, lo);
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
                        cudaStream_t st, double* backup) {
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
  if (backup)   // X before the step (R is no longer read: the copy is ordered after the product)
    IBMI_CUDA_TRY(cudaMemcpy2DAsync(backup, sizeof(double) * p, X, sizeof(double) * ldx, sizeof(double) * p, p,
                                    cudaMemcpyDeviceToDevice, st));
  note_launch();
  k_symmetrize_full<<<nblk(p * p), 256, 0, st>>>(P->nsX, p, X, ldx);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

// ------------------------------------------------- paper's estimate ----
//
// eq. error for the set I = [lo, hi): B = (H A)[I, I^c] (the (1,2) block of
// H A, i.e. H_I A_{I,I^c} + H_{I,I^c} A_{I^c}) and its spectral norm by power
// iteration on B^T B.

struct EpiStoreB {
  double* B; int64_t ldb;
  __device__ void begin() {}
  __device__ void end() {}
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) { B[i * ldb + j] = acc; }
};

// y = B x (B m x n, row-major); one warp per row.
__global__ void k_gemv(const double* B, int64_t m, int64_t n, const double* x, double* y) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s = fma(B[row * n + j], x[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// x = B^T y; one thread per column.
__global__ void k_gemvT(const double* B, int64_t m, int64_t n, const double* y, double* x) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s = fma(B[i * n + j], y[i], s);
  x[j] = s;
}

// v <- x / ||x||, sigma = sqrt(||x||) (x = B^T B v with ||v|| = 1); one CTA.
__global__ void k_normalize(double* x, int64_t n, double* v, double* sigma) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s = fma(x[j], x[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    red[0] = sqrt(t);
    sigma[0] = sqrt(red[0]);
  }
  __syncthreads();
  const double nrm = red[0];
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) v[j] = nrm > 0.0 ? x[j] / nrm : 0.0;
}

__global__ void k_fill_ones(double* v, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) v[j] = 1.0 / sqrt((double)n) * (1.0 + 1e-3 * (double)(j % 7));
}

ibmi_status paper_estimate_f64(ibmi_plan_s* P, const double* A, int64_t lda, const double* H, int64_t ldh,
                               cudaStream_t st, double* out) {
  const int K = (int)P->lo.size();
  const int64_t p = P->d.p, lo = P->lo[K - 1], m = P->hi[K - 1] - lo, n = p - m;
  if (n == 0) { *out = 0.0; return IBMI_OK; }
  if (!P->pe) {
    IBMI_CUDA_TRY(cudaMalloc(&P->pe, sizeof(double) * (m * n + 2 * n + m + 4)));
  }
  double* B = P->pe;
  double* v = B + m * n;
  double* x = v + n;
  double* y = x + n;
  double* sig = y + m;
  const GapMap gap{lo, m}, id{0, 0};
  {
    ProfScope ps(IBMI_K_RESIDUAL, st, 2.0 * (double)m * n * p);
    F64Operands op{H + lo * ldh, ldh, id, id, A, lda, id, gap, m, n, p};
    IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStoreB{B, n}, st)));
  }
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  note_launch();
  k_fill_ones<<<nblk(n), 256, 0, st>>>(v, n);
  for (int it = 0; it < 60; ++it) {
    note_launch(3);
    k_gemv<<<(unsigned)((m + 7) / 8), 256, 0, st>>>(B, m, n, v, y);
    k_gemvT<<<nblk(n), 256, 0, st>>>(B, m, n, y, x);
    k_normalize<<<1, 1024, 0, st>>>(x, n, v, sig);
  }
  IBMI_CUDA_TRY(cudaGetLastError());
  IBMI_CUDA_TRY(cudaMemcpyAsync(out, sig, sizeof(double), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  return IBMI_OK;
}

__global__ void k_set_identity(double* H, int64_t ldh, int64_t p) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * p) return;
  int64_t i = idx / p, j = idx - i * p;
  H[i * ldh + j] = (i == j) ? 1.0 : 0.0;
}

// S = A with the strict upper triangle taken from the lower one: only
// elements A[i][j] with i >= j are read.  32 x 32 tiles through shared memory;
// a tile above the diagonal is the transpose of its mirror below it.
__global__ void k_sym_from_lower(const double* A, int64_t lda, int64_t p, double* S, int64_t lds) {
  __shared__ double t[32][33];
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const bool upper = J0 > I0;
  const int64_t R0 = upper ? J0 : I0, C0 = upper ? I0 : J0;   // source tile, on or below the diagonal
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = R0 + r, j = C0 + tx;
    t[r][tx] = (i < p && j < p && i >= j) ? A[i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = I0 + r, j = J0 + tx;
    if (i >= p || j >= p) continue;
    double v;
    if (upper) v = t[tx][r];                      // S[i][j] = A[j][i]
    else if (I0 > J0) v = t[r][tx];
    else v = r >= tx ? t[r][tx] : t[tx][r];       // diagonal tile
    S[i * lds + j] = v;
  }
}

ibmi_status sym_from_lower(const double* A, int64_t lda, int64_t p, double* S, int64_t lds, cudaStream_t st) {
  const unsigned nt = (unsigned)((p + 31) / 32);
  note_launch();
  k_sym_from_lower<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(A, lda, p, S, lds);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status set_identity(double* H, int64_t ldh, int64_t p, cudaStream_t st) {
  note_launch();
  k_set_identity<<<nblk(p * p), 256, 0, st>>>(H, ldh, p);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

}  // namespace ibmi
