// Internal plan object and the host-side drivers of each hot-path step.
#pragma once
#include <math.h>

#include <algorithm>

#include "cadence.h"
#include "common.cuh"

struct ibmi_plan_s {
  ibmi_plan_desc d{};
  std::vector<int64_t> lo, hi;   // sets I_k = [lo_k, hi_k)
  int64_t mmax = 0;
  int device = 0;
  // persistent per-set invariants (eq. IBMI terms that do not depend on H)
  std::vector<double*> ainv;     // A_I^{-1}, m x m
  std::vector<double*> w;        // W = A_I^{-1} A_{I,:}, m x p, zero columns on I
  double* pool = nullptr;        // one allocation backing ainv / w / scratch
  size_t pool_bytes = 0;
  // batched factorisation scratch (all K blocks padded to mmax, blockIdx.z = k)
  double* bat_L = nullptr;       // K x mmax x mmax Cholesky factors
  double* bat_R = nullptr;       // K x mmax x ncols right-hand sides / solutions
  double* bat_linv = nullptr;    // K x mmax x 32 inverted diagonal tiles
  int64_t* dlo = nullptr;        // device copies of lo_k, m_k and of the pool offsets
  int64_t* dm = nullptr;         // of A_I^{-1} and W for each set
  int64_t* doff_ainv = nullptr;
  int64_t* doff_w = nullptr;
  int64_t* doffA = nullptr;      // batched groups: element offset in A of block z's matrix (else NULL);
                                 // then dstatus holds one status word per block
  int tile_batch = 0;            // batched groups: sets per matrix (tile choice of the FP64 products)
  void* bat_pool = nullptr;
  // scratch
  double* S = nullptr;           // mmax x mmax, a4 result before symmetrisation
  double* partials = nullptr;    // residual partial sums
  int64_t n_partials = 0;
  double* dscalar = nullptr;     // device scalar results
  ibmi::DevStatus* dstatus = nullptr;
  // paper's estimate (eq. error): B = (H A)[I_K, I_K^c] and power-iteration vectors
  double* pe = nullptr;
  // Newton-Schulz buffers (allocated on first use)
  double* nsR = nullptr;
  double* nsX = nullptr;
  // host-variant staging (allocated on first use)
  double* dA = nullptr;
  double* dAs = nullptr;         // p x p: A symmetrised from its lower triangle (every solve)
  double* dH = nullptr;
  // mixed-precision state (allocated at plan time when precision == MIXED)
  void* mixed = nullptr;
  // IBMI_INIT_SCHUR: one-set plan over the complement [hi_1, p) of the first
  // set, whose block inverse is the initial guess (guess.cu)
  ibmi_plan_s* guess = nullptr;
  // ibmi_invert_block_diag scratch (allocated on first use): X of one set
  // (mmax x p) and the last set's rows of H (m_K x p)
  double* bdX = nullptr;
  double* bdRows = nullptr;
};

namespace ibmi {

struct RefineState;
constexpr int CHOL_NB = 32;

// Stop-test cadence: cadence.h.

// a2 for all sets at once, FP64: A_I^{-1} for every set and, with full_w,
// W = A_I^{-1} A_{I,:} (zero columns on I) -- the mixed path forms W on tensor
// cores instead.  Non-SPD blocks are reported through plan->dstatus (read by
// the caller after a stream sync).
// leave_y (with full_w false): stop after the forward solve, leaving Y = L^{-1}
// of set k in P->bat_R + k * mmax * mmax (row pitch mmax) for the caller.
// tc (mixed path): blocks of order >= kTcCholMinOrder take the Cholesky's
// trailing updates beyond each 256-column block column on the tensor cores,
// FP64-accurate (refine_syrk_sub); the block column itself stays DFMA.
ibmi_status invariants_all(ibmi_plan_s* P, const double* A, int64_t lda, bool full_w, cudaStream_t st,
                           bool leave_y = false, RefineState* tc = nullptr);
constexpr int64_t kTcCholMinOrder = 512;    // block order from which tc applies
constexpr int64_t kTcCholPanel = 256;       // block-column width of that factorisation

// a3 + a4 for set k on an FP64 iterate H.
ibmi_status sweep_step_f64(ibmi_plan_s* P, int k, double* H, int64_t ldh, cudaStream_t st);

// a6: rho_F = ||I - A H||_F / sqrt(p), FP64, value left in *dout (device).
// a_lower: A is read from its lower triangle only.
ibmi_status residual_f64_dev(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                             double* partials, int64_t n_partials, double* dout, cudaStream_t st,
                             bool a_lower = false);

// ||(H A)[rows] - I[rows]||_F / sqrt(p) for the m rows [row0, row0 + m) of an
// iterate given as an m x p strip (row pitch ldh); value left in *dout.
ibmi_status residual_rows_f64_dev(const double* Hrows, int64_t ldh, int64_t m, int64_t row0, const double* A,
                                  int64_t lda, int64_t p, double* partials, int64_t n_partials, double* dout,
                                  cudaStream_t st);

// H[lo + i, lo + j] = (S[i, j] + S[j, i]) / 2 for an m x m S (row pitch m).
ibmi_status symmetrize_into(const double* S, int64_t m, double* H, int64_t ldh, int64_t lo, cudaStream_t st);

// Device memory of the current device (plain or managed): the pointer checks
// of the entry points.
bool is_device_ptr(const void* ptr);

// a7: one Newton-Schulz step X <- sym(X + X (I - A X)) in FP64 (scratch
// P->nsR, P->nsX).  backup (p x p, row pitch p; may be P->nsR): receives X
// before the step, so that a step that does not help can be undone.
ibmi_status ns_step_f64(ibmi_plan_s* P, const double* A, int64_t lda, double* X, int64_t ldx,
                        cudaStream_t st, double* backup = nullptr);

// Copies a p x p FP64 matrix between device buffers (row pitches in elements).
inline ibmi_status copy_square(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t p, cudaStream_t st) {
  IBMI_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(double) * ldd, src, sizeof(double) * lds, sizeof(double) * p, p,
                                  cudaMemcpyDeviceToDevice, st));
  return IBMI_OK;
}

ibmi_status set_identity(double* H, int64_t ldh, int64_t p, cudaStream_t st);

// IBMI_INIT_SCHUR (guess.cu): workspace of the complement block of the first
// set; H = identity with H[I_1^c, I_1^c] = A_{I_1^c}^{-1} (R: the mixed path's
// refinement state, whose sliced Y^T Y serves blocks of order >= 1024; NULL:
// FP64); its algorithmic flops; NOT_SPD of that block (bad_block = K) after
// a stream sync.
struct RefineState;
ibmi_status schur_guess_create(ibmi_plan_s* P);
void schur_guess_destroy(ibmi_plan_s* P);
ibmi_status schur_guess_launch(ibmi_plan_s* P, const double* A, int64_t lda, double* H, int64_t ldh,
                               cudaStream_t st, RefineState* R);
// The guess block alone: A_{I_1^c}^{-1} into T0 ((p - hi_1) x (p - hi_1), row pitch ldt).
ibmi_status schur_guess_block(ibmi_plan_s* P, const double* A, int64_t lda, double* T0, int64_t ldt,
                              cudaStream_t st, RefineState* R);
double schur_guess_flops(const ibmi_plan_s* P);
ibmi_status schur_guess_status(ibmi_plan_s* P, cudaStream_t st, ibmi_result* res);

// S (ld lds) = the symmetric matrix whose lower triangle is A's; the strict
// upper triangle of A is never read.
ibmi_status sym_from_lower(const double* A, int64_t lda, int64_t p, double* S, int64_t lds, cudaStream_t st);

// eq. error on the last set: ||(H A)[I_K, I_K^c]||_2 (FP64 GEMM, then power
// iteration on B^T B); host value in *out (syncs the stream).
ibmi_status paper_estimate_f64(ibmi_plan_s* P, const double* A, int64_t lda, const double* H, int64_t ldh,
                               cudaStream_t st, double* out);

}  // namespace ibmi
