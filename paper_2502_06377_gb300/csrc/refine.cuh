// FP64-accurate residual and Newton-Schulz refinement on tcgen05 (internal).
#pragma once
#include <cuda_bf16.h>

#include <vector>

#include "tc_gemm.cuh"

namespace ibmi {

// Error-free sliced product (Ozaki scheme): every row of an FP64 matrix is
// written as 2^e_i * sum_s d_s 2^{-6-7s} with signed integer digits
// |d_s| <= 64.  Digits are exact in BF16, a digit product is at most 2^12, so
// a single slice-pair product accumulated in FP32 over K <= 4096 terms is an
// exact integer; pair products are summed per digit group q = s + u in int32
// and combined once in FP64.  The iterate X = A^{-1} is strongly diagonal, so
// its digits are fixed-point relative to a large row maximum; it gets ten
// digits (69 bits) against eight (55 bits) for A, which keeps the error of
// I - X A below the FP64 rounding of a direct evaluation.
constexpr int OZ_S = 10;        // maximum digit slices per operand
constexpr int OZ_SX = 10;       // digits of the iterate
constexpr int OZ_SA = 8;        // digits of A
constexpr int OZ_QMAX = 9;      // highest digit group kept (52 pair products)
constexpr int OZ_KCHUNK = 4096; // exactness bound on K per accumulation
constexpr int OZ_NONFINITE_EXP = 1 << 20;   // row exponent marking an Inf or NaN in the row: every
                                            // value recombined from it is NaN
constexpr int NS_S = 5;         // digit slices of the Newton-Schulz update operands (34 bits,
                                // digit groups q <= 4: 15 exact pair products)

struct RefineState {
  int64_t p = 0, ldp = 0;
  int bn = 224;                   // N tile of the digit-pair products (by order; see refine_create)
  __nv_bfloat16* Ao[OZ_SA] = {};  // digit slices of A (rows), p x ldp
  __nv_bfloat16* Xo[OZ_S] = {};   // digit slices of the iterate X
  int* expA = nullptr;            // row exponents
  int* expX = nullptr;
  int* expQ = nullptr;
  int* T = nullptr;               // (OZ_QMAX+1) x p x ldp int32 group sums
  __nv_bfloat16* Qo[NS_S] = {};   // leading digit slices of Q = I - X A
  __nv_bfloat16* Af[2] = {};      // BF16 hi/lo of A (cheap residual)
  double* Xn = nullptr;           // p x p FP64 scratch: X + X Q^T of an update, X - Xprev of a correction
  double* Q = nullptr;            // p x p FP64: Q = I - X A of the last residual
  double* partials = nullptr;     // reduction partials
  int64_t n_partials = 0;
  double* dout = nullptr;         // device scalars
  double* pv = nullptr;           // power-iteration vectors (2 p) and estimate
  float* sqA = nullptr;           // per row of A and of the last residual's X: sum of (x 2^-e)^2
  float* sqX = nullptr;
  int* err = nullptr;
  CUtensorMap mAo[OZ_SA], mXo[OZ_S], mQo[NS_S], mAf[2];
  CUtensorMap mXo_b[NS_S];        // the first X digit planes with BN-row boxes (as a right operand)
  void* pool = nullptr;
  // W of all sets in one pass (refine_plan_w): set k's rows sit in a slot of
  // whole 128-row tiles starting at row w_off[k] of a stacked view of the X
  // digit region (5 planes of w_rows rows) and of the T region.
  int64_t w_rows = 0;              // 0: W is formed set by set
  std::vector<int64_t> w_off;
  int* expW = nullptr;             // row exponents of the stacked A_I^{-1}
  int2* w_kr = nullptr;            // K-tile range of every 128-row tile
  CUtensorMap mXw[5];
  void* wpool = nullptr;
};

ibmi_status refine_create(RefineState* R, int64_t p, int* err);
void refine_destroy(RefineState* R);

// Digit slices of A (once per matrix) and its BF16 hi/lo split.
ibmi_status refine_set_matrix(RefineState* R, const double* A, int64_t lda, cudaStream_t st);

// rho_F = ||I - X A||_F / sqrt(p) (= ||I - A X||_F / sqrt(p) for symmetric
// A, X), accurate to FP64 rounding; leaves Q = I - X A (FP64) and the digit
// slices of X for ns_update.  Host value in *rho (syncs the stream).
ibmi_status refine_residual(RefineState* R, const double* X, int64_t ldx, cudaStream_t st, double* rho);

// X <- sym(X + X Q^T) = sym(X (2I - A X)), the update of eq. newton; the
// product X Q^T uses the five leading digits of X and of Q, digit groups
// <= qmax of their exact pair products (qmax = 4: all 15 pairs, 2^-34
// relative truncation; 3: 10 pairs), so its error stays proportional to Q.
// Must follow a residual of the same X: a direct one leaves the digits of X
// the update uses, after a correction (below) reslice_x slices them first.
// backup (p x p, row pitch p), if given, receives X before the update.
// symmetric_x (X exactly symmetric, as every iterate of the mixed path): X Q^T
// = X - X A X is symmetric, so only the product's tiles on and below the
// diagonal are formed (half the pair products) and mirrored; else the whole
// product is formed and X + X Q^T symmetrised.
ibmi_status refine_ns_update(RefineState* R, double* X, int64_t ldx, cudaStream_t st, int qmax = NS_S - 1,
                             double* backup = nullptr, bool reslice_x = false, bool symmetric_x = false);

// W = A_I^{-1} A_{I,:} (m x p, zero columns on I) from exact digit products
// (five digits of A_I^{-1}, four of A), written as three BF16 slices with
// row pitch ldp.  Needs refine_set_matrix first; uses the X digit planes.
ibmi_status refine_form_w(RefineState* R, const double* Ainv, int64_t m, int64_t lo, int64_t hi, __nv_bfloat16* W0,
                          __nv_bfloat16* W1, __nv_bfloat16* W2, cudaStream_t st);

// A_I^{-1} = Y^T Y of one diagonal block from Y = L^{-1} (m x m, row pitch
// ldy, lower triangular) as an error-free sliced product on tensor cores:
// five 7-bit digits of each row of Z = Y^T (34 bits), digit groups q <= 4 (15
// pair products in one all-pairs launch), recombined exactly and rounded once
// to FP64 into Ainv (m x m, row pitch m).  Borrows the X digit planes and the
// FP64 scratch.
ibmi_status refine_block_inverse(RefineState* R, const double* Y, int64_t ldy, int64_t m, double* Ainv,
                                 cudaStream_t st);

// The trailing update of a blocked Cholesky step for nbat blocks, C_b -=
// L_b L_b^T on and below the diagonal (C_b = C + b zc: M x M at row pitch
// ldc; L_b = L + b zl: M x nb at row pitch ldl, nb a multiple of 64 and at
// most 4096; M <= p), FP64-accurate on tensor cores: the rows of L_b sliced
// into eight 7-bit digits (56 bits below each row's maximum, FP64's 53 and
// three more), the 43 exact pair products of digit groups q <= 8 on the tiles
// that reach the diagonal, for as many blocks per launch as the planes hold,
// recombined exactly and subtracted in FP64.  Borrows the X digit planes and
// the group planes.
ibmi_status refine_syrk_sub(RefineState* R, const double* L, int64_t ldl, int64_t zl, int64_t M, int64_t nb,
                            double* C, int64_t ldc, int64_t zc, int64_t nbat, cudaStream_t st);

// C_b -= A_b B_b for nbat problems (C_b = C + b zc: M x N; A_b = A + b za:
// M x K; B_b = B + b zb: K x N; row pitches ldc, lda, ldb; K a multiple of 64
// and at most 4096; M, N <= p), FP64-accurate on tensor cores as
// refine_syrk_sub (rows of A_b and columns of B_b in eight 7-bit digits, 43
// exact pair products): the trailing update of a blocked triangular solve.
// Borrows the X and A digit planes, the FP64 scratch and the group planes:
// only before refine_set_matrix (the factorisations of the set-up).
ibmi_status refine_gemm_sub(RefineState* R, const double* A, int64_t lda, int64_t za, int64_t M, int64_t K,
                            const double* B, int64_t ldb, int64_t zb, int64_t N, double* C, int64_t ldc, int64_t zc,
                            int64_t nbat, cudaStream_t st);

// The same for the nbat blocks of a batched factorisation at once: Y_b =
// Y + b mmax^2 (mmax x mmax, row pitch mmax, block b padded with an identity
// beyond its order m_b = dm[b]), A_b^{-1} (m_b x m_b, row pitch m_b) to
// pool + doff[b] (dm, doff: device arrays).  As many blocks per launch as the
// planes hold.
ibmi_status refine_block_inverse_all(RefineState* R, const double* Y, int64_t mmax, int64_t nbat, double* pool,
                                     const int64_t* doff, const int64_t* dm, cudaStream_t st);

// Prepares the one-pass formation of W for the sets [lo_k, hi_k): the stacked
// view fits when 5 slots of sum_k ceil(m_k/128)*128 rows fit in the X digit
// and T regions and every set spans at most 4096 columns; otherwise W is
// formed set by set (w_rows stays 0).
ibmi_status refine_plan_w(RefineState* R, const std::vector<int64_t>& lo, const std::vector<int64_t>& hi);

// W_k for every set k at once (needs refine_plan_w with w_rows > 0 and
// refine_set_matrix): the same digit products as refine_form_w, 14 launches
// in all instead of 14 per set.
ibmi_status refine_form_w_all(RefineState* R, const std::vector<const double*>& Ainv, const std::vector<int64_t>& lo,
                              const std::vector<int64_t>& hi, __nv_bfloat16* const* W0, __nv_bfloat16* const* W1,
                              __nv_bfloat16* const* W2, cudaStream_t st);

// The same two residuals split into their kernels (no host synchronisation,
// so they can be captured in a CUDA graph) and the read of the value
// (synchronises the stream, reports a bounded-wait expiry as IBMI_ERR_TIMEOUT).
// qmax < OZ_QMAX keeps only digit groups q <= qmax (qmax + 1 digits of X,
// (qmax + 1)(qmax + 2)/2 pair products for qmax <= 7): Q then carries an
// absolute error of about 2^(e_X + e_A - 7 (qmax + 1)) sqrt(p), for a
// Newton-Schulz step that does not need FP64 accuracy (qmax >= 4, so that the
// update still finds its five digits of X).
// stats: also the statistics refine_read_groups returns (else those two
// values are undefined).
ibmi_status refine_residual_launch(RefineState* R, const double* X, int64_t ldx, cudaStream_t st,
                                   int qmax = OZ_QMAX, bool stats = false);
// Extends the last residual (of the same X, groups <= qfrom) to groups
// <= qto: only the pair products of groups qfrom + 1 .. qto are added (the
// digits of X are prefix-stable, so a wider slicing repeats the first ones).
// stats needs the last full slicing of X to have been made with stats.
ibmi_status refine_residual_extend_launch(RefineState* R, const double* X, int64_t ldx, cudaStream_t st, int qfrom,
                                          int qto, bool stats = false);
// The residual of X from that of the previous iterate Xprev (p x p, row
// pitch p), Q_X = Q_Xprev - (X - Xprev) A, by the same exact digit products
// applied to the difference D = X - Xprev (groups <= qmax, qmax + 1 digits of
// D): since D is small, few groups give Q_X to the accuracy of a full direct
// residual.  Q must hold Q_Xprev; rho and the norm of the last group's part
// of D A go to the values refine_read_groups returns (the third one is left
// as it was).  The digits of X are not sliced (see refine_ns_update).
ibmi_status refine_residual_correct_launch(RefineState* R, const double* X, int64_t ldx, const double* Xprev,
                                           cudaStream_t st, int qmax);
// Extends the last correction from groups <= qfrom to <= qto (only the new
// groups' pair products, subtracted from Q).
ibmi_status refine_residual_correct_extend_launch(RefineState* R, cudaStream_t st, int qfrom, int qto);
// rho of the last digit-sliced residual, the norm (/ sqrt(p)) of its last
// digit group's part (the groups left out fall below it by about 2^-7 each)
// and ||X||_F ||A||_F / p (the last two from a residual launched with stats).
ibmi_status refine_read_groups(RefineState* R, cudaStream_t st, double* rho, double* last_group, double* amp);
// ||I - H A||_F / sqrt(p) from BF16x3 products, for H given by its BF16 hi/lo
// slice maps (about 5 significant digits; the stop test of the sweeps and the
// hand-over to Newton-Schulz); value read by refine_read.
ibmi_status refine_cheap_residual_launch(RefineState* R, const CUtensorMap* mapH2, cudaStream_t st);
ibmi_status refine_read(RefineState* R, cudaStream_t st, double* rho);

// Spectral radius of Q = I - X A (left by the last accurate residual) by
// power iteration: v <- Q v / ||Q v|| from a fixed start, `iters` steps; the
// estimate is the last ||Q v||.  Q is similar to the symmetric
// I - A^{1/2} X A^{1/2} (X symmetric), so its eigenvalues are real and the
// estimate approaches their largest magnitude from below.  The Newton-Schulz
// residual after k steps is Q^(2^k): it converges iff that radius is below 1.
// The kernels only (capturable) and the read of the value.
ibmi_status refine_q_radius_launch(RefineState* R, int iters, cudaStream_t st);
ibmi_status refine_q_radius_read(RefineState* R, cudaStream_t st, double* radius);


}  // namespace ibmi
