// Partial inverse: the diagonal blocks of the IBMI iterate only (Section 6
// proposes approximating block-diagonal parts of the inverse when only those
// are needed).
//
// With two sets I_1 = [0, hi_1) and I_2 = [lo_2, p) (lo_2 <= hi_1) the step
// for I_1 reads T_1 = H[I_1^c, I_1^c] = H[hi_1:, hi_1:], which lies inside
// H[I_2, I_2] as rewritten by the previous step for I_2, and the step for I_2
// reads T_2 = H[0:lo_2, 0:lo_2], inside H[I_1, I_1] as just rewritten (eq.
// IBMI).  So the two diagonal blocks D_1 = H[I_1, I_1], D_2 = H[I_2, I_2]
// evolve on their own: per sweep
//     X_1 = -W_1 D_2[ov:, ov:],  D_1 = sym(A_1^{-1} - X_1 W_1^T),
//     X_2 = -W_2 D_1[:lo_2, :lo_2], D_2 = sym(A_2^{-1} - X_2 W_2^T),
// with ov = hi_1 - lo_2 and W_k = A_{I_k}^{-1} A_{I_k, I_k^c}: the same
// arithmetic as the full sweep, without storing or scattering the
// off-diagonal blocks of H (memory m_1^2 + m_2^2 + m_max p instead of p^2).
// With more sets the complement of a set spans off-diagonal blocks between
// other sets, so the recurrence does not close; only two sets are accepted.
//
// Stop quantity: the last set's rows of the residual, ||(H A - I)[I_2, :]||_F
// / sqrt(p), from the strip H[I_2, :] = [X_2 | D_2]; in exact arithmetic its
// (I_2, I_2) part is zero and the (I_2, I_2^c) part is W_2 (I - T_2 S_2), S_2
// the Schur complement on I_2^c, so it measures how far T_2 = H[I_2^c, I_2^c]
// is from the inverse Schur complement (the quantity eq. error estimates).
// On return D_1 carries, on the overlap rows and columns [lo_2, hi_1), what
// the last step for I_2 wrote there, so that D_1 and D_2 are exactly the
// diagonal blocks of the full iterate after the last sweep.
#include <math.h>

#include <chrono>
#include <cstring>

#include "gemm_f64.cuh"
#include "plan.cuh"

namespace ibmi {

// D_1's overlap rows and columns [lo2, hi1) from the last step for I_2:
// D_1[lo2 + a, j] = D_1[j, lo2 + a] = X_2[a, j] for j < lo2, and
// D_1[lo2 + a, lo2 + b] = D_2[a, b]; a, b < ov.
__global__ void k_patch_overlap(const double* X2, int64_t ldx, const double* D2, int64_t m2, int64_t lo2, int64_t ov,
                                double* D1, int64_t m1) {
  const int64_t a = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= ov || j >= lo2 + ov) return;
  if (j < lo2) {
    const double x = X2[a * ldx + j];
    D1[(lo2 + a) * m1 + j] = x;
    D1[j * m1 + lo2 + a] = x;
  } else {
    D1[(lo2 + a) * m1 + j] = D2[a * m2 + (j - lo2)];
  }
}

static ibmi_status block_diag_impl(ibmi_plan_s* P, const double* A, int64_t lda, double* D, cudaStream_t st,
                                   ibmi_result* res) {
  const ibmi_plan_desc& d = P->d;
  const int64_t p = d.p;
  const int64_t lo2 = P->lo[1], hi1 = P->hi[0], m1 = hi1, m2 = p - lo2, ov = hi1 - lo2;
  const int64_t n1 = p - m1, n2 = p - m2;   // = p - hi1 and lo2
  double* D1 = D;
  double* D2 = D + m1 * m1;
  if (!P->bdX) {
    IBMI_CUDA_TRY(cudaMalloc(&P->bdX, sizeof(double) * (size_t)P->mmax * p));
    IBMI_CUDA_TRY(cudaMalloc(&P->bdRows, sizeof(double) * (size_t)m2 * p));
  }
  IBMI_TRY(sym_from_lower(A, lda, p, P->dAs, p, st));
  A = P->dAs;
  lda = p;
  double flops = 0.0;
  IBMI_CUDA_TRY(cudaMemsetAsync(P->dstatus, 0, sizeof(DevStatus), st));
  IBMI_TRY(invariants_all(P, A, lda, true, st));
  for (int k = 0; k < 2; ++k) {
    const double m = (double)(P->hi[k] - P->lo[k]), n = (double)p - m;
    flops += m * m * m / 3.0 + 2.0 * m * m * m + 2.0 * m * m * n;
  }
  DevStatus hs;
  IBMI_CUDA_TRY(cudaMemcpyAsync(&hs, P->dstatus, sizeof(hs), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs.code == IBMI_ERR_NOT_SPD) {
    res->bad_block = hs.block;
    res->bad_pivot = hs.pivot;
    return IBMI_ERR_NOT_SPD;
  }
  // the initial guess lives in D_2 (T_1 = D_2[ov:, ov:] is all the first step reads)
  if (d.init == IBMI_INIT_IDENTITY) IBMI_TRY(set_identity(D2, m2, m2, st));
  if (d.init == IBMI_INIT_SCHUR) {
    IBMI_TRY(set_identity(D2, m2, m2, st));
    IBMI_TRY(schur_guess_block(P, A, lda, D2 + ov * m2 + ov, m2, st, nullptr));
    IBMI_TRY(schur_guess_status(P, st, res));
    flops += schur_guess_flops(P);
  }
  const GapMap id{0, 0}, gap1{0, m1}, gap2{lo2, m2};
  const double fs = 2.0 * m1 * n1 * n1 + 2.0 * m1 * m1 * n1 + 2.0 * m2 * n2 * n2 + 2.0 * m2 * m2 * n2;
  const double fr = 2.0 * (double)m2 * p * p;
  CheckCadence cad;
  cad.gmin = cad.next = d.check_every;
  ibmi_status status = IBMI_NOT_CONVERGED;
  double* X = P->bdX;
  for (int r = 1;; ++r) {
    {  // set 1: X_1 = -W_1 T_1, T_1 = D_2[ov:, ov:]
      ProfScope ps(IBMI_K_SWEEP_X, st, 2.0 * m1 * n1 * n1);
      F64Operands op{P->w[0], p, id, gap1, D2 + ov * m2 + ov, m2, id, id, m1, n1, n1};
      IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStore{X, n1, -1.0, 0.0}, st)));
    }
    {  // S_1 = A_1^{-1} - X_1 W_1^T, D_1 = sym(S_1)
      ProfScope ps(IBMI_K_SWEEP_S, st, 2.0 * m1 * m1 * n1);
      F64Operands op{X, n1, id, id, P->w[0], p, gap1, id, m1, m1, n1};
      IBMI_CUDA_TRY((launch_gemm_f64<true, false>(op, EpiSweepS{P->ainv[0], P->S, m1}, st)));
    }
    IBMI_TRY(symmetrize_into(P->S, m1, D1, m1, 0, st));
    {  // set 2: X_2 = -W_2 T_2, T_2 = D_1[:lo2, :lo2]
      ProfScope ps(IBMI_K_SWEEP_X, st, 2.0 * m2 * n2 * n2);
      F64Operands op{P->w[1], p, id, gap2, D1, m1, id, id, m2, n2, n2};
      IBMI_CUDA_TRY((launch_gemm_f64<true, true>(op, EpiStore{X, n2, -1.0, 0.0}, st)));
    }
    {
      ProfScope ps(IBMI_K_SWEEP_S, st, 2.0 * m2 * m2 * n2);
      F64Operands op{X, n2, id, id, P->w[1], p, gap2, id, m2, m2, n2};
      IBMI_CUDA_TRY((launch_gemm_f64<true, false>(op, EpiSweepS{P->ainv[1], P->S, m2}, st)));
    }
    IBMI_TRY(symmetrize_into(P->S, m2, D2, m2, 0, st));
    flops += fs;
    res->sweeps = r;
    if (r < cad.next && r < d.max_sweeps) continue;
    // the last set's rows of H: [X_2 | D_2]
    double* rows = P->bdRows;
    IBMI_CUDA_TRY(cudaMemcpy2DAsync(rows, sizeof(double) * p, X, sizeof(double) * n2, sizeof(double) * n2, m2,
                                    cudaMemcpyDeviceToDevice, st));
    IBMI_CUDA_TRY(cudaMemcpy2DAsync(rows + n2, sizeof(double) * p, D2, sizeof(double) * m2, sizeof(double) * m2,
                                    m2, cudaMemcpyDeviceToDevice, st));
    IBMI_TRY(residual_rows_f64_dev(rows, p, m2, lo2, A, lda, p, P->partials, P->n_partials, P->dscalar, st));
    double v[2];
    IBMI_CUDA_TRY(cudaMemcpyAsync(v, P->dscalar, sizeof(v), cudaMemcpyDeviceToHost, st));
    IBMI_CUDA_TRY(cudaStreamSynchronize(st));
    flops += fr;
    res->resid_f = v[0];
    if (!isfinite(v[0])) { status = IBMI_ERR_NONFINITE; break; }
    if (v[0] <= d.tol) { status = IBMI_OK; break; }
    if (r >= d.max_sweeps) break;
    cad.after(r, v[0], d.tol);
  }
  if (ov > 0) {
    note_launch();
    k_patch_overlap<<<dim3((unsigned)((hi1 + 255) / 256), (unsigned)ov), 256, 0, st>>>(X, n2, D2, m2, lo2, ov, D1,
                                                                                    m1);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  res->flops = flops;
  return status;
}

}  // namespace ibmi

using namespace ibmi;

extern "C" ibmi_status ibmi_invert_block_diag(ibmi_plan_t P, const double* A, int64_t lda, double* D, void* stream,
                                              ibmi_result* out) {
  ibmi_result tmp;
  ibmi_result* res = out ? out : &tmp;
  memset(res, 0, sizeof(*res));
  res->bad_block = -1;
  res->bad_pivot = -1;
  res->resid_f = NAN;
  res->paper_est = NAN;
  ibmi_status s;
  if (!P || !A || !D || lda < P->d.p) {
    s = IBMI_ERR_INVALID_ARG;
  } else if (P->lo.size() != 2 || P->d.precision != IBMI_FP64 || P->d.stop_rule != IBMI_STOP_RESID_F) {
    set_last_error("ibmi_invert_block_diag: needs a plan with two sets, IBMI_FP64 and IBMI_STOP_RESID_F");
    s = IBMI_ERR_INVALID_ARG;
  } else if (!is_device_ptr(A) || !is_device_ptr(D)) {
    s = IBMI_ERR_INVALID_ARG;
  } else {
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    s = block_diag_impl(P, A, lda, D, st, res);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && s == IBMI_OK) { set_last_error(cudaGetErrorString(e)); s = IBMI_ERR_CUDA; }
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  res->status = s;
  return s;
}
