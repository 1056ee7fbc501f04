// Initial guess T_0 = A_{I_1^c}^{-1} (IBMI_INIT_SCHUR): the inverse of A's
// diagonal block on the complement of the first set, one of the initial
// guesses compared in Section 5.6 (Table 6); Section 2.4 allows any SPD
// approximation of the inverse Schur complement there.
//
// The complement of the first set I_1 = [0, hi_1) is the contiguous range
// [hi_1, p), so its block is factorised by the same batched machinery as the
// sets' diagonal blocks (a2): an internal one-set plan over [hi_1, p) runs the
// FP64 Cholesky and forms the inverse, FP64 Y^T Y (Y = L^{-1}) or, for the
// mixed path with a block of order >= 1024, the exact sliced Y^T Y on the
// tensor cores (as for the sets' own blocks).
#include "plan.cuh"
#include "refine.cuh"

namespace ibmi {

ibmi_status schur_guess_create(ibmi_plan_s* P) {
  if (P->lo.size() < 2) return IBMI_OK;   // one set: no complement, the guess is never read
  const int64_t p = P->d.p, lo = P->hi[0], n = p - lo;
  ibmi_plan_s* G = new ibmi_plan_s();
  P->guess = G;
  G->d = P->d;
  G->d.K = 1;
  G->lo = {lo};
  G->hi = {p};
  G->mmax = n;
  G->device = P->device;
  if (cudaMalloc(&G->pool, sizeof(double) * (size_t)n * n) != cudaSuccess) {
    cudaGetLastError();
    return IBMI_ERR_OOM;
  }
  G->ainv.push_back(G->pool);
  G->w.push_back(nullptr);
  const size_t bat_doubles = (size_t)(n * n + n * n + n * CHOL_NB);
  if (cudaMalloc(&G->bat_pool, sizeof(double) * bat_doubles + sizeof(int64_t) * 4) != cudaSuccess ||
      cudaMalloc(&G->dstatus, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    return IBMI_ERR_OOM;
  }
  double* b = (double*)G->bat_pool;
  G->bat_L = b; b += n * n;
  G->bat_R = b; b += n * n;
  G->bat_linv = b; b += n * CHOL_NB;
  int64_t* ib = (int64_t*)b;
  G->dlo = ib; G->dm = ib + 1; G->doff_ainv = ib + 2; G->doff_w = ib + 3;
  const int64_t packed[4] = {lo, n, 0, 0};
  IBMI_CUDA_TRY(cudaMemcpy(ib, packed, sizeof(packed), cudaMemcpyHostToDevice));
  return IBMI_OK;
}

void schur_guess_destroy(ibmi_plan_s* P) {
  ibmi_plan_s* G = P->guess;
  if (!G) return;
  cudaFree(G->pool);
  cudaFree(G->bat_pool);
  cudaFree(G->dstatus);
  delete G;
  P->guess = nullptr;
}

ibmi_status schur_guess_block(ibmi_plan_s* P, const double* A, int64_t lda, double* T0, int64_t ldt,
                              cudaStream_t st, RefineState* R) {
  ibmi_plan_s* G = P->guess;
  if (!G) return IBMI_OK;
  const int64_t n = G->mmax;
  IBMI_CUDA_TRY(cudaMemsetAsync(G->dstatus, 0, sizeof(DevStatus), st));
  const bool tc = R != nullptr && n >= 1024;
  IBMI_TRY(invariants_all(G, A, lda, false, st, tc, R));
  if (tc) IBMI_TRY(refine_block_inverse(R, G->bat_R, n, n, G->pool, st));
  return copy_square(T0, ldt, G->pool, n, n, st);
}

ibmi_status schur_guess_launch(ibmi_plan_s* P, const double* A, int64_t lda, double* H, int64_t ldh,
                               cudaStream_t st, RefineState* R) {
  IBMI_TRY(set_identity(H, ldh, P->d.p, st));
  if (!P->guess) return IBMI_OK;
  const int64_t lo = P->guess->lo[0];
  return schur_guess_block(P, A, lda, H + lo * ldh + lo, ldh, st, R);
}

double schur_guess_flops(const ibmi_plan_s* P) {
  if (!P->guess) return 0.0;
  const double n = (double)P->guess->mmax;
  return n * n * n / 3.0 + 2.0 * n * n * n;
}

ibmi_status schur_guess_status(ibmi_plan_s* P, cudaStream_t st, ibmi_result* res) {
  if (!P->guess) return IBMI_OK;
  DevStatus hs;
  IBMI_CUDA_TRY(cudaMemcpyAsync(&hs, P->guess->dstatus, sizeof(hs), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs.code == IBMI_ERR_NOT_SPD) {
    res->bad_block = (int32_t)P->lo.size();   // the complement block of the initial guess
    res->bad_pivot = hs.pivot;
    return IBMI_ERR_NOT_SPD;
  }
  return IBMI_OK;
}

}  // namespace ibmi
