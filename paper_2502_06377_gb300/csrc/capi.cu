// C ABI entry points (include/ibmi.h): plan validation and workspace,
// Algorithm 1 driver (sweep loop, stop test, Newton-Schulz tail), residual.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>

#include "gemm_f64.cuh"
#include "mixed.cuh"
#include "plan.cuh"
#include "refine.cuh"

namespace ibmi {

static thread_local std::string g_last_error;
void set_last_error(const std::string& s) { g_last_error = s; }

// Default layout of the sets (Section 4): cores [floor(k p/K), floor((k+1) p/K)),
// widened by h on each side with a neighbour.
static void default_sets(int64_t p, int32_t K, int64_t h, std::vector<int64_t>& lo,
                         std::vector<int64_t>& hi) {
  lo.resize(K);
  hi.resize(K);
  for (int32_t k = 0; k < K; ++k) {
    int64_t b0 = (int64_t)k * p / K, b1 = (int64_t)(k + 1) * p / K;
    lo[k] = std::max<int64_t>(0, b0 - h);
    hi[k] = std::min<int64_t>(p, b1 + h);
  }
}

static ibmi_status validate_sets(int64_t p, const std::vector<int64_t>& lo, const std::vector<int64_t>& hi) {
  const size_t K = lo.size();
  if (K == 0 || hi.size() != K) return IBMI_ERR_INVALID_ARG;
  if (lo[0] != 0 || hi[K - 1] != p) return IBMI_ERR_INVALID_ARG;
  for (size_t k = 0; k < K; ++k) {
    if (!(lo[k] >= 0 && lo[k] < hi[k] && hi[k] <= p)) return IBMI_ERR_INVALID_ARG;
    if (K > 1 && hi[k] - lo[k] >= p) return IBMI_ERR_INVALID_ARG;   // empty complement
    if (k > 0) {
      if (!(lo[k] > lo[k - 1] && hi[k] > hi[k - 1])) return IBMI_ERR_INVALID_ARG;
      if (lo[k] > hi[k - 1]) return IBMI_ERR_INVALID_ARG;            // gap: not covered
    }
  }
  return IBMI_OK;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == dev;   // another GPU's memory would be a peer access or a fault
}

static double flops_sweep(const ibmi_plan_s* P) {
  double f = 0;
  for (size_t k = 0; k < P->lo.size(); ++k) {
    double m = (double)(P->hi[k] - P->lo[k]), n = (double)P->d.p - m;
    f += 2.0 * m * n * n + 2.0 * m * m * n;
  }
  return f;
}

static double flops_plan(const ibmi_plan_s* P) {
  double f = 0;
  for (size_t k = 0; k < P->lo.size(); ++k) {
    double m = (double)(P->hi[k] - P->lo[k]), n = (double)P->d.p - m;
    f += m * m * m / 3.0 + 2.0 * m * m * m + 2.0 * m * m * n;
  }
  return f;
}

static ibmi_status ensure_ns_buffers(ibmi_plan_s* P) {
  if (P->nsR) return IBMI_OK;
  const size_t b = sizeof(double) * (size_t)P->d.p * P->d.p;
  IBMI_CUDA_TRY(cudaMalloc(&P->nsR, b));
  IBMI_CUDA_TRY(cudaMalloc(&P->nsX, b));
  return IBMI_OK;
}

// Reads rho_F computed on the device (syncs the stream).
static ibmi_status residual_host(ibmi_plan_s* P, const double* A, int64_t lda, const double* H,
                                 int64_t ldh, cudaStream_t st, double* rho) {
  IBMI_TRY(residual_f64_dev(A, lda, H, ldh, P->d.p, P->partials, P->n_partials, P->dscalar, st));
  double v[2];
  IBMI_CUDA_TRY(cudaMemcpyAsync(v, P->dscalar, sizeof(v), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  *rho = v[0];
  return IBMI_OK;
}

static ibmi_status invert_impl(ibmi_plan_s* P, const double* A, int64_t lda, double* H, int64_t ldh,
                               cudaStream_t st, ibmi_result* res) {
  const int64_t p = P->d.p;
  const int K = (int)P->lo.size();
  const ibmi_plan_desc& d = P->d;
  const double sqrtp = sqrt((double)p);
  double flops = 0.0;
  // only A's lower triangle is read: the solve runs on its symmetric copy
  IBMI_TRY(sym_from_lower(A, lda, p, P->dAs, p, st));
  A = P->dAs;
  lda = p;
  // one set is the whole matrix: H = A^{-1} from the FP64 block inverse,
  // whatever the precision
  const bool mixed = d.precision == IBMI_MIXED && K > 1;
  if (mixed) {
    ibmi_status s = mixed_run(P, A, lda, H, ldh, st, res, &flops);
    res->flops = flops;
    return s;
  }
  // a2: invariants
  IBMI_CUDA_TRY(cudaMemsetAsync(P->dstatus, 0, sizeof(DevStatus), st));
  IBMI_TRY(invariants_all(P, A, lda, K > 1, st));   // one set needs no W (its sweep sets H = A^{-1})
  flops += flops_plan(P);
  DevStatus hs;
  IBMI_CUDA_TRY(cudaMemcpyAsync(&hs, P->dstatus, sizeof(hs), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs.code == IBMI_ERR_NOT_SPD) {
    res->bad_block = hs.block;
    res->bad_pivot = hs.pivot;
    return IBMI_ERR_NOT_SPD;
  }
  if (d.init == IBMI_INIT_IDENTITY) IBMI_TRY(set_identity(H, ldh, p, st));
  if (d.init == IBMI_INIT_SCHUR) {
    IBMI_TRY(schur_guess_launch(P, A, lda, H, ldh, st, nullptr));
    IBMI_TRY(schur_guess_status(P, st, res));
    flops += schur_guess_flops(P);
  }
  // Algorithm 1: sweeps with the stop test every check_every sweeps
  ibmi_status status = IBMI_NOT_CONVERGED;
  bool to_ns = false;
  int r = 0;
  const double fs = flops_sweep(P), fr = 2.0 * (double)p * p * p;
  CheckCadence cad;
  cad.gmin = cad.next = d.check_every;
  const double target = d.ns_theta > 0.0 ? std::max(d.tol, d.ns_theta / sqrtp) : d.tol;
  while (true) {
    ++r;
    for (int k = 0; k < K; ++k) IBMI_TRY(sweep_step_f64(P, k, H, ldh, st));
    flops += fs;
    res->sweeps = r;
    if (r < cad.next && r < d.max_sweeps) continue;
    if (d.stop_rule == IBMI_STOP_PAPER_EST) {
      // eq. error on the last set; the residual is evaluated once at the end
      double e;
      IBMI_TRY(paper_estimate_f64(P, A, lda, H, ldh, st, &e));
      res->paper_est = e;
      cad.next = r + d.check_every;
      if (!isfinite(e)) { status = IBMI_ERR_NONFINITE; break; }
      if (e <= d.tol || r >= d.max_sweeps) {
        double rho;
        IBMI_TRY(residual_host(P, A, lda, H, ldh, st, &rho));
        flops += fr;
        res->resid_f = rho;
        status = e <= d.tol ? IBMI_OK : IBMI_NOT_CONVERGED;
        break;
      }
      continue;
    }
    double rho;
    IBMI_TRY(residual_host(P, A, lda, H, ldh, st, &rho));
    flops += fr;
    res->resid_f = rho;
    if (!isfinite(rho)) { status = IBMI_ERR_NONFINITE; break; }
    if (rho <= d.tol) { status = IBMI_OK; break; }
    if (d.ns_theta > 0.0 && rho * sqrtp <= d.ns_theta) { to_ns = true; break; }
    if (r >= d.max_sweeps) break;
    cad.after(r, rho, target);
  }
  if (to_ns) {
    IBMI_TRY(ensure_ns_buffers(P));
    status = IBMI_NOT_CONVERGED;
    double prev = res->resid_f;
    for (int s = 0; s < d.ns_max; ++s) {
      IBMI_TRY(ns_step_f64(P, A, lda, H, ldh, st, P->nsR));   // nsR keeps the iterate before the step
      flops += 2.0 * fr;
      double rho;
      IBMI_TRY(residual_host(P, A, lda, H, ldh, st, &rho));
      flops += fr;
      res->ns_steps = s + 1;
      if (!(rho < prev)) {
        // a step that does not reduce the residual (or overflows) ends the
        // tail, and H goes back to the better iterate before it
        IBMI_TRY(copy_square(H, ldh, P->nsR, p, p, st));
        break;
      }
      res->resid_f = rho;
      if (rho <= d.tol) { status = IBMI_OK; break; }
      prev = rho;
    }
  }
  res->flops = flops;
  return status;
}

}  // namespace ibmi

using namespace ibmi;

extern "C" {

void ibmi_plan_desc_init(ibmi_plan_desc* d) {
  if (!d) return;
  memset(d, 0, sizeof(*d));
  d->K = 2;
  d->h = 0;
  d->precision = IBMI_FP64;
  d->tol = 1e-10;
  d->max_sweeps = 500;
  d->stop_rule = IBMI_STOP_RESID_F;
  d->check_every = 1;
  d->ns_theta = 0.0;
  d->ns_max = 8;
  d->init = IBMI_INIT_IDENTITY;
}

ibmi_status ibmi_plan(const ibmi_plan_desc* desc, ibmi_plan_t* out) {
  if (!desc || !out) return IBMI_ERR_INVALID_ARG;
  *out = nullptr;
  const ibmi_plan_desc& d = *desc;
  if (d.p < 2 || d.K < 1 || d.K > d.p || d.h < 0) return IBMI_ERR_INVALID_ARG;
  if (d.p > (int64_t)1 << 20) return IBMI_ERR_INVALID_ARG;
  if (d.precision != IBMI_FP64 && d.precision != IBMI_MIXED) return IBMI_ERR_INVALID_ARG;
  if (d.stop_rule != IBMI_STOP_RESID_F && d.stop_rule != IBMI_STOP_PAPER_EST) return IBMI_ERR_INVALID_ARG;
  if (d.stop_rule == IBMI_STOP_PAPER_EST && d.precision == IBMI_MIXED) {
    set_last_error("the paper's estimate is offered as stop rule on the FP64 path only");
    return IBMI_ERR_INVALID_ARG;
  }
  if (d.init != IBMI_INIT_IDENTITY && d.init != IBMI_INIT_USER && d.init != IBMI_INIT_SCHUR)
    return IBMI_ERR_INVALID_ARG;
  if (d.max_sweeps < 1 || d.check_every < 1 || d.ns_max < 0 || !(d.tol >= 0.0) || !(d.ns_theta >= 0.0))
    return IBMI_ERR_INVALID_ARG;
  ibmi_plan_s* P = new ibmi_plan_s();
  P->d = d;
  P->d.lo = P->d.hi = nullptr;
  if (d.lo || d.hi) {
    if (!d.lo || !d.hi) { delete P; return IBMI_ERR_INVALID_ARG; }
    P->lo.assign(d.lo, d.lo + d.K);
    P->hi.assign(d.hi, d.hi + d.K);
  } else {
    default_sets(d.p, d.K, d.h, P->lo, P->hi);
  }
  if (validate_sets(d.p, P->lo, P->hi) != IBMI_OK) { delete P; return IBMI_ERR_INVALID_ARG; }
  cudaGetDevice(&P->device);
  const int64_t p = d.p;
  int64_t mmax = 0, ainv_elems = 0, w_elems = 0;
  for (int k = 0; k < d.K; ++k) {
    int64_t m = P->hi[k] - P->lo[k];
    mmax = std::max(mmax, m);
    ainv_elems += m * m;
    w_elems += m * p;
  }
  P->mmax = mmax;
  P->n_partials = gemm_f64_ctas(p, p);
  const bool mixed = d.precision == IBMI_MIXED;
  if (mixed) w_elems = 0;   // the mixed path keeps W only as BF16 slices
  const int64_t scratch = mmax * mmax /*S*/ + P->n_partials + 4;
  const size_t total = sizeof(double) * (size_t)(ainv_elems + w_elems + scratch);
  if (cudaMalloc(&P->pool, total) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return IBMI_ERR_OOM;
  }
  P->pool_bytes = total;
  if (cudaMalloc(&P->dAs, sizeof(double) * (size_t)d.p * d.p) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(P->pool);
    delete P;
    return IBMI_ERR_OOM;
  }
  double* q = P->pool;
  std::vector<int64_t> hoff_ainv(d.K), hoff_w(d.K, 0), hm(d.K);
  for (int k = 0; k < d.K; ++k) {
    int64_t m = P->hi[k] - P->lo[k];
    hm[k] = m;
    hoff_ainv[k] = q - P->pool;
    P->ainv.push_back(q); q += m * m;
  }
  for (int k = 0; k < d.K; ++k) {
    int64_t m = P->hi[k] - P->lo[k];
    if (mixed) { P->w.push_back(nullptr); continue; }
    hoff_w[k] = q - P->pool;
    P->w.push_back(q); q += m * p;
  }
  P->S = q; q += mmax * mmax;
  P->partials = q; q += P->n_partials;
  P->dscalar = q; q += 4;
  // batched factorisation scratch
  const int64_t ncols = mixed ? mmax : p;
  const size_t bat_doubles = (size_t)d.K * (mmax * mmax + mmax * ncols + mmax * CHOL_NB);
  if (cudaMalloc(&P->bat_pool, sizeof(double) * bat_doubles + sizeof(int64_t) * 4 * d.K) != cudaSuccess ||
      cudaMalloc(&P->dstatus, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    ibmi_plan_destroy(P);
    return IBMI_ERR_OOM;
  }
  double* b = (double*)P->bat_pool;
  P->bat_L = b; b += d.K * mmax * mmax;
  P->bat_R = b; b += d.K * mmax * ncols;
  P->bat_linv = b; b += d.K * mmax * CHOL_NB;
  int64_t* ib = (int64_t*)b;
  P->dlo = ib; P->dm = ib + d.K; P->doff_ainv = ib + 2 * d.K; P->doff_w = ib + 3 * d.K;
  std::vector<int64_t> packed;
  packed.insert(packed.end(), P->lo.begin(), P->lo.end());
  packed.insert(packed.end(), hm.begin(), hm.end());
  packed.insert(packed.end(), hoff_ainv.begin(), hoff_ainv.end());
  packed.insert(packed.end(), hoff_w.begin(), hoff_w.end());
  if (cudaMemcpy(ib, packed.data(), sizeof(int64_t) * packed.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    ibmi_plan_destroy(P);
    return IBMI_ERR_CUDA;
  }
  if (d.precision == IBMI_MIXED && P->lo.size() > 1) {   // one set: the FP64 block inverse is H
    ibmi_status s = mixed_create(P);
    if (s != IBMI_OK) { ibmi_plan_destroy(P); return s; }
  }
  if (d.init == IBMI_INIT_SCHUR) {
    ibmi_status s = schur_guess_create(P);
    if (s != IBMI_OK) { ibmi_plan_destroy(P); return s; }
  }
  *out = P;
  return IBMI_OK;
}

ibmi_status ibmi_plan_destroy(ibmi_plan_t P) {
  if (!P) return IBMI_ERR_INVALID_ARG;
  if (P->mixed) mixed_destroy(P);
  schur_guess_destroy(P);
  cudaFree(P->bdX);
  cudaFree(P->bdRows);
  cudaFree(P->pool);
  cudaFree(P->bat_pool);
  cudaFree(P->dstatus);
  cudaFree(P->nsR);
  cudaFree(P->nsX);
  cudaFree(P->pe);
  cudaFree(P->dA);
  cudaFree(P->dAs);
  cudaFree(P->dH);
  delete P;
  return IBMI_OK;
}

ibmi_status ibmi_plan_sets(ibmi_plan_t P, int32_t* K, int64_t* lo, int64_t* hi) {
  if (!P) return IBMI_ERR_INVALID_ARG;
  if (K) *K = (int32_t)P->lo.size();
  for (size_t k = 0; k < P->lo.size(); ++k) {
    if (lo) lo[k] = P->lo[k];
    if (hi) hi[k] = P->hi[k];
  }
  return IBMI_OK;
}

ibmi_status ibmi_invert(ibmi_plan_t P, const double* A, int64_t lda, double* H, int64_t ldh,
                        void* stream, ibmi_result* out) {
  ibmi_result tmp;
  ibmi_result* res = out ? out : &tmp;
  memset(res, 0, sizeof(*res));
  res->bad_block = -1;
  res->bad_pivot = -1;
  res->resid_f = NAN;
  res->paper_est = NAN;
  ibmi_status s;
  if (!P || !A || !H || lda < P->d.p || ldh < P->d.p) {
    s = IBMI_ERR_INVALID_ARG;
  } else if (!is_device_ptr(A) || !is_device_ptr(H)) {
    s = IBMI_ERR_INVALID_ARG;
  } else {
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    s = invert_impl(P, A, lda, H, ldh, st, res);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && s == IBMI_OK) { set_last_error(cudaGetErrorString(e)); s = IBMI_ERR_CUDA; }
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  res->status = s;
  return s;
}

ibmi_status ibmi_invert_host(ibmi_plan_t P, const double* A_host, int64_t lda, double* H_host, int64_t ldh,
                             void* stream, ibmi_result* out) {
  if (!P || !A_host || !H_host || lda < P->d.p || ldh < P->d.p) return IBMI_ERR_INVALID_ARG;
  const int64_t p = P->d.p;
  const size_t row = sizeof(double) * p;
  cudaStream_t st = (cudaStream_t)stream;
  if (!P->dA) {
    IBMI_CUDA_TRY(cudaMalloc(&P->dA, row * p));
    IBMI_CUDA_TRY(cudaMalloc(&P->dH, row * p));
  }
  auto t0 = std::chrono::steady_clock::now();
  IBMI_CUDA_TRY(cudaMemcpy2DAsync(P->dA, row, A_host, sizeof(double) * lda, row, p, cudaMemcpyHostToDevice, st));
  if (P->d.init == IBMI_INIT_USER)
    IBMI_CUDA_TRY(cudaMemcpy2DAsync(P->dH, row, H_host, sizeof(double) * ldh, row, p, cudaMemcpyHostToDevice, st));
  ibmi_status s = ibmi_invert(P, P->dA, p, P->dH, p, stream, out);
  if (s == IBMI_OK || s == IBMI_NOT_CONVERGED) {
    IBMI_CUDA_TRY(cudaMemcpy2DAsync(H_host, sizeof(double) * ldh, P->dH, row, row, p, cudaMemcpyDeviceToHost, st));
    IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (out) out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

ibmi_status ibmi_residual(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                          void* stream, double* out) {
  if (!A || !H || !out || p < 1 || lda < p || ldh < p) return IBMI_ERR_INVALID_ARG;
  if (!is_device_ptr(A) || !is_device_ptr(H)) return IBMI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = gemm_f64_ctas(p, p);
  double* buf = nullptr;
  IBMI_CUDA_TRY(cudaMallocAsync(&buf, sizeof(double) * (n + 2 + p * p), st));
  double* As = buf + n + 2;   // A from its lower triangle
  ibmi_status s = sym_from_lower(A, lda, p, As, p, st);
  if (s == IBMI_OK) s = residual_f64_dev(As, p, H, ldh, p, buf, n, buf + n, st);
  double v[2] = {NAN, NAN};
  if (s == IBMI_OK) {
    cudaMemcpyAsync(v, buf + n, sizeof(v), cudaMemcpyDeviceToHost, st);
  }
  cudaFreeAsync(buf, st);
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  *out = v[0];
  return s;
}

ibmi_status ibmi_residual_tc(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                             void* stream, double* out) {
  if (!A || !H || !out || p < 1 || lda < p || ldh < p || p > (int64_t)1 << 16) return IBMI_ERR_INVALID_ARG;
  if (!is_device_ptr(A) || !is_device_ptr(H)) return IBMI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  IBMI_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
  IBMI_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  double* As = nullptr;   // A from its lower triangle
  if (cudaMalloc(&As, sizeof(double) * p * p) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(err);
    return IBMI_ERR_OOM;
  }
  RefineState R;
  ibmi_status s = sym_from_lower(A, lda, p, As, p, st);
  if (s == IBMI_OK) s = refine_create(&R, p, err);
  if (s == IBMI_OK) s = refine_set_matrix(&R, As, p, st);
  if (s == IBMI_OK) s = refine_residual(&R, H, ldh, st, out);
  cudaStreamSynchronize(st);
  refine_destroy(&R);
  cudaFree(As);
  cudaFree(err);
  return s;
}

ibmi_status ibmi_refine(const double* A, int64_t lda, double* X, int64_t ldx, int64_t p, int32_t precision,
                        double tol, int32_t ns_max, void* stream, ibmi_result* out) {
  ibmi_result tmp;
  ibmi_result* res = out ? out : &tmp;
  memset(res, 0, sizeof(*res));
  res->bad_block = -1;
  res->bad_pivot = -1;
  res->resid_f = NAN;
  res->paper_est = NAN;
  if (!A || !X || p < 2 || lda < p || ldx < p || p > (int64_t)1 << 16 || ns_max < 0 || !(tol >= 0.0) ||
      (precision != IBMI_FP64 && precision != IBMI_MIXED))
    return (ibmi_status)(res->status = IBMI_ERR_INVALID_ARG);
  if (!is_device_ptr(A) || !is_device_ptr(X)) return (ibmi_status)(res->status = IBMI_ERR_INVALID_ARG);
  cudaStream_t st = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  const double fr = 2.0 * (double)p * p * p;
  ibmi_status s = IBMI_NOT_CONVERGED;
  double* As = nullptr;   // A from its lower triangle
  if (cudaMalloc(&As, sizeof(double) * p * p) != cudaSuccess) {
    cudaGetLastError();
    return (ibmi_status)(res->status = IBMI_ERR_OOM);
  }
  struct FreeOnExit {
    double* q;
    ~FreeOnExit() { cudaFree(q); }   // synchronises the device first
  } keep{As};
  {
    const ibmi_status e = sym_from_lower(A, lda, p, As, p, st);
    if (e != IBMI_OK) return (ibmi_status)(res->status = e);
  }
  A = As;
  lda = p;
  if (precision == IBMI_MIXED) {
    int* err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return (ibmi_status)(res->status = IBMI_ERR_OOM);
    }
    struct FreeWord {
      int* q;
      ~FreeWord() { cudaFree(q); }   // after refine_destroy below (reverse order of scope)
    } keep_err{err};
    IBMI_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    RefineState R;
    s = refine_create(&R, p, err);
    if (s == IBMI_OK) s = refine_set_matrix(&R, A, lda, st);
    double* Xprev = nullptr;   // X before the last update
    if (s == IBMI_OK && ns_max > 0 && cudaMalloc(&Xprev, sizeof(double) * p * p) != cudaSuccess) {
      cudaGetLastError();
      s = IBMI_ERR_OOM;
    }
    double prev = INFINITY;
    for (int it = 0; s == IBMI_OK; ++it) {
      double rho;
      s = refine_residual(&R, X, ldx, st, &rho);
      if (s != IBMI_OK) break;
      res->flops += fr;
      if (it > 0 && !(rho < prev)) {   // the last update did not help: undo it
        s = copy_square(X, ldx, Xprev, p, p, st);
        if (s == IBMI_OK) s = IBMI_NOT_CONVERGED;
        break;
      }
      res->resid_f = rho;
      if (!isfinite(rho)) { s = IBMI_ERR_NONFINITE; break; }
      if (rho <= tol) { s = IBMI_OK; break; }
      if (it >= ns_max) { s = IBMI_NOT_CONVERGED; break; }
      prev = rho;
      s = refine_ns_update(&R, X, ldx, st, NS_S - 1, Xprev);
      res->flops += fr;
      res->ns_steps = it + 1;
    }
    cudaStreamSynchronize(st);
    cudaFree(Xprev);
    refine_destroy(&R);
  } else {
    ibmi_plan_s P;
    P.d.p = p;
    P.n_partials = gemm_f64_ctas(p, p);
    const size_t b = sizeof(double) * (size_t)p * p;
    struct FreeBuffers {   // the three buffers below, also on an early return
      ibmi_plan_s* P;
      ~FreeBuffers() {
        cudaFree(P->nsR);
        cudaFree(P->nsX);
        cudaFree(P->partials);
        P->nsR = P->nsX = nullptr;
        P->partials = nullptr;
      }
    } keep_bufs{&P};
    if (cudaMalloc(&P.nsR, b) != cudaSuccess || cudaMalloc(&P.nsX, b) != cudaSuccess ||
        cudaMalloc(&P.partials, sizeof(double) * (P.n_partials + 4)) != cudaSuccess) {
      cudaGetLastError();
      return (ibmi_status)(res->status = IBMI_ERR_OOM);
    }
    P.dscalar = P.partials + P.n_partials;
    double prev = INFINITY;
    for (int it = 0;; ++it) {
      double rho;
      s = residual_host(&P, A, lda, X, ldx, st, &rho);
      if (s != IBMI_OK) break;
      res->flops += fr;
      if (it > 0 && !(rho < prev)) {   // the last step did not help: undo it (nsR holds X before it)
        s = copy_square(X, ldx, P.nsR, p, p, st);
        if (s == IBMI_OK) s = IBMI_NOT_CONVERGED;
        break;
      }
      res->resid_f = rho;
      if (!isfinite(rho)) { s = IBMI_ERR_NONFINITE; break; }
      if (rho <= tol) { s = IBMI_OK; break; }
      if (it >= ns_max) { s = IBMI_NOT_CONVERGED; break; }
      prev = rho;
      s = ns_step_f64(&P, A, lda, X, ldx, st, P.nsR);
      if (s != IBMI_OK) break;
      res->flops += 2.0 * fr;
      res->ns_steps = it + 1;
    }
    cudaStreamSynchronize(st);
  }
  res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  res->status = s;
  return s;
}

const char* ibmi_status_string(ibmi_status s) {
  switch (s) {
    case IBMI_OK: return "IBMI_OK";
    case IBMI_ERR_INVALID_ARG: return "IBMI_ERR_INVALID_ARG";
    case IBMI_ERR_NOT_SPD: return "IBMI_ERR_NOT_SPD";
    case IBMI_NOT_CONVERGED: return "IBMI_NOT_CONVERGED";
    case IBMI_ERR_NONFINITE: return "IBMI_ERR_NONFINITE";
    case IBMI_ERR_BUDGET: return "IBMI_ERR_BUDGET";
    case IBMI_ERR_OOM: return "IBMI_ERR_OOM";
    case IBMI_ERR_TIMEOUT: return "IBMI_ERR_TIMEOUT";
    case IBMI_ERR_CUDA: return "IBMI_ERR_CUDA";
    case IBMI_NOT_READY: return "IBMI_NOT_READY";
    case IBMI_ERR_CANCELLED: return "IBMI_ERR_CANCELLED";
  }
  return "IBMI_UNKNOWN";
}

const char* ibmi_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ------------------------------------------------------------- profiling --
#include <atomic>
#include <mutex>
namespace ibmi {
namespace {
struct ProfClass {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  int64_t launches = 0;
  double flops = 0.0;
  double alg = 0.0;
  double ms = 0.0;
};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;                    // guards g_prof and the event pool
ProfClass g_prof[IBMI_K_COUNT];
std::vector<cudaEvent_t> g_event_pool;
std::atomic<int64_t> g_launches{0};
// Open scopes, innermost last (per thread: one stream each).  A scope opened
// inside another pauses it, so every interval of device time goes to one
// class only.
struct OpenScope {
  int k;
  cudaEvent_t ev;
};
thread_local std::vector<OpenScope> g_open;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool prof_on() { return g_prof_on.load(std::memory_order_relaxed); }

void prof_begin(int k, cudaStream_t st) {
  if (!g_prof_on.load(std::memory_order_relaxed) || k < 0 || k >= IBMI_K_COUNT) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_open.empty() && g_open.back().ev) {   // pause the enclosing scope
    cudaEvent_t e = take_event();
    cudaEventRecord(e, st);
    g_prof[g_open.back().k].ev.emplace_back(g_open.back().ev, e);
    g_open.back().ev = nullptr;
  }
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  g_open.push_back(OpenScope{k, e});
}

void prof_end(int k, cudaStream_t st, double flops, double alg) {
  if (g_open.empty() || g_open.back().k != k) return;
  if (!g_prof_on.load(std::memory_order_relaxed)) {   // turned off inside the scope
    g_open.pop_back();
    return;
  }
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  if (g_open.back().ev) g_prof[k].ev.emplace_back(g_open.back().ev, e);
  g_prof[k].launches += 1;
  g_prof[k].flops += flops;
  g_prof[k].alg += alg;
  g_open.pop_back();
  if (!g_open.empty()) {   // resume the enclosing scope
    cudaEvent_t r = take_event();
    cudaEventRecord(r, st);
    g_open.back().ev = r;
  }
}
}  // namespace ibmi

extern "C" {
void ibmi_prof_enable(int on) {
  using namespace ibmi;
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto& c : g_prof) {
    for (auto& pr : c.ev) {
      cudaEventSynchronize(pr.second);
      g_event_pool.push_back(pr.first);
      g_event_pool.push_back(pr.second);
    }
    c = ProfClass();
  }
  g_launches.store(0);
  g_prof_on.store(on != 0);
}

ibmi_status ibmi_prof_get(int32_t k, int64_t* launches, double* ms, double* flops) {
  using namespace ibmi;
  if (k < 0 || k >= IBMI_K_COUNT) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_prof_mu);
  ProfClass& c = g_prof[k];
  for (auto& pr : c.ev) {
    float t = 0.f;
    cudaEventSynchronize(pr.second);
    if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) c.ms += t;
    g_event_pool.push_back(pr.first);
    g_event_pool.push_back(pr.second);
  }
  c.ev.clear();
  if (launches) *launches = c.launches;
  if (ms) *ms = c.ms;
  if (flops) *flops = c.flops;
  return IBMI_OK;
}

ibmi_status ibmi_prof_get_alg(int32_t k, double* alg_flops) {
  using namespace ibmi;
  if (k < 0 || k >= IBMI_K_COUNT || !alg_flops) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_prof_mu);
  *alg_flops = g_prof[k].alg;
  return IBMI_OK;
}

int64_t ibmi_launch_count(void) { return ibmi::g_launches.load(); }
}  // extern "C"
