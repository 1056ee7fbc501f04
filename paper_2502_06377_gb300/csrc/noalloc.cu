// ibmi_residual_noalloc: the FP64 residual ||I - A H||_F / sqrt(p) without
// any device allocation, for callers that must not allocate (see ibmi.h).
//
// The per-tile partial sums and the two result scalars live in a file-scope
// device array of fixed size.  Host code cannot use the array's name as a
// device address, so the address is looked up once per device with
// cudaGetSymbolAddress and then passed to the kernels.
#include <mutex>

#include "gemm_f64.cuh"
#include "plan.cuh"

namespace ibmi {

// ceil(p / 64)^2 tile partials (orders up to 8192) plus rho and the raw sum.
constexpr int64_t NOALLOC_MAX_P = 8192;
constexpr int64_t NOALLOC_PARTIALS = (NOALLOC_MAX_P / F64_BM) * (NOALLOC_MAX_P / F64_BN);
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_PARTIALS + 2];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device (looked up on the
// first call for that device).
static ibmi_status noalloc_scratch(double** out) {
  int dev = 0;
  IBMI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return IBMI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    IBMI_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_addr[dev] = (double*)ptr;
  }
  *out = g_noalloc_addr[dev];
  return IBMI_OK;
}

}  // namespace ibmi

extern "C" ibmi_status ibmi_residual_noalloc(const double* A, int64_t lda, const double* H, int64_t ldh, int64_t p,
                                             void* stream, double* out) {
  using namespace ibmi;
  if (!A || !H || !out || p < 1 || lda < p || ldh < p) return IBMI_ERR_INVALID_ARG;
  if (p > NOALLOC_MAX_P) {
    set_last_error("ibmi_residual_noalloc: order exceeds the fixed scratch (p <= 8192)");
    return IBMI_ERR_INVALID_ARG;
  }
  if (!is_device_ptr(A) || !is_device_ptr(H)) return IBMI_ERR_INVALID_ARG;
  double* scratch = nullptr;
  IBMI_TRY(noalloc_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = gemm_f64_ctas(p, p);   // <= NOALLOC_PARTIALS; each call writes every partial it reads
  // A is read from its lower triangle, like every other entry point
  IBMI_TRY(residual_f64_dev(A, lda, H, ldh, p, scratch, n, scratch + NOALLOC_PARTIALS, st, true));
  double v = 0.0;
  IBMI_CUDA_TRY(cudaMemcpyAsync(&v, scratch + NOALLOC_PARTIALS, sizeof(double), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  *out = v;
  return IBMI_OK;
}
