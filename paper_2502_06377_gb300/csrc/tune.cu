// Partition and ordering search for one matrix (ibmi_tune), the point
// orderings it searches over (ibmi_order_points) and the symmetric
// permutation of a matrix on the device (ibmi_permute).
//
// Section 5.4 (Tables 3-4) finds the overlap of the sets decisive for
// convergence and the number of sets less so; Section 5.7 finds the ordering
// of the rows decisive too (contiguous sets over an ordering that keeps the
// weight near the diagonal converge, a red-black ordering of the same matrix
// does not), and the closing discussion of Section 5 recommends orderings
// that concentrate the matrix near its diagonal.  The orderings below are
// computed from point coordinates, for covariance matrices of point sets.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "plan.cuh"

namespace ibmi {

// --------------------------------------------------------------- orders ----

// Hilbert index of integer coordinates x[0..dim) in [0, 2^bits) by Skilling's
// transform ("Programming the Hilbert curve", AIP Conf. Proc. 707, 2004):
// undo the excess work of the axes from the top bit down, Gray-encode, then
// interleave the bits (top bit of axis 0 first).
static uint64_t hilbert_index(std::vector<uint32_t> x, int bits) {
  const int n = (int)x.size();
  const uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    const uint32_t P = Q - 1;
    for (int i = 0; i < n; ++i) {
      if (x[i] & Q) {
        x[0] ^= P;                      // invert the low bits of axis 0
      } else {
        const uint32_t t = (x[0] ^ x[i]) & P;   // exchange the low bits of axes 0 and i
        x[0] ^= t;
        x[i] ^= t;
      }
    }
  }
  for (int i = 1; i < n; ++i) x[i] ^= x[i - 1];   // Gray encode
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (x[n - 1] & Q) t ^= Q - 1;
  for (int i = 0; i < n; ++i) x[i] ^= t;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < n; ++i) h = (h << 1) | ((x[i] >> b) & 1u);
  return h;
}

// k-d order: split [b, e) at its median across the coordinate of widest
// spread (ties by index), recursively; the leaves left to right.
static void kd_order(const double* pts, int dim, std::vector<int64_t>& idx, int64_t b, int64_t e) {
  if (e - b <= 1) return;
  int best = 0;
  double spread = -1.0;
  for (int d = 0; d < dim; ++d) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t k = b; k < e; ++k) {
      lo = std::min(lo, pts[idx[k] * dim + d]);
      hi = std::max(hi, pts[idx[k] * dim + d]);
    }
    if (hi - lo > spread) { spread = hi - lo; best = d; }
  }
  const int64_t mid = b + (e - b) / 2;
  std::nth_element(idx.begin() + b, idx.begin() + mid, idx.begin() + e, [&](int64_t u, int64_t v) {
    const double a = pts[u * dim + best], c = pts[v * dim + best];
    return a < c || (a == c && u < v);
  });
  kd_order(pts, dim, idx, b, mid);
  kd_order(pts, dim, idx, mid, e);
}

// ----------------------------------------------------------- permutation --

// B[i][j] = S[q[i]][q[j]] with S the symmetric matrix whose lower triangle is
// A's (element (r, c) read from (max, min)); q on the device.
__global__ void k_sym_gather(const double* A, int64_t lda, int64_t p, const int64_t* q, double* B, int64_t ldb) {
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  int64_t r = q[i], c = q[j];
  if (c > r) {
    const int64_t t = r;
    r = c;
    c = t;
  }
  B[i * ldb + j] = A[r * lda + c];
}

static ibmi_status gather(const double* A, int64_t lda, int64_t p, const int64_t* dq, double* B, int64_t ldb,
                          cudaStream_t st) {
  note_launch();
  k_sym_gather<<<dim3((unsigned)((p + 255) / 256), (unsigned)p), 256, 0, st>>>(A, lda, p, dq, B, ldb);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

}  // namespace ibmi

using namespace ibmi;

extern "C" ibmi_status ibmi_order_points(const double* pts, int64_t n, int32_t dim, int32_t order, int64_t* perm) {
  if (!pts || !perm || n < 1 || dim < 1 || dim > 16) return IBMI_ERR_INVALID_ARG;
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  switch (order) {
    case IBMI_ORDER_IDENTITY:
      break;
    case IBMI_ORDER_XSORT:
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t u, int64_t v) { return pts[u * dim] < pts[v * dim]; });
      break;
    case IBMI_ORDER_HILBERT: {
      const int bits = std::max(1, std::min(20, 62 / dim));
      std::vector<double> lo(dim, INFINITY), hi(dim, -INFINITY);
      for (int64_t k = 0; k < n; ++k)
        for (int d = 0; d < dim; ++d) {
          lo[d] = std::min(lo[d], pts[k * dim + d]);
          hi[d] = std::max(hi[d], pts[k * dim + d]);
        }
      const double cells = (double)((1u << bits) - 1);
      std::vector<uint64_t> key(n);
      std::vector<uint32_t> x(dim);
      for (int64_t k = 0; k < n; ++k) {
        for (int d = 0; d < dim; ++d) {
          const double w = hi[d] - lo[d];
          const double u = w > 0.0 ? (pts[k * dim + d] - lo[d]) / w : 0.0;
          x[d] = (uint32_t)std::min(cells, std::max(0.0, std::floor(u * cells + 0.5)));
        }
        key[k] = hilbert_index(x, bits);
      }
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t u, int64_t v) { return key[u] < key[v]; });
      break;
    }
    case IBMI_ORDER_KD:
      kd_order(pts, dim, idx, 0, n);
      break;
    case IBMI_ORDER_REDBLACK: {
      int64_t k = 0;
      for (int64_t i = 0; i < n; i += 2) idx[k++] = i;
      for (int64_t i = 1; i < n; i += 2) idx[k++] = i;
      break;
    }
    default:
      return IBMI_ERR_INVALID_ARG;
  }
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(pts[idx[k] * dim])) return IBMI_ERR_INVALID_ARG;
  std::copy(idx.begin(), idx.end(), perm);
  return IBMI_OK;
}

static bool valid_perm(const int64_t* perm, int64_t p) {
  std::vector<char> seen(p, 0);
  for (int64_t i = 0; i < p; ++i) {
    if (perm[i] < 0 || perm[i] >= p || seen[perm[i]]) return false;
    seen[perm[i]] = 1;
  }
  return true;
}

extern "C" ibmi_status ibmi_permute(const double* A, int64_t lda, int64_t p, const int64_t* perm, int32_t inverse,
                                    double* B, int64_t ldb, void* stream) {
  if (!A || !B || !perm || p < 1 || lda < p || ldb < p || A == B) return IBMI_ERR_INVALID_ARG;
  if (!valid_perm(perm, p)) return IBMI_ERR_INVALID_ARG;
  if (!is_device_ptr(A) || !is_device_ptr(B)) return IBMI_ERR_INVALID_ARG;
  std::vector<int64_t> q(perm, perm + p);
  if (inverse)
    for (int64_t i = 0; i < p; ++i) q[perm[i]] = i;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t* dq = nullptr;
  IBMI_CUDA_TRY(cudaMallocAsync(&dq, sizeof(int64_t) * p, st));
  ibmi_status s = IBMI_OK;
  if (cudaMemcpyAsync(dq, q.data(), sizeof(int64_t) * p, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    s = IBMI_ERR_CUDA;
  }
  if (s == IBMI_OK) s = gather(A, lda, p, dq, B, ldb, st);
  cudaFreeAsync(dq, st);
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  return s;
}

extern "C" ibmi_status ibmi_tune(const double* A, int64_t lda, int64_t p, const int64_t* const* perms, int32_t n_perms,
                                 const ibmi_plan_desc* base, void* stream, ibmi_tune_candidate* best,
                                 ibmi_tune_candidate* all, int32_t max_all, int32_t* n_all) {
  if (!A || !base || !best || p < 2 || lda < p || n_perms < 0 || (n_perms > 0 && !perms) || max_all < 0 ||
      (max_all > 0 && !all))
    return IBMI_ERR_INVALID_ARG;
  for (int32_t o = 0; o < n_perms; ++o)
    if (!perms[o] || !valid_perm(perms[o], p)) return IBMI_ERR_INVALID_ARG;
  if (!is_device_ptr(A)) return IBMI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // candidate partitions: K in {2, 3, 4, 6, 8} with cores of at least 64
  // rows, overlap 2h of 10, 20 and 30% of the core
  struct Part {
    int32_t K;
    int64_t h;
  };
  std::vector<Part> parts;
  for (int32_t K : {2, 3, 4, 6, 8}) {
    const int64_t core = p / K;
    if (core < 64) continue;
    for (double f : {0.1, 0.2, 0.3}) {
      const int64_t h = std::max<int64_t>(1, (int64_t)llround(0.5 * f * (double)core));
      bool dup = false;
      for (const Part& q : parts) dup |= (q.K == K && q.h == h);
      if (!dup) parts.push_back({K, h});
    }
  }
  if (parts.empty()) return IBMI_ERR_INVALID_ARG;
  double* Ap = nullptr;
  double* H = nullptr;
  int64_t* dq = nullptr;
  struct FreeAll {
    double** a; double** h; int64_t** q;
    ~FreeAll() { cudaFree(*a); cudaFree(*h); cudaFree(*q); }
  } keep{&Ap, &H, &dq};
  IBMI_CUDA_TRY(cudaMalloc(&Ap, sizeof(double) * p * p));
  IBMI_CUDA_TRY(cudaMalloc(&H, sizeof(double) * p * p));
  IBMI_CUDA_TRY(cudaMalloc(&dq, sizeof(int64_t) * p));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  IBMI_CUDA_TRY(cudaEventCreate(&e0));
  IBMI_CUDA_TRY(cudaEventCreate(&e1));
  struct FreeEv {
    cudaEvent_t a, b;
    ~FreeEv() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } keep_ev{e0, e1};
  int32_t count = 0;
  bool have = false;
  memset(best, 0, sizeof(*best));
  best->status = IBMI_NOT_CONVERGED;
  best->seconds = INFINITY;
  for (int32_t o = -1; o < n_perms; ++o) {
    const double* M = A;
    int64_t ldm = lda;
    if (o >= 0) {   // the permuted matrix P A P^T
      IBMI_CUDA_TRY(cudaMemcpyAsync(dq, perms[o], sizeof(int64_t) * p, cudaMemcpyHostToDevice, st));
      IBMI_TRY(gather(A, lda, p, dq, Ap, p, st));
      M = Ap;
      ldm = p;
    }
    for (const Part& q : parts) {
      ibmi_plan_desc d = *base;
      d.p = p;
      d.K = q.K;
      d.h = q.h;
      d.lo = d.hi = nullptr;
      if (d.init == IBMI_INIT_USER) d.init = IBMI_INIT_IDENTITY;
      ibmi_plan_t plan = nullptr;
      ibmi_tune_candidate c{};
      c.order = o;
      c.K = q.K;
      c.h = q.h;
      c.seconds = INFINITY;
      c.resid_f = NAN;
      ibmi_status s = ibmi_plan(&d, &plan);
      if (s == IBMI_OK) {
        ibmi_result r;
        cudaEventRecord(e0, st);
        s = ibmi_invert(plan, M, ldm, H, p, st, &r);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c.sweeps = r.sweeps;
        c.ns_steps = r.ns_steps;
        c.resid_f = r.resid_f;
        c.seconds = (double)ms / 1000.0;
        ibmi_plan_destroy(plan);
      }
      c.status = s;
      if (s == IBMI_ERR_CUDA || s == IBMI_ERR_TIMEOUT) return s;
      if (count < max_all) all[count] = c;
      ++count;
      if (s == IBMI_OK && c.seconds < best->seconds) {
        *best = c;
        have = true;
      }
    }
  }
  if (n_all) *n_all = count;
  return have ? IBMI_OK : IBMI_NOT_CONVERGED;
}
