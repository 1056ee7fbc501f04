// Batched inversion on the device: a group of matrices of one size bucket and
// partition runs the mixed-precision pipeline (Algorithm 1 with BF16x3 sweep
// products, BF16x3 stop tests and the Newton-Schulz tail with FP64-accurate
// digit-sliced residuals) in lockstep.  Every launch covers one step of every
// matrix of the group that takes that step: the tcgen05 kernels walk the
// output tiles of all of them through 3-D tensor maps whose third coordinate
// is the matrix, the elementwise kernels take the matrix from blockIdx.z.
// Each matrix keeps its own decisions (its sweep count, slice level, hand-over,
// digit groups of each tail residual, a residual after an exact one taken as
// its correction Q - (X - Xprev) A), so its arithmetic is exactly what it
// would be in a group of one; matrices that take different decisions are
// covered by different launches of the same round.  The host synchronises
// once per round of the group (one sweep and its stop test for the sweeping
// matrices, one tail step for the others), not once per matrix and test.
//
// Layout (per group of n matrices of padded order pb, ldp = pb rounded up to
// 64): every per-matrix plane is stacked, matrix b at offset b * rows * ld of
// its plane, planes of one kind one after another.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "batch_dev.cuh"
#include "oz_pairs.cuh"
#include "oz_rows.cuh"
#include "tail_plan.h"

namespace ibmi {

namespace {

constexpr int kBN = 128;              // N tile of the sweep products and the BF16x3 stop test
constexpr int kFirstGroups = 7;       // digit groups of the first tail residual (orders below 2048)
constexpr int kNextGroups = 8;        // ... and of the next ones while rho^2 > 1e3 tol
constexpr int kWDigitsA = 5, kWDigitsB = 4, kWGroups = 4;   // W = A_I^{-1} A_{I,:}: 34-bit x 27-bit digits

__device__ __forceinline__ int pick(const int* sel, int i) { return sel ? sel[i] : i; }

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// A64[b] = [[S_b, 0], [0, I]], S_b symmetric from the lower triangle of A_b.
__global__ void k_b_embed(const BatchMat* in, int64_t pb, double* A64) {
  const int b = blockIdx.z;
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= pb) return;
  const BatchMat q = in[b];
  double v;
  if (i < q.p && j < q.p) v = i >= j ? q.A[i * q.lda + j] : q.A[j * q.lda + i];
  else v = i == j ? 1.0 : 0.0;
  A64[(b * pb + i) * pb + j] = v;
}

// H_b = leading p_b x p_b block of X64[b].
__global__ void k_b_unpad(const BatchMat* in, const int* sel, int64_t pb, const double* X64) {
  const int b = pick(sel, blockIdx.z);
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const BatchMat q = in[b];
  if (i >= q.p || j >= q.p) return;
  q.H[i * q.ldh + j] = X64[(b * pb + i) * pb + j];
}

// Hf[b] = I and its three BF16 slices.
__global__ void k_b_init_h(int64_t pb, int64_t ldp, float* Hf, __nv_bfloat16* s0, __nv_bfloat16* s1,
                           __nv_bfloat16* s2) {
  const int64_t b = blockIdx.z, i = blockIdx.y, c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ldp) return;
  const int64_t idx = (b * pb + i) * ldp + c;
  const float x = (c == i) ? 1.f : 0.f;
  Hf[idx] = x;
  s0[idx] = __float2bfloat16_rn(x);
  s1[idx] = __float2bfloat16_rn(0.f);
  s2[idx] = __float2bfloat16_rn(0.f);
}

// All three slices of H from the FP32 master (a matrix entering three slices).
__global__ void k_b_reslice(const int* sel, int64_t pb, int64_t ldp, const float* Hf, __nv_bfloat16* s0,
                            __nv_bfloat16* s1, __nv_bfloat16* s2) {
  const int64_t b = pick(sel, blockIdx.z), i = blockIdx.y, c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ldp) return;
  const int64_t idx = (b * pb + i) * ldp + c;
  split3(Hf[idx], s0[idx], s1[idx], s2[idx]);
}

// Digit slices of selected rows: row r of the launch is row (r % rows) of
// matrix sel[r / rows]; its input at src + (b * rows + i) * lds + (b * sstride),
// placed at columns [c0, c0 + ncols) of output row b * orows + orow0 + i.
struct SliceRows {
  const double* src; int64_t lds, sstride;
  int64_t rows, ncols, c0, orows, orow0, ldp;
  int nslices;
  int* expo;
};
__global__ void k_b_slices(const int* sel, SliceRows a, SlicePtrs out) {
  const int64_t b = pick(sel, (int)(blockIdx.x / a.rows)), i = blockIdx.x % a.rows;
  oz_slice_row(a.src + b * a.sstride + i * a.lds, b * a.orows + a.orow0 + i, a.ncols, a.c0, a.ldp, out, a.nslices,
               a.expo, nullptr);
}

// BF16 hi/lo of the stacked FP64 rows (the stop test's A operand): row i of
// the launch is row i of the stack (row pitch ldx), ncols values, zero beyond.
__global__ void k_b_split2(const double* X, int64_t ldx, int64_t ncols, int64_t ldp, __nv_bfloat16* s0,
                           __nv_bfloat16* s1) {
  const int64_t i = blockIdx.y, c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ldp) return;
  const float x = c < ncols ? (float)X[i * ldx + c] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  s0[i * ldp + c] = h;
  s1[i * ldp + c] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// W slices of set k: W = 2^{e_i + f_j - 12} sum_{q <= 4} T_q 2^{-7q} on the
// columns of I^c, zero on I and on the padding.
__global__ void k_b_wcombine(const int* TW, int64_t plane, int64_t rows_w, int64_t woff, int64_t m, int64_t pb,
                             int64_t ldp, const int* expW, const int* expA, int64_t lo, int64_t hi,
                             __nv_bfloat16* W0, __nv_bfloat16* W1, __nv_bfloat16* W2) {
  const int64_t b = blockIdx.z, i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ldp) return;
  float w = 0.f;
  if (j < pb && (j < lo || j >= hi)) {
    const int64_t r = b * rows_w + woff + i;
    w = ozr_to_float(oz_value(TW, plane, r * ldp + j, kWGroups, expW[r] + expA[b * pb + j] - 12));
  }
  const int64_t o = (b * m + i) * ldp + j;
  __nv_bfloat16 x0, x1, x2;
  split3(w, x0, x1, x2);
  W0[o] = x0;
  W1[o] = x1;
  W2[o] = x2;
}

// a3 epilogue of matrix bat: X = -acc written to H[lo + i, j] and H[j, lo + i]
// (FP32 master and slices), j in I^c.
struct EpiBSweepX : tc::EpiBase {
  float* Hf; __nv_bfloat16* H0; __nv_bfloat16* H1; __nv_bfloat16* H2;
  int64_t ldp, lo, hi, p, m, bstride;
  __device__ __forceinline__ void put(int64_t idx, float x) const {
    __nv_bfloat16 a, b, d;
    split3(x, a, b, d);
    Hf[idx] = x;
    H0[idx] = a;
    H1[idx] = b;
    if (H2) H2[idx] = d;
  }
  __device__ __forceinline__ void warp_tile(int64_t row0, int64_t j0, int, const float* __restrict__ stage,
                                            int lane) const {
    const int64_t off = (int64_t)bat * bstride;
    {
      const int64_t i = row0 + lane;
      if (i < m) {
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
          const int64_t j = j0 + c;
          if (j < p && (j < lo || j >= hi)) put(off + j * ldp + lo + i, -stage[lane * 17 + c]);
        }
      }
    }
    const int c = lane & 15;
    const int64_t j = j0 + c;
    if (j >= p || (j >= lo && j < hi)) return;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
      const int r = 2 * k + (lane >> 4);
      const int64_t i = row0 + r;
      if (i < m) put(off + (lo + i) * ldp + j, -stage[r * 17 + c]);
    }
  }
};

// a4 of matrix bat (one K split): the finish in the epilogue.  P = X W^T on
// the tiles on and below the diagonal; each element (i, j), j <= i, gives
// x = A_I^{-1}[i, j] - P[i, j] (FP32), written to H[I, I] at (i, j) and, from
// the same x, at (j, i), so the block is exactly symmetric: the first pass
// writes (i, j) along rows and keeps x in the warp's stage, the second writes
// (j, i) with one lane per row i.
struct EpiBSymFinish : tc::EpiBase {
  const double* Ainv; int64_t abstride, m, lo, pb, ldp;
  float* Hf; __nv_bfloat16* s0; __nv_bfloat16* s1; __nv_bfloat16* s2;
  __device__ __forceinline__ void put(int64_t o, float x) const {
    Hf[o] = x;
    __nv_bfloat16 t0, t1, t2;
    split3(x, t0, t1, t2);
    s0[o] = t0;
    s1[o] = t1;
    if (s2) s2[o] = t2;
  }
  __device__ __forceinline__ void warp_tile(int64_t row0, int64_t j0, int, const float* __restrict__ stage_in,
                                            int lane) const {
    float* stage = const_cast<float*>(stage_in);   // this warp's own stage: x goes back in place
    const double* Ab = Ainv + (int64_t)bat * abstride;
    const int64_t o0 = ((int64_t)bat * pb + lo) * ldp + lo;
    const int c = lane & 15;
    const int64_t j = j0 + c;
    double a[16];   // all loads of A_I^{-1} in flight before the first store
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int64_t i = row0 + 2 * k + (lane >> 4);
      a[k] = i < m && j <= i ? Ab[i * m + j] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = 2 * k + (lane >> 4);
      const int64_t i = row0 + r;
      if (i < m && j <= i) {
        const float x = (float)(a[k] - (double)stage[r * 17 + c]);
        stage[r * 17 + c] = x;
        put(o0 + i * ldp + j, x);
      }
    }
    __syncwarp();
    const int64_t i = row0 + lane;
#pragma unroll 4
    for (int cc = 0; cc < 16; ++cc) {
      const int64_t jj = j0 + cc;
      if (i < m && jj < i) put(o0 + jj * ldp + i, stage[lane * 17 + cc]);
    }
  }
};

// BF16x3 stop test of matrix bat: per unit and epilogue warp, the sum of
// (delta_ij - acc)^2 over the tile's entries inside the matrix.
struct EpiBResidSq : tc::EpiBase {
  double* partials; int64_t nparts, p;
  double s = 0.0;
  __device__ __forceinline__ void operator()(int64_t i, int64_t j0, int, const float (&v)[16]) {
    if (i >= p) return;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (j0 + c < p) {
        const double r = (i == j0 + c ? 1.0 : 0.0) - (double)v[c];
        s += r * r;
      }
    }
  }
  __device__ __forceinline__ void unit_end(int q, int tile) {
    double x = s;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) partials[(int64_t)bat * nparts + (int64_t)tile * 4 + q] = x;
    s = 0.0;
  }
};

// out[b * 4] = sqrt(sum of matrix b's partials) / sqrt(p_b): one CTA per selected matrix.
__global__ void k_b_sum(const int* sel, const double* partials, int64_t nparts, const BatchMat* in, double* out) {
  const int b = pick(sel, blockIdx.x);
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nparts; i += blockDim.x) s += partials[(int64_t)b * nparts + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    out[(int64_t)b * 4] = sqrt(t) / sqrt((double)in[b].p);
  }
}

// X64[b] = (double) Hf[b] on the pb x pb block.
__global__ void k_b_export(const int* sel, int64_t pb, int64_t ldp, const float* Hf, double* X64) {
  const int64_t b = pick(sel, blockIdx.z), i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= pb) return;
  X64[(b * pb + i) * pb + j] = (double)Hf[(b * pb + i) * ldp + j];
}

// Q = I - C with C = 2^{e_i + f_j - 12} sum_{q <= qm[z]} T_q 2^{-7q} of
// matrix sel[z] (FP64, pb x pb), or with sub[z] (a correction) Q = Q - C in
// place; and per-CTA sums of Q^2.
__global__ void k_b_combine(const int* sel, const int* T, int64_t plane, int64_t pb, int64_t ldp, const int* ex,
                            const int* ea, const int* qm, const int* sub, double* Q, double* partials,
                            int64_t nparts) {
  // four consecutive columns per thread, one int4 load per group plane (row
  // pitch ldp, a multiple of 64)
  const int64_t b = pick(sel, blockIdx.z), i = blockIdx.y, j0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  const int qmax = qm[blockIdx.z];   // highest digit group of this matrix's residual
  const bool corr = sub[blockIdx.z] != 0;
  float sq = 0.f;
  if (j0 < pb) {
    const int* Tb = T + b * pb * ldp + i * ldp + j0;
    int4 t4[10];
#pragma unroll
    for (int q = 0; q < 10; ++q)
      t4[q] = q <= qmax ? *reinterpret_cast<const int4*>(Tb + q * plane) : make_int4(0, 0, 0, 0);
    const int exi = ex[b * pb + i] - 12;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      const int64_t j = j0 + c4;
      if (j >= pb) break;
      int t[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) t[q] = c4 == 0 ? t4[q].x : (c4 == 1 ? t4[q].y : (c4 == 2 ? t4[q].z : t4[q].w));
      const int64_t o = (b * pb + i) * pb + j;
      const double c = oz_groups_value(t, exi + ea[b * pb + j]);
      const double q = corr ? Q[o] - c
                            : (i == j ? 1.0 - c : ozr_bits_to_double(ozr_double_to_bits(c) ^ 0x8000000000000000ull));
      const float qf = ozr_to_float(q);
      sq += qf * qf;
      Q[o] = q;
    }
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    partials[b * nparts + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// Newton-Schulz update of the symmetric X of matrix sel[z] from the lower
// tiles of X Q^T (symmetric: X - X A X), in place: for j <= i,
// X[i][j] + 2^{e_i + g_j - 12} sum T_q 2^{-7q} goes to (i, j) and (j, i), and
// D <- the step's difference at both (the correction of the next residual
// slices it).  One block per tile on or below the diagonal; it reads its
// elements before writing the mirror tile, which no block reads.
__global__ void k_b_update_lower(const int* sel, const int* T, int64_t plane, int64_t pb, int64_t ldp, const int* ex,
                                 const int* eq, int qmax, double* X64, double* D) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double tv[32][33], td[32][33];
  const int64_t b = pick(sel, blockIdx.z);
  double* X = X64 + b * pb * pb;
  double* Dm = D + b * pb * pb;
  const int* Tb = T + b * pb * ldp;
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = I0 + r, j = J0 + tx;
    if (i < pb && j <= i) {
      const double xo = X[i * pb + j];
      const double v = xo + oz_value(Tb, plane, i * ldp + j, qmax, ex[b * pb + i] + eq[b * pb + j] - 12);
      const double d = v - xo;
      tv[r][tx] = v;
      td[r][tx] = d;
      X[i * pb + j] = v;
      Dm[i * pb + j] = d;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = J0 + r, i = I0 + tx;   // (j, i), the mirror of (i, j) with j < i
    if (i < pb && j < i) {
      X[j * pb + i] = tv[tx][r];
      Dm[j * pb + i] = td[tx][r];
    }
  }
}

// N tile of the digit-pair launches, as in the single-matrix path (64-wide
// tiles for orders 512..1024, which halve a tile's serial chain of pairs,
// measured slower: they double the operand bytes per MMA).
int oz_bn(int64_t p) { return p > 1536 ? 224 : (p > 384 ? 128 : 64); }

template <class F>
ibmi_status with_bn(int bn, F&& f) {
  switch (bn) {
    case 224: return f(std::integral_constant<int, 224>{});
    case 128: return f(std::integral_constant<int, 128>{});
    default: return f(std::integral_constant<int, 64>{});
  }
}

int count_pairs(int na, int nb, int qlo, int qhi) {
  int c = 0;
  for (int q = qlo; q <= qhi; ++q)
    for (int a = 0; a <= q; ++a) c += (a < na && q - a < nb) ? 1 : 0;
  return c;
}

}  // namespace

// ----------------------------------------------------------------- group --

struct DevGroup::Impl {
  int64_t pb = 0, ldp = 0, mmax = 0;
  int K = 0, n = 0, bn = 64;
  std::vector<int64_t> lo, hi, m;
  int64_t rows_w = 0, ainv_total = 0, nparts_c = 0, nparts_r = 0;
  std::vector<int64_t> woff, aoff;
  ibmi_plan_s F;                         // FP64 factorisation of all n K blocks
  void* pool = nullptr;
  size_t pool_bytes = 0;
  // device buffers
  BatchMat* din = nullptr;
  double* A64 = nullptr;
  double* X64 = nullptr;
  double* Q = nullptr;
  double* Xprev = nullptr;
  float* Hf = nullptr;
  __nv_bfloat16* Hs[3] = {};
  std::vector<__nv_bfloat16*> Ws[3];
  __nv_bfloat16* Ao[OZ_SA] = {};
  __nv_bfloat16* Xo[OZ_SX] = {};
  __nv_bfloat16* Qo[NS_S] = {};
  __nv_bfloat16* Af[2] = {};
  __nv_bfloat16* XW[kWDigitsA] = {};
  int* T = nullptr;
  int* TW = nullptr;
  int *expA = nullptr, *expX = nullptr, *expQ = nullptr, *expW = nullptr;
  int2* w_kr = nullptr;
  double* partials = nullptr;
  double* dout = nullptr;
  int* dsel = nullptr;                   // selection lists of one round
  int* err = nullptr;
  // tensor maps (3-D: the matrix is the third coordinate)
  CUtensorMap mapH[3];
  std::vector<CUtensorMap> mapW[3];
  CUtensorMap mAo[OZ_SA], mXo[OZ_SX], mQo[NS_S], mAf[2], mXW[kWDigitsA];
  int rounds = 0;

  ~Impl() {
    cudaFree(pool);
    cudaFree(F.bat_pool);
    cudaFree(F.pool);
    cudaFree(F.dstatus);
  }
};

namespace {

struct Alloc {
  uint8_t* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* r = (T*)(base + off);
    off += (count * sizeof(T) + 255) / 256 * 256;
    return r;
  }
};

}  // namespace

DevGroup::DevGroup() : d(new Impl()) {}
DevGroup::~DevGroup() { delete d; }
int DevGroup::rounds() const { return d->rounds; }
int DevGroup::capacity() const { return d->n; }
size_t DevGroup::bytes() const {
  const Impl& g = *d;
  const size_t Z = (size_t)g.n * g.K;
  return g.pool_bytes + sizeof(double) * (Z * (2 * g.mmax * g.mmax + g.mmax * CHOL_NB) + (size_t)g.n * g.ainv_total);
}

size_t DevGroup::bytes_per_matrix(int64_t pb, int K, int64_t h) {
  const int64_t ldp = (pb + 63) / 64 * 64;
  const double p = (double)pb, l = (double)ldp;
  const double m = std::min(p, p / K + 2.0 * (double)h), rows_w = K * (ceil(m / 128.0) * 128.0);
  double b = 8.0 * (4.0 * p * p);                           // A64, X64, Q, Xprev
  b += 4.0 * p * l + 2.0 * 3.0 * p * l;                     // Hf, Hs
  b += 2.0 * 3.0 * K * m * l + 4.0 * 8.0 * m * m;           // W slices, split-K partials
  b += 2.0 * (OZ_SA + OZ_SX + NS_S + 2) * p * l;           // digit planes
  b += 4.0 * (OZ_QMAX + 1) * p * l;                         // group planes
  b += 2.0 * kWDigitsA * rows_w * l + 4.0 * (kWGroups + 1) * rows_w * l;   // W formation
  b += 8.0 * K * (2.0 * m * m + 32.0 * m);                  // FP64 factorisation
  return (size_t)b + (1 << 16);
}

ibmi_status DevGroup::create(int64_t pb, int K, int64_t h, int n) {
  Impl& g = *d;
  g.pb = pb;
  g.ldp = (pb + 63) / 64 * 64;
  g.K = K;
  g.n = n;
  g.bn = oz_bn(pb);
  g.lo.resize(K);
  g.hi.resize(K);
  g.m.resize(K);
  g.woff.resize(K);
  g.aoff.resize(K);
  for (int k = 0; k < K; ++k) {
    const int64_t b0 = (int64_t)k * pb / K, b1 = (int64_t)(k + 1) * pb / K;
    g.lo[k] = std::max<int64_t>(0, b0 - h);
    g.hi[k] = std::min<int64_t>(pb, b1 + h);
    g.m[k] = g.hi[k] - g.lo[k];
    g.mmax = std::max(g.mmax, g.m[k]);
    g.woff[k] = g.rows_w;
    g.rows_w += (g.m[k] + 127) / 128 * 128;
    g.aoff[k] = g.ainv_total;
    g.ainv_total += g.m[k] * g.m[k];
    if (g.m[k] >= pb) return IBMI_ERR_INVALID_ARG;
  }
  g.nparts_c = pb * nblk((pb + 3) / 4);   // k_b_combine: one partial per CTA of four-column threads
  g.nparts_r = ((pb + 127) / 128) * ((pb + kBN - 1) / kBN) * 4;
  const int64_t nparts = std::max(g.nparts_c, g.nparts_r);
  // FP64 factorisation plan over the n K blocks
  ibmi_plan_s& F = g.F;
  F.d.p = pb;
  F.mmax = g.mmax;
  F.tile_batch = K;   // tiles as for one matrix, whatever the group size
  const int Z = n * K;
  std::vector<int64_t> zlo(Z), zm(Z), zoff(Z), zoffA(Z), zero(Z, 0);
  for (int b = 0; b < n; ++b)
    for (int k = 0; k < K; ++k) {
      const int z = b * K + k;
      zlo[z] = g.lo[k];
      zm[z] = g.m[k];
      zoff[z] = (int64_t)b * g.ainv_total + g.aoff[k];
      zoffA[z] = (int64_t)b * pb * pb;
    }
  F.lo.assign(zlo.begin(), zlo.end());
  F.hi.resize(Z);
  for (int z = 0; z < Z; ++z) F.hi[z] = zlo[z] + zm[z];
  const size_t bat = (size_t)Z * (g.mmax * g.mmax + g.mmax * g.mmax + g.mmax * CHOL_NB);
  IBMI_CUDA_TRY(cudaMalloc(&F.bat_pool, sizeof(double) * bat + sizeof(int64_t) * 5 * Z));
  IBMI_CUDA_TRY(cudaMalloc(&F.pool, sizeof(double) * (size_t)n * g.ainv_total));
  IBMI_CUDA_TRY(cudaMalloc(&F.dstatus, sizeof(DevStatus) * Z));
  double* fb = (double*)F.bat_pool;
  F.bat_L = fb; fb += (size_t)Z * g.mmax * g.mmax;
  F.bat_R = fb; fb += (size_t)Z * g.mmax * g.mmax;
  F.bat_linv = fb; fb += (size_t)Z * g.mmax * CHOL_NB;
  int64_t* ib = (int64_t*)fb;
  F.dlo = ib; F.dm = ib + Z; F.doff_ainv = ib + 2 * Z; F.doff_w = ib + 3 * Z; F.doffA = ib + 4 * Z;
  std::vector<int64_t> packed;
  for (auto* v : {&zlo, &zm, &zoff, &zero, &zoffA}) packed.insert(packed.end(), v->begin(), v->end());
  IBMI_CUDA_TRY(cudaMemcpy(ib, packed.data(), sizeof(int64_t) * packed.size(), cudaMemcpyHostToDevice));
  for (int k = 0; k < K; ++k) F.ainv.push_back(nullptr);
  // the group's pool
  const int64_t pl = pb * g.ldp;   // one plane of one matrix
  size_t bytes = 0;
  {
    const size_t per = (size_t)n;
    auto add = [&](size_t b) { bytes += (b + 255) / 256 * 256; };
    add(sizeof(BatchMat) * per);
    for (int i = 0; i < 4; ++i) add(sizeof(double) * per * pb * pb);
    add(sizeof(float) * per * pl);
    for (int s = 0; s < 3; ++s) add(2 * per * pl);
    for (int s = 0; s < 3; ++s)
      for (int k = 0; k < K; ++k) add(2 * per * g.m[k] * g.ldp);
    for (int s = 0; s < OZ_SA + OZ_SX + NS_S + 2; ++s) add(2 * per * pl);
    for (int s = 0; s < kWDigitsA; ++s) add(2 * per * g.rows_w * g.ldp);
    add(sizeof(int) * (size_t)(OZ_QMAX + 1) * per * pl);
    add(sizeof(int) * (size_t)(kWGroups + 1) * per * g.rows_w * g.ldp);
    add(sizeof(int) * 3 * per * pb);
    add(sizeof(int) * per * g.rows_w);
    add(sizeof(int2) * (g.rows_w / 128));
    add(sizeof(double) * per * nparts);
    add(sizeof(double) * per * 4);
    add(sizeof(int) * 16 * per);
    add(256);
  }
  if (cudaMalloc(&g.pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IBMI_ERR_OOM;
  }
  g.pool_bytes = bytes;
  Alloc a{(uint8_t*)g.pool};
  const size_t nn = (size_t)n;
  g.din = a.take<BatchMat>(nn);
  g.A64 = a.take<double>(nn * pb * pb);
  g.X64 = a.take<double>(nn * pb * pb);
  g.Q = a.take<double>(nn * pb * pb);
  g.Xprev = a.take<double>(nn * pb * pb);
  g.Hf = a.take<float>(nn * pl);
  for (int s = 0; s < 3; ++s) g.Hs[s] = a.take<__nv_bfloat16>(nn * pl);
  for (int s = 0; s < 3; ++s)
    for (int k = 0; k < K; ++k) g.Ws[s].push_back(a.take<__nv_bfloat16>(nn * g.m[k] * g.ldp));
  for (int s = 0; s < OZ_SA; ++s) g.Ao[s] = a.take<__nv_bfloat16>(nn * pl);
  for (int s = 0; s < OZ_SX; ++s) g.Xo[s] = a.take<__nv_bfloat16>(nn * pl);
  for (int s = 0; s < NS_S; ++s) g.Qo[s] = a.take<__nv_bfloat16>(nn * pl);
  for (int s = 0; s < 2; ++s) g.Af[s] = a.take<__nv_bfloat16>(nn * pl);
  for (int s = 0; s < kWDigitsA; ++s) g.XW[s] = a.take<__nv_bfloat16>(nn * g.rows_w * g.ldp);
  g.T = a.take<int>((size_t)(OZ_QMAX + 1) * nn * pl);
  g.TW = a.take<int>((size_t)(kWGroups + 1) * nn * g.rows_w * g.ldp);
  g.expA = a.take<int>(nn * pb);
  g.expX = a.take<int>(nn * pb);
  g.expQ = a.take<int>(nn * pb);
  g.expW = a.take<int>(nn * g.rows_w);
  g.w_kr = a.take<int2>(g.rows_w / 128);
  g.partials = a.take<double>(nn * nparts);
  g.dout = a.take<double>(nn * 4);
  g.dsel = a.take<int>(16 * nn);
  g.err = a.take<int>(64);
  // digit rows of the W slots beyond each set's rows stay zero
  for (int s = 0; s < kWDigitsA; ++s) IBMI_CUDA_TRY(cudaMemset(g.XW[s], 0, 2 * nn * g.rows_w * g.ldp));
  {  // K-tile range of every 128-row tile of the W slots: the columns of its set
    std::vector<int2> kr(g.rows_w / 128);
    for (int k = 0; k < K; ++k)
      for (int64_t t = g.woff[k] / 128; t < (g.woff[k] + g.m[k] + 127) / 128; ++t)
        kr[t] = make_int2((int)(g.lo[k] / tc::BK), (int)((g.hi[k] + tc::BK - 1) / tc::BK));
    IBMI_CUDA_TRY(cudaMemcpy(g.w_kr, kr.data(), sizeof(int2) * kr.size(), cudaMemcpyHostToDevice));
  }
  bool ok = true;
  for (int s = 0; s < 3; ++s) {
    ok &= tc::make_map_bf16_3d(&g.mapH[s], g.Hs[s], n, pb, pb, g.ldp, 128);
    g.mapW[s].resize(K);
    for (int k = 0; k < K; ++k) ok &= tc::make_map_bf16_3d(&g.mapW[s][k], g.Ws[s][k], n, g.m[k], pb, g.ldp, 128);
  }
  for (int s = 0; s < OZ_SA; ++s) ok &= tc::make_map_bf16_3d(&g.mAo[s], g.Ao[s], n, pb, pb, g.ldp, g.bn);
  for (int s = 0; s < OZ_SX; ++s) ok &= tc::make_map_bf16_3d(&g.mXo[s], g.Xo[s], n, pb, pb, g.ldp, 128);
  for (int s = 0; s < NS_S; ++s) ok &= tc::make_map_bf16_3d(&g.mQo[s], g.Qo[s], n, pb, pb, g.ldp, g.bn);
  for (int s = 0; s < 2; ++s) ok &= tc::make_map_bf16_3d(&g.mAf[s], g.Af[s], n, pb, pb, g.ldp, kBN);
  for (int s = 0; s < kWDigitsA; ++s) ok &= tc::make_map_bf16_3d(&g.mXW[s], g.XW[s], n, g.rows_w, pb, g.ldp, 128);
  return ok ? IBMI_OK : IBMI_ERR_CUDA;
}

// ------------------------------------------------------------------ run ----

namespace {

enum Phase { SWEEP = 0, TAIL = 1, DONE = 2, FALLBACK = 3, FAILED = 4 };
enum TailAct { T_NONE = 0, T_ENTER, T_CERTIFY, T_STEP, T_EXTEND };

struct MState {
  Phase phase = SWEEP;
  int level = 0, r = 0, stalled = 0, s = 0, qc = 0;
  double best = INFINITY, last_cheap = INFINITY, handover_below = INFINITY, handover_rho = 0.0, prev = INFINITY;
  bool early = false, reslice = false, restore = false;
  bool exact = false;     // the last residual is exact (all groups, or a correction of an exact one)
  bool corr = false;      // this round's residual is a correction of the last one
  bool xo_delta = false;  // the X digit planes hold the last correction's difference, not X
  bool waiting = false;   // ready for a tail action, held back to share its launches
  TailAct act = T_NONE;
  int next_q = 0;   // groups of the residual this round's tail action computes
};

}  // namespace

ibmi_status DevGroup::run(const BatchMat* mats, int nrun, const ibmi_batch_opts& o, double theta, cudaStream_t st,
                          ibmi_result* res, int* fallback) {
  Impl& g = *d;
  if (nrun < 1 || nrun > g.n) return IBMI_ERR_INVALID_ARG;
  const int n = nrun, cap = g.n, K = g.K;   // matrices of this run, of the group's buffers
  const int64_t pb = g.pb, ldp = g.ldp, pl = pb * g.ldp;
  IBMI_CUDA_TRY(cudaMemcpyAsync(g.din, mats, sizeof(BatchMat) * n, cudaMemcpyHostToDevice, st));
  IBMI_CUDA_TRY(cudaMemsetAsync(g.err, 0, sizeof(int), st));
  IBMI_CUDA_TRY(cudaMemsetAsync(g.F.dstatus, 0, sizeof(DevStatus) * n * K, st));
  std::vector<MState> ms(n);
  std::vector<double> flops(n, 0.0);
  for (int b = 0; b < n; ++b) {
    memset(&res[b], 0, sizeof(ibmi_result));
    res[b].bad_block = -1;
    res[b].bad_pivot = -1;
    res[b].resid_f = NAN;
    res[b].paper_est = NAN;
    fallback[b] = 0;
  }
  double fs = 0.0, fplan = 0.0;
  for (int k = 0; k < K; ++k) {
    const double m = (double)g.m[k], nn = (double)pb - m;
    fs += 2.0 * m * nn * nn + 2.0 * m * m * nn;
    fplan += m * m * m / 3.0 + 2.0 * m * m * m + 2.0 * m * m * nn;
  }
  const double fr = 2.0 * (double)pb * pb * pb;
  const int full_pairs = count_pairs(OZ_SX, OZ_SA, 0, OZ_QMAX);
  const dim3 g2(nblk(pb), (unsigned)pb, (unsigned)n);
  // --- setup: padded inputs, FP64 factorisations, A's digits, W, H = I
  note_launch();
  k_b_embed<<<g2, 256, 0, st>>>(g.din, pb, g.A64);
  IBMI_CUDA_TRY(cudaGetLastError());
  {  // the FP64 factorisations of this run's n K blocks
    const size_t zall = g.F.lo.size();
    g.F.lo.resize((size_t)n * K);
    g.F.hi.resize((size_t)n * K);
    const ibmi_status fs_ = invariants_all(&g.F, g.A64, pb, false, st);
    g.F.lo.resize(zall);
    g.F.hi.resize(zall);
    for (size_t z = 0; z < zall; ++z) {
      g.F.lo[z] = g.lo[z % K];
      g.F.hi[z] = g.hi[z % K];
    }
    IBMI_TRY(fs_);
  }
  {
    SlicePtrs sp{};
    for (int s = 0; s < OZ_SA; ++s) sp.s[s] = g.Ao[s];
    SliceRows a{g.A64, pb, pb * pb, pb, pb, 0, pb, 0, ldp, OZ_SA, g.expA};
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch(2);
    k_b_slices<<<(unsigned)(n * pb), 256, 0, st>>>(nullptr, a, sp);
    k_b_split2<<<dim3(nblk(ldp), (unsigned)(n * pb)), 256, 0, st>>>(g.A64, pb, pb, ldp, g.Af[0], g.Af[1]);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  {  // W = A_I^{-1} A_{I,:} for all sets and matrices: 5 digits of A_I^{-1} x 4 of A, groups <= 4
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    SlicePtrs sp{};
    for (int s = 0; s < kWDigitsA; ++s) sp.s[s] = g.XW[s];
    for (int k = 0; k < K; ++k) {
      SliceRows a{g.F.pool + g.aoff[k], g.m[k], g.ainv_total, g.m[k], g.m[k], g.lo[k], g.rows_w, g.woff[k], ldp,
                  kWDigitsA, g.expW};
      note_launch();
      k_b_slices<<<(unsigned)(n * g.m[k]), 256, 0, st>>>(nullptr, a, sp);
    }
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  {
    double alg = 0.0;
    for (int k = 0; k < K; ++k) alg += 2.0 * (double)g.m[k] * g.m[k] * (double)(pb - g.m[k]);
    alg *= n;
    const int grid_n = (int)((pb + g.bn - 1) / g.bn), grid_m = (int)(g.rows_w / 128);
    // all pair products of all matrices in one persistent launch, each row
    // tile over its set's K range
    tc::OzPairMaps maps;
    for (int s = 0; s < kWDigitsA; ++s) maps.a[s] = g.mXW[s];
    for (int u = 0; u < kWDigitsB; ++u) maps.b[u] = g.mAo[u];
    tc::OzPairArgs w{};
    int np = 0;
    for (int q = 0; q <= kWGroups; ++q) {
      bool first = true;
      for (int s = 0; s <= q; ++s) {
        const int u = q - s;
        if (s >= kWDigitsA || u >= kWDigitsB) continue;
        w.s[np] = (int8_t)s;
        w.u[np] = (int8_t)u;
        w.q[np] = (int8_t)q;
        w.first[np] = first ? 1 : 0;
        first = false;
        ++np;
      }
    }
    int kt_max = 1;
    for (int k = 0; k < K; ++k)
      kt_max = std::max<int>(kt_max, (int)((g.hi[k] + tc::BK - 1) / tc::BK - g.lo[k] / tc::BK));
    w.n = np;
    w.grid_n = grid_n;
    w.tiles = grid_n * grid_m;
    w.kt_total = kt_max;
    w.chunk = OZ_KCHUNK / tc::BK;
    w.T = g.TW;
    w.plane = (int64_t)cap * g.rows_w * ldp;
    w.ldt = ldp;
    w.M = g.rows_w;
    w.N = pb;
    w.err = g.err;
    w.nb = n;
    w.bsel = nullptr;
    w.tstride = g.rows_w * ldp;
    w.mkr = g.w_kr;
    tc::oz_make_segments(w);
    {
      ProfScope ps(IBMI_K_INVARIANTS_TC, st, 2.0 * np * n * (double)g.rows_w * pb * (double)pb, alg);
      IBMI_TRY(with_bn(g.bn, [&](auto bnc) -> ibmi_status {
        IBMI_CUDA_TRY(tc::launch_oz_pairs<decltype(bnc)::value>(maps, w, st));
        return IBMI_OK;
      }));
    }
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    for (int k = 0; k < K; ++k) {
      note_launch();
      k_b_wcombine<<<dim3(nblk(ldp), (unsigned)g.m[k], (unsigned)n), 256, 0, st>>>(
          g.TW, (int64_t)cap * g.rows_w * ldp, g.rows_w, g.woff[k], g.m[k], pb, ldp, g.expW, g.expA, g.lo[k], g.hi[k],
          g.Ws[0][k], g.Ws[1][k], g.Ws[2][k]);
    }
    note_launch();
    k_b_init_h<<<dim3(nblk(ldp), (unsigned)pb, (unsigned)n), 256, 0, st>>>(pb, ldp, g.Hf, g.Hs[0], g.Hs[1], g.Hs[2]);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  {  // NOT_SPD blocks
    std::vector<DevStatus> hs(n * K);
    IBMI_CUDA_TRY(cudaMemcpyAsync(hs.data(), g.F.dstatus, sizeof(DevStatus) * n * K, cudaMemcpyDeviceToHost, st));
    IBMI_CUDA_TRY(cudaStreamSynchronize(st));
    for (int b = 0; b < n; ++b) {
      flops[b] += fplan;
      for (int k = 0; k < K; ++k)
        if (hs[b * K + k].code == IBMI_ERR_NOT_SPD && ms[b].phase != FAILED) {
          ms[b].phase = FAILED;
          res[b].status = IBMI_ERR_NOT_SPD;
          res[b].bad_block = k;
          res[b].bad_pivot = hs[b * K + k].pivot;
        }
    }
  }
  const double tol = o.tol;
  const int max_sweeps = o.max_sweeps, ns_max = o.ns_max;
  // --- rounds
  std::vector<int> hsel(16 * cap);
  std::vector<double> hout(4 * n);
  g.rounds = 0;
  for (int round = 0;; ++round) {
    g.rounds = round;
    // Matrices ready to enter the tail (or to certify) wait while more
    // matrices are still sweeping than are waiting, so that tails run
    // together and their launches cover many matrices; the slowest
    // matrix's own path is not lengthened.
    int nsweep = 0, nwait = 0;
    for (int b = 0; b < n; ++b) {
      nsweep += ms[b].phase == SWEEP;
      nwait += ms[b].phase == TAIL && ms[b].waiting;
    }
    if (nwait >= std::max(1, nsweep))
      for (int b = 0; b < n; ++b) ms[b].waiting = false;
    // selection lists of this round
    std::vector<int> L[2], Lres, Lsw, Lexp, Lupd, Lrx, Lrs, Ldir, Lcor;
    std::vector<int> qlo, qhi, csub;   // digit-group range and correction flag of each residual (positions of Lrs)
    for (int b = 0; b < n; ++b) {
      MState& m = ms[b];
      if (m.phase == SWEEP) {
        L[m.level].push_back(b);
        Lsw.push_back(b);
        if (m.reslice) Lres.push_back(b);
      } else if (m.phase == TAIL && !m.waiting) {
        if (m.act == T_ENTER || m.act == T_CERTIFY) Lexp.push_back(b);
        if (m.act == T_STEP) Lupd.push_back(b);
        if (m.act == T_STEP && m.xo_delta) Lrx.push_back(b);
        const bool corr = m.act == T_STEP && m.corr;
        Lrs.push_back(b);
        (corr ? Lcor : Ldir).push_back(b);
        csub.push_back(corr ? 1 : 0);
        qlo.push_back(m.act == T_EXTEND ? m.qc + 1 : 0);
        qhi.push_back(m.act == T_EXTEND ? OZ_QMAX : m.next_q);
      }
    }
    if (Lsw.empty() && Lrs.empty()) break;   // (waiting matrices are released once nothing sweeps)
    // upload all lists of the round at once
    int nsel = 0;
    auto put = [&](const std::vector<int>& v) -> int* {
      if (v.empty() || nsel + (int)v.size() > 16 * cap) return nullptr;
      int* dptr = g.dsel + nsel;
      std::copy(v.begin(), v.end(), hsel.begin() + nsel);
      nsel += (int)v.size();
      return dptr;
    };
    int* dL0 = put(L[0]);
    int* dL1 = put(L[1]);
    int* dLres = put(Lres);
    int* dLsw = put(Lsw);
    int* dLexp = put(Lexp);
    int* dLupd = put(Lupd);
    int* dLrx = put(Lrx);
    int* dLrs = put(Lrs);
    int* dLdir = put(Ldir);
    int* dLcor = put(Lcor);
    int* dqm = put(qhi);
    int* dcsub = put(csub);
    std::vector<int> qr2;
    for (size_t i = 0; i < qlo.size(); ++i) {
      qr2.push_back(qlo[i]);
      qr2.push_back(qhi[i]);
    }
    if (nsel & 1) put(std::vector<int>{0});   // int2 alignment
    const int2* dqr = (const int2*)put(qr2);
    if (nsel) IBMI_CUDA_TRY(cudaMemcpyAsync(g.dsel, hsel.data(), sizeof(int) * nsel, cudaMemcpyHostToDevice, st));
    // --- sweeps
    if (!Lres.empty()) {
      note_launch();
      k_b_reslice<<<dim3(nblk(ldp), (unsigned)pb, (unsigned)Lres.size()), 256, 0, st>>>(dLres, pb, ldp, g.Hf,
                                                                                        g.Hs[0], g.Hs[1], g.Hs[2]);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    for (int k = 0; k < K && !Lsw.empty(); ++k) {
      const int64_t lo = g.lo[k], hi = g.hi[k], m = g.m[k], nn = pb - m;
      const tc::TileRanges kr = tc::complement_tiles(lo, hi, pb, tc::BK);
      const tc::TileRanges nr = tc::complement_tiles(lo, hi, pb, kBN);
      for (int lev = 0; lev < 2; ++lev) {
        if (L[lev].empty()) continue;
        const int S = lev == 0 ? 2 : 3;
        int* dl = lev == 0 ? dL0 : dL1;
        const int nl = (int)L[lev].size();
        {  // a3: X = -W T
          tc::Maps maps;
          for (int s = 0; s < S; ++s) {
            maps.a[s] = g.mapW[s][k];
            maps.b[s] = g.mapH[s];
          }
          tc::Tiles t{m, 0, 0, nr.r0_end, nr.r1_begin, kr.r0_end, kr.r1_begin, kr.r1_end, 1, g.err};
          t.nb = nl;
          t.bsel = dl;
          EpiBSweepX epi;
          epi.Hf = g.Hf; epi.H0 = g.Hs[0]; epi.H1 = g.Hs[1]; epi.H2 = S == 3 ? g.Hs[2] : nullptr;
          epi.ldp = ldp; epi.lo = lo; epi.hi = hi; epi.p = pb; epi.m = m; epi.bstride = pl;
          ProfScope ps(IBMI_K_SWEEP_X, st, (S == 2 ? 3.0 : 6.0) * 2.0 * nl * m * nn * nn, 2.0 * nl * m * nn * nn);
          if (S == 2) IBMI_CUDA_TRY((tc::launch<2, kBN>(maps, t, nr.count(), (int)((m + 127) / 128), epi, st)));
          else IBMI_CUDA_TRY((tc::launch<3, kBN>(maps, t, nr.count(), (int)((m + 127) / 128), epi, st)));
        }
        {  // a4: P = X W^T (lower tiles; one K split, so that a matrix's sums do not
           // depend on its group: the group's matrices fill the GPU) and
           // H[I, I] = A_I^{-1} - P in the epilogue
          tc::Maps maps;
          for (int s = 0; s < S; ++s) {
            maps.a[s] = g.mapH[s];
            maps.b[s] = g.mapW[s][k];
          }
          const int ntn = (int)((m + kBN - 1) / kBN);
          tc::Tiles t{m, lo, 0, ntn, ntn, kr.r0_end, kr.r1_begin, kr.r1_end, 1, g.err};
          t.lower = 1;
          t.nb = nl;
          t.bsel = dl;
          EpiBSymFinish epi;
          epi.Ainv = g.F.pool + g.aoff[k]; epi.abstride = g.ainv_total; epi.m = m; epi.lo = lo; epi.pb = pb;
          epi.ldp = ldp; epi.Hf = g.Hf; epi.s0 = g.Hs[0]; epi.s1 = g.Hs[1]; epi.s2 = S == 3 ? g.Hs[2] : nullptr;
          ProfScope ps(IBMI_K_SWEEP_S, st,
                       (S == 2 ? 3.0 : 6.0) * 2.0 * nl * nn * (double)(ntn * (ntn + 1) / 2) * kBN * kBN,
                       2.0 * nl * m * m * nn);
          if (S == 2) IBMI_CUDA_TRY((tc::launch<2, kBN>(maps, t, ntn, (int)((m + 127) / 128), epi, st)));
          else IBMI_CUDA_TRY((tc::launch<3, kBN>(maps, t, ntn, (int)((m + 127) / 128), epi, st)));
        }
      }
    }
    if (!Lsw.empty()) {  // BF16x3 stop test of every sweeping matrix
      tc::Maps maps;
      maps.a[0] = g.mapH[0];
      maps.a[1] = g.mapH[1];
      maps.b[0] = g.mAf[0];
      maps.b[1] = g.mAf[1];
      const int nkt = (int)((pb + tc::BK - 1) / tc::BK);
      const int grid_n = (int)((pb + kBN - 1) / kBN), grid_m = (int)((pb + 127) / 128);
      tc::Tiles t{pb, 0, 0, grid_n, 0, 0, 0, nkt, 1, g.err};
      t.nb = (int)Lsw.size();
      t.bsel = dLsw;
      EpiBResidSq epi;
      epi.partials = g.partials;
      epi.nparts = g.nparts_r;
      epi.p = pb;
      {
        ProfScope ps(IBMI_K_RESIDUAL, st, 3.0 * 2.0 * (double)Lsw.size() * fr / 2.0, (double)Lsw.size() * fr);
        IBMI_CUDA_TRY((tc::launch<2, kBN>(maps, t, grid_n, grid_m, epi, st)));
      }
      note_launch();
      k_b_sum<<<(unsigned)Lsw.size(), 256, 0, st>>>(dLsw, g.partials, g.nparts_r, g.din, g.dout);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    // --- tail: exports, updates, then residuals (fresh by digit groups, or extended)
    if (!Lexp.empty()) {
      note_launch();
      k_b_export<<<dim3(nblk(pb), (unsigned)pb, (unsigned)Lexp.size()), 256, 0, st>>>(dLexp, pb, ldp, g.Hf, g.X64);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    auto pairs = [&](const CUtensorMap* ma, int nsa, const CUtensorMap* mb, int nsb, int qmin, int qmax, int* dl,
                     int nl, int kclass, double alg, const int2* qr, int lower = 0) -> ibmi_status {
      tc::OzPairMaps maps;
      for (int s = 0; s < nsa; ++s) maps.a[s] = ma[s];
      for (int u = 0; u < nsb; ++u) maps.b[u] = mb[u];
      tc::OzPairArgs a{};
      int np = 0;
      for (int q = qmin; q <= qmax; ++q) {
        bool first = true;
        for (int s = 0; s <= q; ++s) {
          const int u = q - s;
          if (s >= nsa || u >= nsb) continue;
          a.s[np] = (int8_t)s;
          a.u[np] = (int8_t)u;
          a.q[np] = (int8_t)q;
          a.first[np] = first ? 1 : 0;
          first = false;
          ++np;
        }
      }
      a.n = np;
      a.grid_n = (int)((pb + g.bn - 1) / g.bn);
      a.tiles = a.grid_n * (int)((pb + 127) / 128);
      a.kt_total = (int)((pb + tc::BK - 1) / tc::BK);
      a.chunk = OZ_KCHUNK / tc::BK;
      a.T = g.T;
      a.plane = (int64_t)cap * pl;
      a.ldt = ldp;
      a.M = pb;
      a.N = pb;
      a.err = g.err;
      a.nb = nl;
      a.bsel = dl;
      a.tstride = pl;
      a.qr = qr;
      a.lower = lower;
      if (lower) a.tiles = tc::oz_lower_tiles((int)((pb + 127) / 128), a.grid_n, g.bn);
      tc::oz_make_segments(a);
      ProfScope ps(kclass, st, (lower ? 1.0 : 2.0) * np * (double)nl * pb * pb * (double)a.kt_total * tc::BK, alg);
      return with_bn(g.bn, [&](auto bnc) -> ibmi_status {
        IBMI_CUDA_TRY(tc::launch_oz_pairs<decltype(bnc)::value>(maps, a, st));
        return IBMI_OK;
      });
    };
    auto slice = [&](const double* src, __nv_bfloat16* const* planes, int ns, int* expo, int* dl, int nl) {
      SlicePtrs sp{};
      for (int s = 0; s < ns; ++s) sp.s[s] = planes[s];
      SliceRows a{src, pb, pb * pb, pb, pb, 0, pb, 0, ldp, ns, expo};
      ProfScope ps(IBMI_K_OTHER, st, 0.0);
      note_launch();
      k_b_slices<<<(unsigned)(nl * pb), 256, 0, st>>>(dl, a, sp);
      return cudaGetLastError();
    };
    if (!Lupd.empty()) {  // X <- sym(X + X Q^T) from the last residual's digits of X and Q
      const int nl = (int)Lupd.size();
      // after a correction the X planes hold its difference: the digits of X first
      if (!Lrx.empty()) IBMI_CUDA_TRY(slice(g.X64, g.Xo, NS_S, g.expX, dLrx, (int)Lrx.size()));
      IBMI_CUDA_TRY(slice(g.Q, g.Qo, NS_S, g.expQ, dLupd, nl));
      // X Q^T = X - X A X is symmetric (X is): its lower tiles only, mirrored
      IBMI_TRY(pairs(g.mXo, NS_S, g.mQo, NS_S, 0, NS_S - 1, dLupd, nl, IBMI_K_NS, 0.5 * nl * fr, nullptr, 1));
      ProfScope ps(IBMI_K_OTHER, st, 0.0);
      note_launch();
      const unsigned nt = (unsigned)((pb + 31) / 32);
      k_b_update_lower<<<dim3(nt, nt, (unsigned)nl), dim3(32, 8), 0, st>>>(
          dLupd, g.T, (int64_t)cap * pl, pb, ldp, g.expX, g.expQ, NS_S - 1, g.X64, g.Xprev);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    if (!Lrs.empty()) {  // residuals: fresh (groups 0..q), extended (qc+1..9) and corrections, one launch
      const int nl = (int)Lrs.size();
      // digits of X (prefix-stable), or of the step's difference X - Xprev for a correction
      if (!Ldir.empty()) IBMI_CUDA_TRY(slice(g.X64, g.Xo, OZ_SX, g.expX, dLdir, (int)Ldir.size()));
      if (!Lcor.empty()) IBMI_CUDA_TRY(slice(g.Xprev, g.Xo, OZ_SX, g.expX, dLcor, (int)Lcor.size()));
      int q0 = OZ_QMAX, q1 = 0;
      double alg = 0.0;
      for (int i = 0; i < nl; ++i) {
        q0 = std::min(q0, qlo[i]);
        q1 = std::max(q1, qhi[i]);
        alg += fr * count_pairs(OZ_SX, OZ_SA, qlo[i], qhi[i]) / full_pairs;
      }
      IBMI_TRY(pairs(g.mXo, OZ_SX, g.mAo, OZ_SA, q0, q1, dLrs, nl, IBMI_K_RESIDUAL, alg, dqr));
      ProfScope ps(IBMI_K_OTHER, st, 0.0);
      note_launch(2);
      k_b_combine<<<dim3(nblk((pb + 3) / 4), (unsigned)pb, (unsigned)nl), 256, 0, st>>>(
          dLrs, g.T, (int64_t)cap * pl, pb, ldp, g.expX, g.expA, dqm, dcsub, g.Q, g.partials, g.nparts_c);
      k_b_sum<<<(unsigned)nl, 256, 0, st>>>(dLrs, g.partials, g.nparts_c, g.din, g.dout);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    // --- read every value of the round (one synchronisation)
    int herr = 0;
    IBMI_CUDA_TRY(cudaMemcpyAsync(hout.data(), g.dout, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, st));
    IBMI_CUDA_TRY(cudaMemcpyAsync(&herr, g.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    IBMI_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr != 0) {
      set_last_error("tcgen05 kernel: bounded wait expired");
      return IBMI_ERR_TIMEOUT;
    }
    // --- decisions, matrix by matrix (the single-matrix pipeline's rules below order 2048)
    for (int b = 0; b < n; ++b) {
      MState& m = ms[b];
      const double rho = hout[4 * b];
      const double sqrtp = sqrt((double)mats[b].p);
      if (m.phase == SWEEP) {
        m.reslice = false;
        ++m.r;
        res[b].sweeps = m.r;
        flops[b] += fs + fr;
        res[b].resid_f = rho;
        m.last_cheap = rho;
        if (!isfinite(rho)) { m.phase = FAILED; res[b].status = IBMI_ERR_NONFINITE; continue; }
        if (theta > 0.0 && rho * sqrtp <= theta && rho <= m.handover_below) {
          m.phase = TAIL; m.act = T_ENTER; m.early = true; m.handover_rho = rho; m.s = 0;
          m.prev = INFINITY; m.exact = m.corr = m.xo_delta = false;
          m.next_q = rho <= tol ? OZ_QMAX : kFirstGroups;
          m.waiting = true;
          continue;
        }
        m.stalled = rho > 0.95 * m.best ? m.stalled + 1 : 0;
        m.best = fmin(m.best, rho);
        if (theta > 0.0 && m.stalled >= 3) {
          if (m.level == 0) {
            m.level = 1; m.stalled = 0; m.best = INFINITY; m.reslice = true;
          } else if (rho * sqrtp <= 8.0 * theta) {
            m.phase = TAIL; m.act = T_ENTER; m.early = false; m.handover_rho = rho; m.s = 0;
            m.prev = INFINITY; m.exact = m.corr = m.xo_delta = false;
            m.next_q = kFirstGroups;
            m.waiting = true;
            continue;
          } else {
            m.phase = FALLBACK;   // the single-matrix path measures the spectral radius here
            continue;
          }
        }
        if (rho <= tol || m.r >= max_sweeps) {   // BF16x3 cannot certify tol: the FP64-accurate residual
          m.phase = TAIL; m.act = T_CERTIFY; m.next_q = OZ_QMAX;
          m.exact = m.corr = m.xo_delta = false;
          m.waiting = true;
          continue;
        }
      } else if (m.phase == TAIL && !m.waiting) {
        const TailAct act = m.act;
        if (act == T_CERTIFY) {
          flops[b] += fr;
          res[b].resid_f = rho;
          if (rho <= tol) { m.phase = DONE; res[b].status = IBMI_OK; }
          else if (m.r >= max_sweeps || !isfinite(rho)) m.phase = FALLBACK;
          else { m.phase = SWEEP; m.act = T_NONE; }
          continue;
        }
        if (act == T_STEP) {
          flops[b] += fr;   // the update's 15 pairs
          ++m.s;
          res[b].ns_steps += 1;
        }
        const int qdone = act == T_EXTEND ? OZ_QMAX : m.next_q;
        flops[b] += fr * (act == T_EXTEND ? count_pairs(OZ_SX, OZ_SA, m.qc + 1, OZ_QMAX)
                                          : count_pairs(OZ_SX, OZ_SA, 0, qdone)) / full_pairs;
        m.qc = qdone;
        // a correction of an exact residual is exact (its groups reach below
        // 1% of tol, corr_groups), and so is a residual of all groups
        const bool was_corr = act == T_STEP && m.corr;
        m.exact = was_corr || m.qc == OZ_QMAX;
        m.xo_delta = was_corr;
        m.corr = false;
        const bool worse = m.s > 0 && !(rho < m.prev) && act != T_EXTEND;
        if (!worse) {
          res[b].resid_f = rho;
          if (!isfinite(rho)) { m.phase = FAILED; res[b].status = IBMI_ERR_NONFINITE; continue; }
          if (rho <= tol && !m.exact) { m.act = T_EXTEND; continue; }   // certify with all groups
          if (rho <= tol) { m.phase = DONE; res[b].status = IBMI_OK; continue; }
        }
        if (m.s >= ns_max || worse) {
          if (m.early && m.r < max_sweeps) {   // back to the sweeps, whose state the tail left untouched
            m.phase = SWEEP; m.act = T_NONE;
            m.handover_below = 0.5 * m.handover_rho;
            continue;
          }
          m.phase = FALLBACK;
          continue;
        }
        // one Newton-Schulz step, then the next residual: after an exact
        // one its correction Q - (X - Xprev) A
        m.prev = rho;
        m.act = T_STEP;
        const double rho_hat = rho * rho;
        m.corr = m.exact;
        m.next_q = m.corr ? tail::correction_groups(rho, tol, OZ_QMAX)
                          : (rho_hat <= tol ? OZ_QMAX : (rho * rho > 1e3 * tol ? kNextGroups : OZ_QMAX));
      }
    }
  }
  // results of the converged matrices
  std::vector<int> Ldone;
  for (int b = 0; b < n; ++b) {
    res[b].flops = flops[b];
    if (ms[b].phase == DONE) Ldone.push_back(b);
    if (ms[b].phase == FALLBACK) fallback[b] = 1;
    res[b].status = ms[b].phase == DONE ? IBMI_OK : (ms[b].phase == FAILED ? res[b].status : IBMI_NOT_CONVERGED);
  }
  if (!Ldone.empty()) {
    std::copy(Ldone.begin(), Ldone.end(), hsel.begin());
    IBMI_CUDA_TRY(cudaMemcpyAsync(g.dsel, hsel.data(), sizeof(int) * Ldone.size(), cudaMemcpyHostToDevice, st));
    note_launch();
    k_b_unpad<<<dim3(nblk(pb), (unsigned)pb, (unsigned)Ldone.size()), 256, 0, st>>>(g.din, g.dsel, pb, g.X64);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  return IBMI_OK;
}

}  // namespace ibmi
