// FP64-accurate residual (sliced error-free products on tcgen05) and the
// Newton-Schulz update of eq. newton, for the mixed-precision path.
#include <math.h>

#include <type_traits>

#include "refine.cuh"
#include "oz_pairs.cuh"
#include "oz_rows.cuh"

namespace ibmi {


// ------------------------------------------------------------ slicing ----
// (row slicing and group recombination: oz_rows.cuh)

__global__ void k_oz_slices(const double* X, int64_t ldx, int64_t ncols, int64_t c0, int64_t ldp, SlicePtrs out,
                            int nslices, int* expo, float* rowsq) {
  const int64_t i = blockIdx.x;
  oz_slice_row(X + i * ldx, i, ncols, c0, ldp, out, nslices, expo, rowsq);
}

__global__ void k_fsplit2(const double* X, int64_t ldx, int64_t p, int64_t ldp, __nv_bfloat16* s0,
                          __nv_bfloat16* s1) {
  const int64_t i = blockIdx.y, c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ldp) return;
  const int64_t idx = i * ldp + c;
  float x = c < p ? (float)X[i * ldx + c] : 0.f;
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  s0[idx] = h;
  s1[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// 2-D grids for the elementwise kernels: row = blockIdx.y, column =
// blockIdx.x * 256 + threadIdx.x (no 64-bit index division).
static inline dim3 grid2(int64_t cols, int64_t rows) {
  return dim3((unsigned)((cols + 255) / 256), (unsigned)rows);
}

// ---------------------------------------------------------- epilogues ----

// Group sum T_q[i, j] (+)= exact FP32 pair product (an integer below 2^24).
struct EpiOzAcc : tc::EpiBase {
  int* T; int64_t ldt, M, N; int first;
  // The warp's 32 x 16 block (rows row0.., columns j0..) from shared memory:
  // lane = (row 8k + lane/4, columns 4(lane%4)..+3), int4 read-modify-write,
  // 8 rows of 64 bytes per instruction.
  __device__ __forceinline__ void warp_tile(int64_t row0, int64_t j0, int, const float* __restrict__ stage,
                                            int lane) const {
    // all staged values into registers first, then the loads, then the stores
    const int c = (lane & 3) * 4, r0 = lane >> 2;
    int4 a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float* sv = stage + (8 * k + r0) * 17 + c;
      a[k] = make_int4(__float2int_rn(sv[0]), __float2int_rn(sv[1]), __float2int_rn(sv[2]), __float2int_rn(sv[3]));
    }
    int* __restrict__ t0 = T + (row0 + r0) * ldt + j0 + c;
    const bool full = j0 + c + 4 <= N;
    if (full) {
      int4 o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        o[k] = (first || row0 + 8 * k + r0 >= M) ? make_int4(0, 0, 0, 0)
                                                 : *reinterpret_cast<const int4*>(t0 + 8 * k * ldt);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (row0 + 8 * k + r0 >= M) continue;
        o[k].x += a[k].x;
        o[k].y += a[k].y;
        o[k].z += a[k].z;
        o[k].w += a[k].w;
        *reinterpret_cast<int4*>(t0 + 8 * k * ldt) = o[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (row0 + 8 * k + r0 >= M) continue;
        int* t = t0 + 8 * k * ldt;
        const int v[4] = {a[k].x, a[k].y, a[k].z, a[k].w};
        for (int u = 0; u < 4 && j0 + c + u < N; ++u) t[u] = (first ? 0 : t[u]) + v[u];
      }
    }
  }
};

// Cheap residual: per-thread sum of (delta_ij - acc)^2, one partial per warp.
struct EpiResidSq {
  double* partials; int64_t p;
  double s;
  __device__ __forceinline__ void operator()(int64_t i, int64_t j0, int, const float (&v)[16]) {
    if (i >= p) return;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (j0 + c < p) {
        double r = (i == j0 + c ? 1.0 : 0.0) - (double)v[c];
        s += r * r;
      }
    }
  }
  __device__ __forceinline__ void done(int q) {
    double x = s;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) {
      const int64_t cta = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
      partials[cta * 4 + q] = x;
    }
  }
};

// ------------------------------------------------------------ combine ----

// C = 2^{e_i + f_j - 12} sum_{qmin <= q <= qmax} T_q 2^{-7q};  Q = I - C, or
// with `sub` Q = Q - C in place (FP64, ld p); sum Q^2 per CTA, and (second
// half of `partials`) the sum of squares of the last group's part
// 2^{e_i + f_j - 12 - 7 qmax} T_qmax, whose norm scales the truncation error
// of the groups left out.  Four consecutive columns per thread: one int4
// load per group plane (the planes' row pitch ldp is a multiple of 64, so a
// load that starts below p stays inside the row).
__global__ void k_oz_combine(const int* T, int64_t p, int64_t ldp, const int* ex, const int* ea, int qmin,
                             int qmax, int sub, double* Q, double* partials) {
  const int64_t i = blockIdx.y, j0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  float sq = 0.f, gq = 0.f;
  if (j0 < p) {
    const int64_t plane = p * ldp, idx = i * ldp + j0;
    int4 t4[10];
#pragma unroll
    for (int q = 0; q < 10; ++q)
      t4[q] = (q >= qmin && q <= qmax) ? *reinterpret_cast<const int4*>(T + q * plane + idx) : make_int4(0, 0, 0, 0);
    const int exi = ex[i] - 12;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t j = j0 + c;
      if (j >= p) break;
      int t[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) t[q] = c == 0 ? t4[q].x : (c == 1 ? t4[q].y : (c == 2 ? t4[q].z : t4[q].w));
      const int e = exi + ea[j];
      const double v = oz_groups_value(t, e);
      int tl = 0;   // group qmax: float is ample for a norm estimate (parts below ~1e-19
                    // underflow to 0, an overflow reads as an infinite norm)
#pragma unroll
      for (int q = 0; q < 10; ++q)
        if (q == qmax) tl = t[q];
      const float g = ldexpf((float)tl, e - 7 * qmax);
      gq += g * g;
      const double qv = sub ? Q[i * p + j] - v
                            : (i == j ? 1.0 - v : ozr_bits_to_double(ozr_double_to_bits(v) ^ 0x8000000000000000ull));
      const float qf = ozr_to_float(qv);
      sq += qf * qf;
      Q[i * p + j] = qv;
    }
  }
  __shared__ double red[8], redg[8];
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    gq += __shfl_xor_sync(0xffffffffu, gq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = (double)sq;
    redg[threadIdx.x >> 5] = (double)gq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tt = 0.0, tg = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      tt += red[w];
      tg += redg[w];
    }
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x, nb = (int64_t)gridDim.x * gridDim.y;
    partials[b] = tt;
    partials[nb + b] = tg;
  }
}

// out[0] = sqrt(sum of partials[0 .. n)) / sqrt(p) (FP64 sum); with nout = 2
// also out[1] from partials[n .. 2n), and with row data of X and A (sqx: sum
// of (x 2^-ex)^2 per row) out[2] = ||X||_F ||A||_F / p.  The last two are
// estimates for planning and are summed in float (FP64 adds are scarce on
// this GPU and this kernel runs on one SM); the norms are scaled by the
// largest row exponent first.
__device__ __forceinline__ float block_sum_f(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[w];
  return t;
}
__device__ __forceinline__ int block_max_i(int v, int* sh) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = sh[0];
  for (int w = 1; w < (int)(blockDim.x / 32); ++w) t = max(t, sh[w]);
  return t;
}

__global__ void k_sum_partials(const double* partials, int64_t n, int64_t p, double* out, int nout = 1,
                               const float* sqx = nullptr, const int* ex = nullptr, const float* sqa = nullptr,
                               const int* ea = nullptr) {
  __shared__ double red[32];
  __shared__ float redf[32];
  __shared__ int redi[32];
  {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
      out[0] = sqrt(t) / sqrt((double)p);
    }
  }
  if (nout > 1) {
    float s = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (float)partials[n + i];
    const float t = block_sum_f(s, redf);
    if (threadIdx.x == 0) out[1] = sqrt((double)t) / sqrt((double)p);
  }
  if (sqx) {
    int mx = -(1 << 30), ma = -(1 << 30);
    for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
      mx = max(mx, ex[i]);
      ma = max(ma, ea[i]);
    }
    mx = block_max_i(mx, redi);
    ma = block_max_i(ma, redi);
    float sx = 0.f, sa = 0.f;
    for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
      sx += ldexpf(sqx[i], 2 * (ex[i] - mx));
      sa += ldexpf(sqa[i], 2 * (ea[i] - ma));
    }
    sx = block_sum_f(sx, redf);
    sa = block_sum_f(sa, redf);
    if (threadIdx.x == 0) out[2] = ldexp(sqrt((double)sx) * sqrt((double)sa), mx + ma) / (double)p;
  }
}

// D = X - Xprev (X row pitch ldx; Xprev and D row pitch p).
__global__ void k_diff(const double* X, int64_t ldx, const double* Xprev, int64_t p, double* D) {
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < p) D[i * p + j] = X[i * ldx + j] - Xprev[i * p + j];
}

// Newton-Schulz update: Xn = X + 2^{e_i + g_j - 12} sum_{q <= qmax} T_q 2^{-7q}.
// Four consecutive columns per thread, one int4 load per group plane (as
// k_oz_combine).
__global__ void k_oz_update(const int* T, int64_t p, int64_t ldp, const int* ex, const int* eq, int qmax,
                            const double* X, int64_t ldx, double* Xn) {
  const int64_t i = blockIdx.y, j0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (j0 >= p) return;
  const int64_t plane = p * ldp, idx = i * ldp + j0;
  int4 t4[10];
#pragma unroll
  for (int q = 0; q < 10; ++q)
    t4[q] = q <= qmax ? *reinterpret_cast<const int4*>(T + q * plane + idx) : make_int4(0, 0, 0, 0);
  const int exi = ex[i] - 12;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t j = j0 + c;
    if (j >= p) break;
    int t[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) t[q] = c == 0 ? t4[q].x : (c == 1 ? t4[q].y : (c == 2 ? t4[q].z : t4[q].w));
    Xn[i * p + j] = X[i * ldx + j] + oz_groups_value(t, exi + eq[j]);
  }
}

// The update of a symmetric X from the lower tiles of the product: X Q^T =
// X - X A X is symmetric, so X[i][j] + (X Q^T)[i][j] (j <= i) is written at
// (i, j) and (j, i), in place (one block per tile on or below the diagonal
// reads its elements before writing the mirror tile, which no block reads).
__global__ void k_oz_update_lower(const int* T, int64_t p, int64_t ldp, const int* ex, const int* eq, int qmax,
                                  double* X, int64_t ldx) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double t[32][33];
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = I0 + r, j = J0 + tx;
    if (i < p && j <= i) {
      const double v = X[i * ldx + j] + oz_value(T, p * ldp, i * ldp + j, qmax, ex[i] + eq[j] - 12);
      t[r][tx] = v;
      X[i * ldx + j] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = J0 + r, i = I0 + tx;   // element (j, i), the mirror of (i, j) with j < i
    if (i < p && j < i) X[j * ldx + i] = t[tx][r];
  }
}

// X = (Xn + Xn^T) / 2 by 32 x 32 tiles through shared memory (both the tile
// and its mirror read row-wise).
__global__ void k_sym_into(const double* Xn, int64_t p, double* X, int64_t ldx) {
  __shared__ double a[32][33], b[32][33];
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    a[r][tx] = (I0 + r < p && J0 + tx < p) ? Xn[(I0 + r) * p + J0 + tx] : 0.0;
    b[r][tx] = (J0 + r < p && I0 + tx < p) ? Xn[(J0 + r) * p + I0 + tx] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    if (I0 + r < p && J0 + tx < p) X[(I0 + r) * ldx + J0 + tx] = 0.5 * (a[r][tx] + b[tx][r]);
}

// Z = Y^T (m x m; Y row pitch ldy, Z row pitch m), 32 x 32 tiles through shared memory.
__global__ void k_transpose(const double* Y, int64_t ldy, int64_t m, double* Z) {
  __shared__ double t[32][33];
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    t[r][threadIdx.x] = (I0 + r < m && J0 + threadIdx.x < m) ? Y[(I0 + r) * ldy + J0 + threadIdx.x] : 0.0;
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    if (J0 + r < m && I0 + threadIdx.x < m) Z[(J0 + r) * m + I0 + threadIdx.x] = t[threadIdx.x][r];
}

// Ainv[i][j] = 2^{e_i + e_j - 12} sum_{q <= qmax} T_q 2^{-7q} (the product Z Z^T).
// From the group sums of the tiles on and below the diagonal (the product is
// symmetric): element (i, j), j <= i, written at (i, j) and (j, i), by 32 x 32
// tile pairs through shared memory.
__global__ void k_oz_gram(const int* T, int64_t plane, int64_t ldp, int64_t m, const int* ez, int qmax,
                          double* Ainv) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double t[32][33];
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = I0 + r, j = J0 + tx;
    if (i < m && j <= i) {
      const double v = oz_value(T, plane, i * ldp + j, qmax, ez[i] + ez[j] - 12);
      t[r][tx] = v;
      Ainv[i * m + j] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = J0 + r, i = I0 + tx;   // (j, i), the mirror of (i, j) with j < i
    if (i < m && j < i) Ainv[j * m + i] = t[tx][r];
  }
}

// Power iteration on the dense Q (p x p, row pitch p): y = Q v, one warp per row.
__global__ void k_q_gemv(const double* Q, int64_t p, const double* v, double* y) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= p) return;
  const double* row = Q + i * p;
  double s = 0.0;
  for (int64_t j = lane; j < p; j += 32) s += row[j] * v[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[i] = s;
}

// v = y / ||y||, est = ||y|| (one block); init: v = a fixed unit start vector
// with components of both signs and unequal sizes.
__global__ void k_q_normalize(const double* y, int64_t p, double* v, double* est, int init) {
  __shared__ double red[32];
  __shared__ double nrm;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
    const double t = init ? (1.0 + 0.37 * (double)(j % 5)) * ((j & 1) ? -1.0 : 1.0) : y[j];
    s += t * t;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    nrm = sqrt(t);
    if (!init) est[0] = nrm;
  }
  __syncthreads();
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
    const double t = init ? (1.0 + 0.37 * (double)(j % 5)) * ((j & 1) ? -1.0 : 1.0) : y[j];
    v[j] = t * inv;
  }
}

// --------------------------------------------------------------- host ----

static constexpr int RF_BN = 128;   // N tile of the BF16x3 residual
// N tile of the digit-pair GEMMs by order: 224 for large p (p = 4096 gives 608
// tiles of 128 x 224, four full rounds of 152 SMs, one CTA per SM); 128 and
// 64 for smaller p, where 224-wide tiles would be mostly padding and two
// CTAs fit on an SM (more matrices of a batch run side by side).
static int oz_bn_for(int64_t p) { return p > 1536 ? 224 : (p > 384 ? 128 : 64); }

// Calls f(std::integral_constant<int, BN>) for the tile width of R.
template <class F>
static ibmi_status with_bn(const RefineState* R, F&& f) {
  switch (R->bn) {
    case 224: return f(std::integral_constant<int, 224>{});
    case 128: return f(std::integral_constant<int, 128>{});
    default: return f(std::integral_constant<int, 64>{});
  }
}

ibmi_status refine_create(RefineState* R, int64_t p, int* err) {
  R->p = p;
  R->ldp = (p + 63) / 64 * 64;
  R->err = err;
  const int64_t ldp = R->ldp;
  const size_t plane16 = sizeof(__nv_bfloat16) * p * ldp;
  const int64_t tiles = ((p + 127) / 128) * ((p + RF_BN - 1) / RF_BN);
  R->n_partials = std::max<int64_t>(tiles * 4, 2 * p * ((p + 255) / 256)) + 8;
  size_t bytes = plane16 * (OZ_SA + OZ_SX + NS_S + 2) + sizeof(int) * (size_t)(OZ_QMAX + 1) * p * ldp +
                 2 * sizeof(double) * p * p + sizeof(double) * R->n_partials + 3 * sizeof(int) * p +
                 sizeof(double) * (2 * p + 8) + 2 * sizeof(float) * p + 64 * 256;
  if (cudaMalloc(&R->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IBMI_ERR_OOM;
  }
  uint8_t* q = (uint8_t*)R->pool;
  auto take = [&](size_t b) { uint8_t* r = q; q += (b + 255) / 256 * 256; return r; };
  for (int s = 0; s < OZ_SA; ++s) R->Ao[s] = (__nv_bfloat16*)take(plane16);
  for (int s = 0; s < OZ_SX; ++s) R->Xo[s] = (__nv_bfloat16*)take(plane16);
  for (int s = 0; s < NS_S; ++s) R->Qo[s] = (__nv_bfloat16*)take(plane16);
  for (int s = 0; s < 2; ++s) R->Af[s] = (__nv_bfloat16*)take(plane16);
  R->T = (int*)take(sizeof(int) * (size_t)(OZ_QMAX + 1) * p * ldp);
  R->Xn = (double*)take(sizeof(double) * p * p);
  R->Q = (double*)take(sizeof(double) * p * p);
  R->partials = (double*)take(sizeof(double) * R->n_partials);
  R->dout = (double*)take(256);
  R->expA = (int*)take(sizeof(int) * p);
  R->expX = (int*)take(sizeof(int) * p);
  R->expQ = (int*)take(sizeof(int) * p);
  R->pv = (double*)take(sizeof(double) * (2 * p + 8));
  R->sqA = (float*)take(sizeof(float) * p);
  R->sqX = (float*)take(sizeof(float) * p);
  bool ok = true;
  R->bn = oz_bn_for(p);
  for (int s = 0; s < OZ_SA; ++s) ok &= tc::make_map_bf16(&R->mAo[s], R->Ao[s], p, p, ldp, R->bn);
  for (int s = 0; s < OZ_SX; ++s) ok &= tc::make_map_bf16(&R->mXo[s], R->Xo[s], p, p, ldp, 128);
  for (int s = 0; s < NS_S; ++s) ok &= tc::make_map_bf16(&R->mQo[s], R->Qo[s], p, p, ldp, R->bn);
  for (int s = 0; s < NS_S; ++s) ok &= tc::make_map_bf16(&R->mXo_b[s], R->Xo[s], p, p, ldp, R->bn);
  for (int s = 0; s < 2; ++s) ok &= tc::make_map_bf16(&R->mAf[s], R->Af[s], p, p, ldp, RF_BN);
  return ok ? IBMI_OK : IBMI_ERR_CUDA;
}

void refine_destroy(RefineState* R) {
  cudaFree(R->pool);
  R->pool = nullptr;
  cudaFree(R->wpool);
  R->wpool = nullptr;
  R->w_rows = 0;
}

static ibmi_status slice_digits(RefineState* R, const double* X, int64_t ldx, __nv_bfloat16* const* dst, int nslices,
                                int* expo, cudaStream_t st, int64_t rows = -1, int64_t ncols = -1, int64_t c0 = 0,
                                float* rowsq = nullptr) {
  SlicePtrs sp;
  for (int s = 0; s < OZ_S; ++s) sp.s[s] = s < nslices ? dst[s] : nullptr;
  if (rows < 0) rows = R->p;
  if (ncols < 0) ncols = R->p;
  note_launch();
  k_oz_slices<<<(unsigned)rows, 256, 0, st>>>(X, ldx, ncols, c0, R->ldp, sp, nslices, expo, rowsq);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status refine_set_matrix(RefineState* R, const double* A, int64_t lda, cudaStream_t st) {
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  IBMI_TRY(slice_digits(R, A, lda, R->Ao, OZ_SA, R->expA, st, -1, -1, 0, R->sqA));
  note_launch();
  k_fsplit2<<<grid2(R->ldp, R->p), 256, 0, st>>>(A, lda, R->p, R->ldp, R->Af[0], R->Af[1]);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

static ibmi_status read_scalar(RefineState* R, cudaStream_t st, double* v) {
  int herr = 0;
  IBMI_CUDA_TRY(cudaMemcpyAsync(v, R->dout, sizeof(double), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaMemcpyAsync(&herr, R->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr != 0) {
    set_last_error("tcgen05 kernel: bounded wait expired");
    return IBMI_ERR_TIMEOUT;
  }
  return IBMI_OK;
}

// Digit-group sums T_q = sum_{s+u=q} (slice_s of the A operand) (slice_u of the
// B operand)^T for q <= qmax, over the K tiles [kt0, kt1): each pair an exact
// FP32 accumulation over at most 4096 terms, added up in int32 into the
// M x N (ld ldp) planes of T.
struct DigitGemm {
  const CUtensorMap* ma; int nsa;
  const CUtensorMap* mb; int nsb;
  int64_t M, N;
  int kt0, kt1;
  int qmax;
  int kclass;
  double alg_first = 0.0;   // algorithmic flops of the product (recorded with its first launch)
};

static ibmi_status digit_gemm(RefineState* R, DigitGemm g, cudaStream_t st) {
  const int64_t p = R->p, ldp = R->ldp;
  const int chunk_tiles = OZ_KCHUNK / tc::BK;
  const int BNr = R->bn;
  const int grid_n = (int)((g.N + BNr - 1) / BNr), grid_m = (int)((g.M + 127) / 128);
  for (int q = 0; q <= g.qmax; ++q) {
    bool first = true;
    for (int s = 0; s <= q; ++s) {
      const int u = q - s;
      if (s >= g.nsa || u >= g.nsb) continue;
      tc::Maps maps;
      maps.a[0] = g.ma[s];
      maps.b[0] = g.mb[u];
      for (int k0 = g.kt0; k0 < g.kt1; k0 += chunk_tiles) {
        const int k1 = std::min(g.kt1, k0 + chunk_tiles);
        // K tiles [k0, k1): an empty first range plus [k0, k1)
        tc::Tiles t{g.M, 0, 0, grid_n, 0, 0, k0, k1, 1, R->err};
        t.pdl = 1;   // digit planes are written only by the slicing kernels
        int* Tq = R->T + (int64_t)q * p * ldp;
        EpiOzAcc epi{{}, Tq, ldp, g.M, g.N, first ? 1 : 0};
        ProfScope ps(g.kclass, st, 2.0 * (double)g.M * g.N * (double)(k1 - k0) * tc::BK, g.alg_first);
        g.alg_first = 0.0;   // the product's algorithmic flops go with its first launch
        IBMI_TRY(with_bn(R, [&](auto bn) -> ibmi_status {
          IBMI_CUDA_TRY((tc::launch<1, decltype(bn)::value>(maps, t, grid_n, grid_m, epi, st)));
          return IBMI_OK;
        }));
        first = false;
      }
    }
  }
  return IBMI_OK;
}

// All pairs (s, u) with qmin <= s + u <= qmax of a p x p x p sliced product in
// one persistent launch (k_oz_pairs), in group order so that the first pair of
// each group stores and the others add (groups below qmin are left as they are).
static ibmi_status pair_products(RefineState* R, const CUtensorMap* ma, int nsa, const CUtensorMap* mb, int nsb,
                                 int qmax, int kclass, cudaStream_t st, int qmin = 0, int lower = 0) {
  const int64_t p = R->p, ldp = R->ldp;
  tc::OzPairMaps maps;
  for (int s = 0; s < nsa; ++s) maps.a[s] = ma[s];
  for (int u = 0; u < nsb; ++u) maps.b[u] = mb[u];
  tc::OzPairArgs g{};
  int n = 0;
  for (int q = qmin; q <= qmax; ++q) {
    bool first = true;
    for (int s = 0; s <= q; ++s) {
      const int u = q - s;
      if (s >= nsa || u >= nsb) continue;
      g.s[n] = (int8_t)s;
      g.u[n] = (int8_t)u;
      g.q[n] = (int8_t)q;
      g.first[n] = first ? 1 : 0;
      first = false;
      ++n;
    }
  }
  g.n = n;
  g.grid_n = (int)((p + R->bn - 1) / R->bn);
  g.tiles = g.grid_n * (int)((p + 127) / 128);
  g.kt_total = (int)((p + tc::BK - 1) / tc::BK);
  g.chunk = OZ_KCHUNK / tc::BK;
  g.T = R->T;
  g.plane = p * ldp;
  g.ldt = ldp;
  g.M = p;
  g.N = p;
  g.err = R->err;
  g.lower = lower;
  if (lower) g.tiles = tc::oz_lower_tiles((int)((p + 127) / 128), g.grid_n, R->bn);
  tc::oz_make_segments(g);
  // the method's share: these pairs out of all pairs of the full product
  // (52 for the residual, 15 for the Newton-Schulz update), of 2 p^3
  auto count_pairs = [](int na, int nb, int qm) {
    int c = 0;
    for (int q = 0; q <= qm; ++q)
      for (int a = 0; a <= q; ++a) c += (a < na && q - a < nb) ? 1 : 0;
    return c;
  };
  const int full = kclass == IBMI_K_NS ? count_pairs(NS_S, NS_S, NS_S - 1) : count_pairs(OZ_SX, OZ_SA, OZ_QMAX);
  ProfScope ps(kclass, st, (lower ? 1.0 : 2.0) * n * (double)p * p * (double)g.kt_total * tc::BK,
               (lower ? 1.0 : 2.0) * (double)p * p * p * n / full);
  return with_bn(R, [&](auto bn) -> ibmi_status {
    IBMI_CUDA_TRY(tc::launch_oz_pairs<decltype(bn)::value>(maps, g, st));
    return IBMI_OK;
  });
}

// W = A_I^{-1} A_{I,:} from digit products, written as BF16 hi/lo (zero on
// the columns of I and on the padding).
__global__ void k_oz_wcombine(const int* T, int64_t plane, int64_t m, int64_t p, int64_t ldp, const int* ea,
                              const int* eb, int qmax, int64_t lo, int64_t hi, __nv_bfloat16* W0, __nv_bfloat16* W1,
                              __nv_bfloat16* W2) {
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ldp) return;
  const int64_t idx = i * ldp + j;
  float w = 0.f;
  if (j < p && (j < lo || j >= hi)) {
    w = ozr_to_float(oz_value(T, plane, idx, qmax, ea[i] + eb[j] - 12));
  }
  const __nv_bfloat16 a = __float2bfloat16_rn(w);
  const float r = w - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r);
  W0[idx] = a;
  W1[idx] = b;
  W2[idx] = __float2bfloat16_rn(r - __bfloat162float(b));
}

ibmi_status refine_form_w(RefineState* R, const double* Ainv, int64_t m, int64_t lo, int64_t hi, __nv_bfloat16* W0,
                          __nv_bfloat16* W1, __nv_bfloat16* W2, cudaStream_t st) {
  const int64_t p = R->p, ldp = R->ldp;
  constexpr int NW_A = 5, NW_B = 4, QW = 4;   // 34-bit A_I^{-1} digits, 27-bit A digits
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    // A_I^{-1} embedded at columns [lo, hi) of an m x p operand (digit planes borrowed from X)
    IBMI_TRY(slice_digits(R, Ainv, m, R->Xo, NW_A, R->expX, st, m, m, lo));
  }
  IBMI_TRY(digit_gemm(R, DigitGemm{R->mXo, NW_A, R->mAo, NW_B, m, p, (int)(lo / tc::BK),
                                   (int)((hi + tc::BK - 1) / tc::BK), QW, IBMI_K_INVARIANTS_TC,
                                   2.0 * (double)m * m * (double)(p - m)}, st));
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  note_launch();
  k_oz_wcombine<<<grid2(ldp, m), 256, 0, st>>>(R->T, p * ldp, m, p, ldp, R->expX, R->expA, QW, lo, hi, W0, W1, W2);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status refine_plan_w(RefineState* R, const std::vector<int64_t>& lo, const std::vector<int64_t>& hi) {
  const int64_t p = R->p, ldp = R->ldp;
  const int K = (int)lo.size();
  R->w_rows = 0;
  R->w_off.assign(K, 0);
  int64_t rows = 0;
  for (int k = 0; k < K; ++k) {
    const int64_t m = hi[k] - lo[k];
    const int64_t kt = (hi[k] + tc::BK - 1) / tc::BK - lo[k] / tc::BK;
    if (kt * tc::BK > OZ_KCHUNK) return IBMI_OK;   // exactness bound per accumulation: set by set
    R->w_off[k] = rows;
    rows += (m + 127) / 128 * 128;
  }
  const size_t xregion = (size_t)((uint8_t*)R->Xo[OZ_SX - 1] - (uint8_t*)R->Xo[0]) + sizeof(__nv_bfloat16) * p * ldp;
  if (5 * sizeof(__nv_bfloat16) * (size_t)rows * ldp > xregion) return IBMI_OK;
  if (5 * (size_t)rows * ldp > (size_t)(OZ_QMAX + 1) * p * ldp) return IBMI_OK;
  const int tiles = (int)(rows / 128);
  if (cudaMalloc(&R->wpool, sizeof(int) * rows + sizeof(int2) * tiles + 256) != cudaSuccess) {
    cudaGetLastError();
    return IBMI_ERR_OOM;
  }
  R->expW = (int*)R->wpool;
  R->w_kr = (int2*)((uint8_t*)R->wpool + (sizeof(int) * rows + 255) / 256 * 256);
  std::vector<int2> kr(tiles);
  for (int k = 0; k < K; ++k) {
    const int64_t m = hi[k] - lo[k];
    for (int64_t t = R->w_off[k] / 128; t < (R->w_off[k] + m + 127) / 128; ++t)
      kr[t] = make_int2((int)(lo[k] / tc::BK), (int)((hi[k] + tc::BK - 1) / tc::BK));
  }
  IBMI_CUDA_TRY(cudaMemcpy(R->w_kr, kr.data(), sizeof(int2) * tiles, cudaMemcpyHostToDevice));
  for (int s = 0; s < 5; ++s)
    if (!tc::make_map_bf16(&R->mXw[s], R->Xo[0] + (int64_t)s * rows * ldp, rows, p, ldp, 128)) return IBMI_ERR_CUDA;
  R->w_rows = rows;
  return IBMI_OK;
}

ibmi_status refine_form_w_all(RefineState* R, const std::vector<const double*>& Ainv, const std::vector<int64_t>& lo,
                              const std::vector<int64_t>& hi, __nv_bfloat16* const* W0, __nv_bfloat16* const* W1,
                              __nv_bfloat16* const* W2, cudaStream_t st) {
  const int64_t p = R->p, ldp = R->ldp, rows = R->w_rows;
  const int K = (int)lo.size();
  constexpr int NW_A = 5, NW_B = 4, QW = 4;   // 34-bit A_I^{-1} digits, 27-bit A digits
  if (rows == 0) return IBMI_ERR_INVALID_ARG;
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    for (int k = 0; k < K; ++k) {   // A_I^{-1} at columns [lo, hi) of set k's slot
      const int64_t m = hi[k] - lo[k];
      __nv_bfloat16* dst[5];
      for (int s = 0; s < NW_A; ++s) dst[s] = R->Xo[0] + (int64_t)s * rows * ldp + R->w_off[k] * ldp;
      IBMI_TRY(slice_digits(R, Ainv[k], m, dst, NW_A, R->expW + R->w_off[k], st, m, m, lo[k]));
    }
  }
  double flops = 0.0;
  for (int k = 0; k < K; ++k)
    flops += 2.0 * (double)((hi[k] - lo[k] + 127) / 128 * 128) * p *
             (double)(((hi[k] + tc::BK - 1) / tc::BK - lo[k] / tc::BK) * tc::BK);
  const int grid_n = (int)((p + R->bn - 1) / R->bn), grid_m = (int)(rows / 128);
  double alg_w = 0.0;   // 2 m^2 (p - m) per set: W = A_I^{-1} A_{I, I^c}
  for (int k = 0; k < K; ++k) {
    const double m = (double)(hi[k] - lo[k]);
    alg_w += 2.0 * m * m * ((double)p - m);
  }
  // all pair products in one persistent launch, each row tile over its set's K range
  tc::OzPairMaps maps;
  for (int s = 0; s < NW_A; ++s) maps.a[s] = R->mXw[s];
  for (int u = 0; u < NW_B; ++u) maps.b[u] = R->mAo[u];
  tc::OzPairArgs g{};
  int n = 0;
  for (int q = 0; q <= QW; ++q) {
    bool first = true;
    for (int s = 0; s <= q; ++s) {
      const int u = q - s;
      if (s >= NW_A || u >= NW_B) continue;
      g.s[n] = (int8_t)s;
      g.u[n] = (int8_t)u;
      g.q[n] = (int8_t)q;
      g.first[n] = first ? 1 : 0;
      first = false;
      ++n;
    }
  }
  int kt_max = 1;
  for (int k = 0; k < K; ++k)
    kt_max = std::max<int>(kt_max, (int)((hi[k] + tc::BK - 1) / tc::BK - lo[k] / tc::BK));
  g.n = n;
  g.grid_n = grid_n;
  g.tiles = grid_n * grid_m;
  g.kt_total = kt_max;
  g.chunk = OZ_KCHUNK / tc::BK;
  g.T = R->T;
  g.plane = rows * ldp;
  g.ldt = ldp;
  g.M = rows;
  g.N = p;
  g.err = R->err;
  g.mkr = R->w_kr;
  tc::oz_make_segments(g);
  {
    ProfScope ps(IBMI_K_INVARIANTS_TC, st, flops * n, alg_w);
    IBMI_TRY(with_bn(R, [&](auto bn) -> ibmi_status {
      IBMI_CUDA_TRY(tc::launch_oz_pairs<decltype(bn)::value>(maps, g, st));
      return IBMI_OK;
    }));
  }
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  for (int k = 0; k < K; ++k) {
    const int64_t m = hi[k] - lo[k];
    note_launch();
    k_oz_wcombine<<<grid2(ldp, m), 256, 0, st>>>(R->T + R->w_off[k] * ldp, rows * ldp, m, p, ldp,
                                                 R->expW + R->w_off[k], R->expA, QW, lo[k], hi[k], W0[k], W1[k],
                                                 W2[k]);
  }
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status refine_read(RefineState* R, cudaStream_t st, double* rho) { return read_scalar(R, st, rho); }

ibmi_status refine_read_groups(RefineState* R, cudaStream_t st, double* rho, double* last_group, double* amp) {
  double v[3];
  int herr = 0;
  IBMI_CUDA_TRY(cudaMemcpyAsync(v, R->dout, sizeof(v), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaMemcpyAsync(&herr, R->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr != 0) {
    set_last_error("tcgen05 kernel: bounded wait expired");
    return IBMI_ERR_TIMEOUT;
  }
  *rho = v[0];
  *last_group = v[1];
  *amp = v[2];
  return IBMI_OK;
}

ibmi_status refine_q_radius_launch(RefineState* R, int iters, cudaStream_t st) {
  const int64_t p = R->p;
  double* v = R->pv;
  double* y = v + p;
  double* est = y + p;
  ProfScope ps(IBMI_K_OTHER, st, 2.0 * (double)iters * p * p);
  note_launch();
  k_q_normalize<<<1, 1024, 0, st>>>(y, p, v, est, 1);
  for (int it = 0; it < iters; ++it) {
    note_launch(2);
    k_q_gemv<<<(unsigned)((p + 7) / 8), 256, 0, st>>>(R->Q, p, v, y);
    k_q_normalize<<<1, 1024, 0, st>>>(y, p, v, est, 0);
  }
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status refine_block_inverse(RefineState* R, const double* Y, int64_t ldy, int64_t m, double* Ainv,
                                 cudaStream_t st) {
  const int64_t p = R->p, ldp = R->ldp;
  if (m < 1 || m > p) return IBMI_ERR_INVALID_ARG;
  constexpr int ND = 5, QG = 4;   // 34-bit digits, groups q <= 4
  double* Z = R->Xn;              // FP64 scratch (p x p)
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch();
    const unsigned nt = (unsigned)((m + 31) / 32);
    k_transpose<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(Y, ldy, m, Z);
    IBMI_CUDA_TRY(cudaGetLastError());
    // rows of Z, zero beyond column m (the last K block reads them)
    IBMI_TRY(slice_digits(R, Z, m, R->Xo, ND, R->expX, st, m, m, 0));
  }
  tc::OzPairMaps maps;
  for (int d = 0; d < ND; ++d) {
    maps.a[d] = R->mXo[d];
    maps.b[d] = R->mXo_b[d];
  }
  tc::OzPairArgs g{};
  int n = 0;
  for (int q = 0; q <= QG; ++q)
    for (int a = 0; a <= q; ++a) {
      g.s[n] = (int8_t)a;
      g.u[n] = (int8_t)(q - a);
      g.q[n] = (int8_t)q;
      g.first[n] = a == 0 ? 1 : 0;
      ++n;
    }
  g.n = n;
  g.grid_n = (int)((m + R->bn - 1) / R->bn);
  g.tiles = g.grid_n * (int)((m + 127) / 128);
  g.kt_total = (int)((m + tc::BK - 1) / tc::BK);
  g.chunk = OZ_KCHUNK / tc::BK;
  g.T = R->T;
  g.plane = p * ldp;
  g.ldt = ldp;
  g.M = m;
  g.N = m;
  g.err = R->err;
  g.lower = 1;   // Y^T Y is symmetric: the tiles on and below the diagonal
  g.tiles = tc::oz_lower_tiles((int)((m + 127) / 128), g.grid_n, R->bn);
  tc::oz_make_segments(g);
  {
    ProfScope ps(IBMI_K_INVARIANTS_TC, st, 1.0 * n * (double)m * m * (double)g.kt_total * tc::BK,
                 (double)m * m * m / 3.0);   // Y^T Y with triangular Y, lower half
    IBMI_TRY(with_bn(R, [&](auto bn) -> ibmi_status {
      IBMI_CUDA_TRY(tc::launch_oz_pairs<decltype(bn)::value>(maps, g, st));
      return IBMI_OK;
    }));
  }
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  note_launch();
  const unsigned nt = (unsigned)((m + 31) / 32);
  k_oz_gram<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(R->T, p * ldp, ldp, m, R->expX, QG, Ainv);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

// Rows of nbat stacked M-row operands, row r = b M + i of the output planes
// (row pitch ldo) from X + b zx + i ldx.
__global__ void k_oz_slices_bat(const double* X, int64_t ldx, int64_t zx, int64_t M, int64_t ncols, int64_t ldo,
                                SlicePtrs out, int nslices, int* expo) {
  const int64_t r = blockIdx.x, b = r / M, i = r - b * M;
  oz_slice_row(X + b * zx + i * ldx, r, ncols, 0, ldo, out, nslices, expo, nullptr);
}

// Z_b = B_b^T for the rows x cols blocks B_b = B + b zb (row pitch ldb); Z_b
// at Z + b rows cols, row pitch rows.
__global__ void k_transpose_rect(const double* B, int64_t ldb, int64_t zb, int64_t rows, int64_t cols, double* Z) {
  __shared__ double t[32][33];
  const int64_t b = blockIdx.z, I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const double* Bb = B + b * zb;
  double* Zb = Z + b * rows * cols;
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    t[r][threadIdx.x] = (I0 + r < rows && J0 + threadIdx.x < cols) ? Bb[(I0 + r) * ldb + J0 + threadIdx.x] : 0.0;
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y)
    if (J0 + r < cols && I0 + threadIdx.x < rows) Zb[(J0 + r) * rows + I0 + threadIdx.x] = t[threadIdx.x][r];
}

// C_b[i][j] -= 2^{ea_i + eb_j - 12} sum_{q <= qmax} T_q[i][j] 2^{-7q} for
// problem b = blockIdx.z (group planes at T + b tstride, exponents at
// ea + b M, eb + b N), on and below the diagonal only with `lower`.
__global__ void k_oz_sub_bat(const int* T, int64_t plane, int64_t ldt, int64_t tstride, const int* ea, const int* eb,
                             int qmax, int64_t M, int64_t N, int lower, double* C, int64_t ldc, int64_t zc) {
  const int64_t b = blockIdx.z, i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M || j >= N || (lower && j > i)) return;
  C[b * zc + i * ldc + j] -= oz_value(T + b * tstride, plane, i * ldt + j, qmax, ea[b * M + i] + eb[b * N + j] - 12);
}

// Digit pairs of groups <= QG of ND-digit operands (8 and 8 by default) for
// nbat problems: A
// operand rows in the X digit planes (nbat M rows), B operand rows in
// `bplanes` (nbat N rows), both at row pitch K; sums into the group planes
// (problem b at row b M).
static ibmi_status pairs_bat(RefineState* R, __nv_bfloat16* const* bplanes, int64_t M, int64_t N, int64_t K,
                             int64_t nbat, int lower, double alg, cudaStream_t st, int ND = 8, int QG = 8) {
  const int64_t p = R->p, ldp = R->ldp;
  tc::OzPairMaps maps;
  bool ok = true;
  for (int d = 0; d < ND; ++d) {
    ok &= tc::make_map_bf16_3d(&maps.a[d], R->Xo[d], nbat, M, K, K, 128);
    ok &= tc::make_map_bf16_3d(&maps.b[d], bplanes[d], nbat, N, K, K, R->bn);
  }
  if (!ok) return IBMI_ERR_CUDA;
  tc::OzPairArgs g{};
  int n = 0;
  for (int q = 0; q <= QG; ++q) {
    bool first = true;
    for (int a = 0; a <= q; ++a) {
      if (a >= ND || q - a >= ND) continue;
      g.s[n] = (int8_t)a;
      g.u[n] = (int8_t)(q - a);
      g.q[n] = (int8_t)q;
      g.first[n] = first ? 1 : 0;
      first = false;
      ++n;
    }
  }
  g.n = n;
  g.grid_n = (int)((N + R->bn - 1) / R->bn);
  g.lower = lower;
  g.tiles = lower ? tc::oz_lower_tiles((int)((M + 127) / 128), g.grid_n, R->bn) : g.grid_n * (int)((M + 127) / 128);
  g.kt_total = (int)(K / tc::BK);
  g.chunk = OZ_KCHUNK / tc::BK;
  g.T = R->T;
  g.plane = p * ldp;
  g.ldt = ldp;
  g.M = M;
  g.N = N;
  g.err = R->err;
  g.nb = (int)nbat;
  g.bsel = nullptr;
  g.tstride = M * ldp;
  tc::oz_make_segments(g);
  ProfScope ps(IBMI_K_INVARIANTS_TC, st, (lower ? 1.0 : 2.0) * n * (double)nbat * M * N * (double)K, alg);
  return with_bn(R, [&](auto bn) -> ibmi_status {
    IBMI_CUDA_TRY(tc::launch_oz_pairs<decltype(bn)::value>(maps, g, st));
    return IBMI_OK;
  });
}

// Ainv_b = 2^{e_i + e_j - 12} sum_{q <= qmax} T_q 2^{-7q} (the product Z Z^T,
// symmetric) for problem b = blockIdx.z: its leading m_b x m_b part at
// pool + off[b] (row pitch m_b), from the lower tiles, by 32 x 32 tile pairs.
__global__ void k_oz_gram_bat(const int* T, int64_t plane, int64_t ldt, int64_t tstride, int64_t mp, const int* ez,
                              int qmax, double* pool, const int64_t* off, const int64_t* dm) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double t[32][33];
  const int64_t b = blockIdx.z, m = dm[b];
  const int* Tb = T + b * tstride;
  const int* eb = ez + b * mp;
  double* Ainv = pool + off[b];
  const int64_t I0 = (int64_t)blockIdx.y * 32, J0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = I0 + r, j = J0 + tx;
    if (i < m && j <= i) {
      const double v = oz_value(Tb, plane, i * ldt + j, qmax, eb[i] + eb[j] - 12);
      t[r][tx] = v;
      Ainv[i * m + j] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = J0 + r, i = I0 + tx;
    if (i < m && j < i) Ainv[j * m + i] = t[tx][r];
  }
}

ibmi_status refine_block_inverse_all(RefineState* R, const double* Y, int64_t mmax, int64_t nbat, double* pool,
                                     const int64_t* doff, const int64_t* dm, cudaStream_t st) {
  constexpr int ND = 5, QG = 4;   // 34-bit digits, groups q <= 4 (15 pairs), as refine_block_inverse
  const int64_t p = R->p, ldp = R->ldp;
  if (mmax < 1 || mmax > p || nbat < 1) return IBMI_ERR_INVALID_ARG;
  const int64_t kp = (mmax + tc::BK - 1) / tc::BK * tc::BK;   // K padded to whole K blocks (zero digits)
  const int64_t per = std::max<int64_t>(1, std::min<int64_t>({nbat, p / mmax, (p * ldp) / (mmax * kp),
                                                              (p * p) / (mmax * mmax)}));
  for (int64_t b0 = 0; b0 < nbat; b0 += per) {
    const int64_t nn = std::min(per, nbat - b0);
    {
      ProfScope ps(IBMI_K_OTHER, st, 0.0);
      note_launch(2);
      const unsigned nt = (unsigned)((mmax + 31) / 32);
      k_transpose_rect<<<dim3(nt, nt, (unsigned)nn), dim3(32, 8), 0, st>>>(Y + b0 * mmax * mmax, mmax, mmax * mmax,
                                                                            mmax, mmax, R->Xn);
      SlicePtrs sa{};
      for (int d = 0; d < ND; ++d) sa.s[d] = R->Xo[d];
      k_oz_slices_bat<<<(unsigned)(nn * mmax), 256, 0, st>>>(R->Xn, mmax, mmax * mmax, mmax, mmax, kp, sa, ND,
                                                              R->expX);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    IBMI_TRY(pairs_bat(R, R->Xo, mmax, mmax, kp, nn, 1, (double)nn * mmax * mmax * mmax / 3.0, st, ND, QG));
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch();
    const unsigned nt = (unsigned)((mmax + 31) / 32);
    k_oz_gram_bat<<<dim3(nt, nt, (unsigned)nn), dim3(32, 8), 0, st>>>(R->T, p * ldp, ldp, mmax * ldp, mmax, R->expX,
                                                                      QG, pool, doff + b0, dm + b0);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  return IBMI_OK;
}

ibmi_status refine_syrk_sub(RefineState* R, const double* L, int64_t ldl, int64_t zl, int64_t M, int64_t nb,
                            double* C, int64_t ldc, int64_t zc, int64_t nbat, cudaStream_t st) {
  constexpr int ND = 8, QG = 8;   // 56-bit digits, groups q <= 8: 43 pair products
  const int64_t p = R->p, ldp = R->ldp;
  if (M <= 0 || nbat <= 0) return IBMI_OK;
  if (nb <= 0 || nb % tc::BK != 0 || nb > OZ_KCHUNK || M > p) return IBMI_ERR_INVALID_ARG;
  // problems per launch: their rows must fit the group planes (p rows) and
  // the digit planes (p ldp elements)
  const int64_t per = std::max<int64_t>(1, std::min<int64_t>({nbat, p / M, (p * ldp) / (M * nb)}));
  for (int64_t b0 = 0; b0 < nbat; b0 += per) {
    const int64_t nn = std::min(per, nbat - b0);
    {
      ProfScope ps(IBMI_K_OTHER, st, 0.0);
      SlicePtrs sp{};
      for (int d = 0; d < ND; ++d) sp.s[d] = R->Xo[d];
      note_launch();
      k_oz_slices_bat<<<(unsigned)(nn * M), 256, 0, st>>>(L + b0 * zl, ldl, zl, M, nb, nb, sp, ND, R->expX);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    IBMI_TRY(pairs_bat(R, R->Xo, M, M, nb, nn, 1, (double)nn * M * M * nb, st));
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch();
    k_oz_sub_bat<<<dim3((unsigned)((M + 255) / 256), (unsigned)M, (unsigned)nn), 256, 0, st>>>(
        R->T, p * ldp, ldp, M * ldp, R->expX, R->expX, QG, M, M, 1, C + b0 * zc, ldc, zc);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  return IBMI_OK;
}

ibmi_status refine_gemm_sub(RefineState* R, const double* A, int64_t lda, int64_t za, int64_t M, int64_t K,
                            const double* B, int64_t ldb, int64_t zb, int64_t N, double* C, int64_t ldc, int64_t zc,
                            int64_t nbat, cudaStream_t st) {
  constexpr int ND = 8, QG = 8;   // as refine_syrk_sub
  const int64_t p = R->p, ldp = R->ldp;
  if (M <= 0 || N <= 0 || nbat <= 0) return IBMI_OK;
  if (K <= 0 || K % tc::BK != 0 || K > OZ_KCHUNK || M > p || N > p) return IBMI_ERR_INVALID_ARG;
  const int64_t mn = std::max(M, N);
  const int64_t per = std::max<int64_t>(1, std::min<int64_t>({nbat, p / mn, (p * ldp) / (mn * K), (p * p) / (N * K)}));
  for (int64_t b0 = 0; b0 < nbat; b0 += per) {
    const int64_t nn = std::min(per, nbat - b0);
    {
      ProfScope ps(IBMI_K_OTHER, st, 0.0);
      note_launch(3);
      // B_b^T (N x K, row pitch K) into the FP64 scratch, then the rows of
      // A_b into the X digit planes and the rows of B_b^T into the A digit
      // planes (both at row pitch K)
      k_transpose_rect<<<dim3((unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32), (unsigned)nn), dim3(32, 8), 0,
                         st>>>(B + b0 * zb, ldb, zb, K, N, R->Xn);
      SlicePtrs sa{}, sb{};
      for (int d = 0; d < ND; ++d) {
        sa.s[d] = R->Xo[d];
        sb.s[d] = R->Ao[d];
      }
      k_oz_slices_bat<<<(unsigned)(nn * M), 256, 0, st>>>(A + b0 * za, lda, za, M, K, K, sa, ND, R->expX);
      k_oz_slices_bat<<<(unsigned)(nn * N), 256, 0, st>>>(R->Xn, K, N * K, N, K, K, sb, ND, R->expQ);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
    IBMI_TRY(pairs_bat(R, R->Ao, M, N, K, nn, 0, 2.0 * (double)nn * M * N * K, st));
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch();
    k_oz_sub_bat<<<dim3((unsigned)((N + 255) / 256), (unsigned)M, (unsigned)nn), 256, 0, st>>>(
        R->T, p * ldp, ldp, M * ldp, R->expX, R->expQ, QG, M, N, 0, C + b0 * zc, ldc, zc);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  return IBMI_OK;
}

ibmi_status refine_q_radius_read(RefineState* R, cudaStream_t st, double* radius) {
  IBMI_CUDA_TRY(cudaMemcpyAsync(radius, R->pv + 2 * R->p, sizeof(double), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  return IBMI_OK;
}

ibmi_status refine_residual(RefineState* R, const double* X, int64_t ldx, cudaStream_t st, double* rho) {
  IBMI_TRY(refine_residual_launch(R, X, ldx, st));
  return read_scalar(R, st, rho);
}

// Q = I - X A from the group sums q <= qmax (or, with `sub`, Q -= the part
// of groups qmin..qmax of the product in the planes) and ||Q||_F / sqrt(p)
// into dout[0]; with `nout` = 2 also the norm of group qmax's part into
// dout[1], with `stats` besides ||X||_F ||A||_F / p into dout[2] (the row
// sums of the last slicing of X).
static ibmi_status combine_residual(RefineState* R, int qmin, int qmax, bool sub, int nout, bool stats,
                                    cudaStream_t st) {
  const int64_t p = R->p, ldp = R->ldp;
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  const dim3 gc = grid2((p + 3) / 4, p);
  const int64_t nb = (int64_t)gc.x * gc.y;
  if (2 * nb > R->n_partials) return IBMI_ERR_INVALID_ARG;
  note_launch();
  k_oz_combine<<<gc, 256, 0, st>>>(R->T, p, ldp, R->expX, R->expA, qmin, qmax, sub ? 1 : 0, R->Q, R->partials);
  IBMI_CUDA_TRY(cudaGetLastError());
  note_launch();
  if (stats)
    k_sum_partials<<<1, 1024, 0, st>>>(R->partials, nb, p, R->dout, 2, R->sqX, R->expX, R->sqA, R->expA);
  else
    k_sum_partials<<<1, 1024, 0, st>>>(R->partials, nb, p, R->dout, nout);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status refine_residual_launch(RefineState* R, const double* X, int64_t ldx, cudaStream_t st, int qmax,
                                   bool stats) {
  const int64_t p = R->p, ldp = R->ldp;
  if (qmax < NS_S - 1 || qmax > OZ_QMAX) return IBMI_ERR_INVALID_ARG;
  const int nsx = std::min(OZ_SX, qmax + 1);   // digits of X that groups <= qmax use
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    IBMI_TRY(slice_digits(R, X, ldx, R->Xo, nsx, R->expX, st, -1, -1, 0, stats ? R->sqX : nullptr));
  }
  IBMI_TRY(pair_products(R, R->mXo, nsx, R->mAo, OZ_SA, qmax, IBMI_K_RESIDUAL, st));
  return combine_residual(R, 0, qmax, false, 1, stats, st);
}

ibmi_status refine_residual_extend_launch(RefineState* R, const double* X, int64_t ldx, cudaStream_t st, int qfrom,
                                          int qto, bool stats) {
  if (qfrom < NS_S - 1 || qto <= qfrom || qto > OZ_QMAX) return IBMI_ERR_INVALID_ARG;
  const int nsx_from = std::min(OZ_SX, qfrom + 1), nsx = std::min(OZ_SX, qto + 1);
  if (nsx > nsx_from) {   // the digits are prefix-stable: the first nsx_from come out the same
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    IBMI_TRY(slice_digits(R, X, ldx, R->Xo, nsx, R->expX, st));
  }
  IBMI_TRY(pair_products(R, R->mXo, nsx, R->mAo, OZ_SA, qto, IBMI_K_RESIDUAL, st, qfrom + 1));
  return combine_residual(R, 0, qto, false, 1, stats, st);
}

ibmi_status refine_residual_correct_launch(RefineState* R, const double* X, int64_t ldx, const double* Xprev,
                                           cudaStream_t st, int qmax) {
  const int64_t p = R->p;
  if (qmax < 0 || qmax > OZ_QMAX) return IBMI_ERR_INVALID_ARG;
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch();
    k_diff<<<grid2(p, p), 256, 0, st>>>(X, ldx, Xprev, p, R->Xn);
    IBMI_CUDA_TRY(cudaGetLastError());
    IBMI_TRY(slice_digits(R, R->Xn, p, R->Xo, std::min(OZ_SX, qmax + 1), R->expX, st));
  }
  IBMI_TRY(pair_products(R, R->mXo, std::min(OZ_SX, qmax + 1), R->mAo, OZ_SA, qmax, IBMI_K_RESIDUAL, st));
  return combine_residual(R, 0, qmax, true, 2, false, st);
}

ibmi_status refine_residual_correct_extend_launch(RefineState* R, cudaStream_t st, int qfrom, int qto) {
  if (qfrom < 0 || qto <= qfrom || qto > OZ_QMAX) return IBMI_ERR_INVALID_ARG;
  const int nsx_from = std::min(OZ_SX, qfrom + 1), nsx = std::min(OZ_SX, qto + 1);
  if (nsx > nsx_from) {   // D is still in the scratch; its first digits come out the same
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    IBMI_TRY(slice_digits(R, R->Xn, R->p, R->Xo, nsx, R->expX, st));
  }
  IBMI_TRY(pair_products(R, R->mXo, nsx, R->mAo, OZ_SA, qto, IBMI_K_RESIDUAL, st, qfrom + 1));
  return combine_residual(R, qfrom + 1, qto, true, 2, false, st);
}

ibmi_status refine_ns_update(RefineState* R, double* X, int64_t ldx, cudaStream_t st, int qmax, double* backup,
                             bool reslice_x, bool symmetric_x) {
  const int64_t p = R->p, ldp = R->ldp;
  if (qmax < 0 || qmax > NS_S - 1) return IBMI_ERR_INVALID_ARG;
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    if (reslice_x) IBMI_TRY(slice_digits(R, X, ldx, R->Xo, NS_S, R->expX, st));
    IBMI_TRY(slice_digits(R, R->Q, p, R->Qo, NS_S, R->expQ, st));
  }
  IBMI_TRY(pair_products(R, R->mXo, NS_S, R->mQo, NS_S, qmax, IBMI_K_NS, st, 0, symmetric_x ? 1 : 0));
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  if (symmetric_x) {
    if (backup)
      IBMI_CUDA_TRY(cudaMemcpy2DAsync(backup, sizeof(double) * p, X, sizeof(double) * ldx, sizeof(double) * p, p,
                                      cudaMemcpyDeviceToDevice, st));
    note_launch();
    const unsigned nt = (unsigned)((p + 31) / 32);
    k_oz_update_lower<<<dim3(nt, nt), dim3(32, 8), 0, st>>>(R->T, p, ldp, R->expX, R->expQ, qmax, X, ldx);
    IBMI_CUDA_TRY(cudaGetLastError());
    return IBMI_OK;
  }
  note_launch();
  k_oz_update<<<grid2((p + 3) / 4, p), 256, 0, st>>>(R->T, p, ldp, R->expX, R->expQ, qmax, X, ldx, R->Xn);
  IBMI_CUDA_TRY(cudaGetLastError());
  if (backup)
    IBMI_CUDA_TRY(cudaMemcpy2DAsync(backup, sizeof(double) * p, X, sizeof(double) * ldx, sizeof(double) * p, p,
                                    cudaMemcpyDeviceToDevice, st));
  note_launch();
  k_sym_into<<<dim3((unsigned)((p + 31) / 32), (unsigned)((p + 31) / 32)), dim3(32, 8), 0, st>>>(R->Xn, p, X, ldx);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status refine_cheap_residual_launch(RefineState* R, const CUtensorMap* mapH2, cudaStream_t st) {
  const int64_t p = R->p;
  tc::Maps maps;
  maps.a[0] = mapH2[0];
  maps.a[1] = mapH2[1];
  maps.b[0] = R->mAf[0];
  maps.b[1] = R->mAf[1];
  const int nkt = (int)((p + tc::BK - 1) / tc::BK);
  const int grid_n = (int)((p + RF_BN - 1) / RF_BN), grid_m = (int)((p + 127) / 128);
  int grid = 0;
  {
    ProfScope ps(IBMI_K_RESIDUAL, st, 3.0 * 2.0 * (double)p * p * p, 2.0 * (double)p * p * p);
    tc::Tiles t{p, 0, 0, grid_n, 0, 0, 0, nkt, 1, R->err};
    EpiResidSq epi{R->partials, p, 0.0};
    IBMI_CUDA_TRY((tc::launch<2, RF_BN>(maps, t, grid_n, grid_m, epi, st, &grid)));
  }
  const int64_t nparts = (int64_t)grid * 4;   // one partial per epilogue warp of each (persistent) CTA
  if (nparts > R->n_partials) return IBMI_ERR_INVALID_ARG;
  {
    ProfScope ps(IBMI_K_OTHER, st, 0.0);
    note_launch();
    k_sum_partials<<<1, 1024, 0, st>>>(R->partials, nparts, p, R->dout);
    IBMI_CUDA_TRY(cudaGetLastError());
  }
  return IBMI_OK;
}

}  // namespace ibmi
