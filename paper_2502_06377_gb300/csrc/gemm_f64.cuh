// FP64 (DFMA) tiled GEMM with index-gap operand maps and functor epilogues.
//
// C[i, j] = sum_l opA(i, l) * opB(l, j) for i < M, j < N, l < K, where
//   opA(i, l) = A[mA(i) * lda + kA(l)]            (A_KMAJOR: row-major M x K)
//             = A[kA(l) * lda + mA(i)]            (otherwise: column-major)
//   opB(l, j) = B[kB(l) * ldb + nB(j)]            (B_NMAJOR: row-major K x N)
//             = B[nB(j) * ldb + kB(l)]            (otherwise: "B^T" storage)
// and every map is a GapMap (identity when len = 0).  The epilogue functor is
// called once per valid (i, j) with the FP64 accumulator.
//
// On GB300 FP64 runs at ~1.2 TFLOP/s (DFMA), about 1/60 of FP32 CUDA-core
// throughput, so this kernel is DFMA-bound by a wide margin: a 64 x 64 tile
// with a 4 x 4 register block per thread keeps shared-memory traffic at
// 0.5 loads per FMA and global traffic negligible.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace ibmi {

constexpr int F64_BM = 64, F64_BN = 64, F64_BK = 16, F64_THREADS = 256;

struct F64Operands {
  const double* A; int64_t lda; GapMap mA, kA;
  const double* B; int64_t ldb; GapMap kB, nB;
  int64_t M, N, K;
  int64_t zA = 0, zB = 0;   // element offset of operand z of a batch (blockIdx.z)
  int batch = 1;
  // Triangular K: opA(i, l) = 0 for l < i and opB(l, j) = 0 for l < j (e.g.
  // Y^T Y with Y lower triangular), so a tile starts its K loop at
  // max(first row, first column), rounded down to the K block.
  bool tri_k = false;
  // Symmetric result: tiles entirely above the diagonal are skipped (the
  // consumer reads element (i, j) with j > i from (j, i)).
  bool lower_tiles = false;
  // Symmetric A known by its lower triangle only (A_KMAJOR): element (r, c)
  // is read from (max(r, c), min(r, c)).
  bool a_lower = false;
  // If > 0: the batch size the tile choice below is made for (a batch of
  // several matrices' blocks then tiles each block as a batch of tile_batch
  // would, so a matrix's arithmetic does not depend on the others).
  int tile_batch = 0;
};

// Threads of a T x T tile: a 4 x 4 register block per thread for T = 64 and
// 4 x 2 for T = 32, so that a 32 x 32 tile runs four warps, one per SM
// partition (each partition's FP64 pipe takes about one FMA every other
// clock; two warps would leave half of the SM's DFMA rate idle when a small
// launch has one CTA per SM).
template <int T>
constexpr int f64_threads() { return (T / 4) * (T / (T == 64 ? 4 : 2)); }

template <bool A_KMAJOR, bool B_NMAJOR, class Epi, int T = F64_BM>
__global__ void __launch_bounds__(f64_threads<T>())
k_gemm_f64(F64Operands op, Epi epi) {
  // T x T output tile; thread (ty, tx) owns rows ty + QX x and columns tx + QY y.
  constexpr int RX = 4, RY = T == 64 ? 4 : 2, QX = T / RX, QY = T / RY, NT = QX * QY;
  static_assert(NT == f64_threads<T>() && T * F64_BK % NT == 0, "tile / thread layout");
  __shared__ double As[F64_BK][T + 1];
  __shared__ double Bs[F64_BK][T + 1];
  const int tx = threadIdx.x % QY, ty = threadIdx.x / QY;
  const int64_t i0 = (int64_t)blockIdx.y * T, j0 = (int64_t)blockIdx.x * T;
  if (op.lower_tiles && j0 >= i0 + T) return;
  op.A += blockIdx.z * op.zA;
  op.B += blockIdx.z * op.zB;
  double acc[RX][RY];
#pragma unroll
  for (int a = 0; a < RX; ++a)
#pragma unroll
    for (int b = 0; b < RY; ++b) acc[a][b] = 0.0;

  const int64_t lstart = op.tri_k ? (i0 > j0 ? i0 : j0) / F64_BK * F64_BK : 0;
  for (int64_t l0 = lstart; l0 < op.K; l0 += F64_BK) {
    // A tile: T x 16 values.
#pragma unroll
    for (int t = 0; t < T * F64_BK / NT; ++t) {
      int e = threadIdx.x + t * NT;
      int r, c;  // r: M within tile, c: K within tile
      if (A_KMAJOR) { r = e / F64_BK; c = e % F64_BK; } else { r = e % T; c = e / T; }
      int64_t i = i0 + r, l = l0 + c;
      double v = 0.0;
      if (i < op.M && l < op.K) {
        if (A_KMAJOR) {
          int64_t ra = op.mA(i), ca = op.kA(l);
          if (op.a_lower && ca > ra) {
            const int64_t t = ra;
            ra = ca;
            ca = t;
          }
          v = op.A[ra * op.lda + ca];
        } else {
          v = op.A[op.kA(l) * op.lda + op.mA(i)];
        }
      }
      As[c][r] = v;
    }
#pragma unroll
    for (int t = 0; t < T * F64_BK / NT; ++t) {
      int e = threadIdx.x + t * NT;
      int r, c;  // r: K within tile, c: N within tile
      if (B_NMAJOR) { r = e / T; c = e % T; } else { r = e % F64_BK; c = e / F64_BK; }
      int64_t l = l0 + r, j = j0 + c;
      double v = 0.0;
      if (l < op.K && j < op.N)
        v = B_NMAJOR ? op.B[op.kB(l) * op.ldb + op.nB(j)] : op.B[op.nB(j) * op.ldb + op.kB(l)];
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < F64_BK; ++k) {
      double a[RX], b[RY];
#pragma unroll
      for (int q = 0; q < RX; ++q) a[q] = As[k][ty + QX * q];
#pragma unroll
      for (int q = 0; q < RY; ++q) b[q] = Bs[k][tx + QY * q];
#pragma unroll
      for (int x = 0; x < RX; ++x)
#pragma unroll
        for (int y = 0; y < RY; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  epi.begin();
#pragma unroll
  for (int x = 0; x < RX; ++x)
#pragma unroll
    for (int y = 0; y < RY; ++y) {
      int64_t i = i0 + ty + QX * x, j = j0 + tx + QY * y;
      if (i < op.M && j < op.N) epi(i, j, acc[x][y]);
    }
  epi.end();
}

// ---------------------------------------------------------------- epilogues --

// C[i*ldc + j] = alpha * acc + beta * C[i*ldc + j]   (beta == 0 never reads C)
struct EpiStore {
  double* C; int64_t ldc; double alpha, beta;
  int64_t zC = 0;
  __device__ void begin() { C += blockIdx.z * zC; }
  __device__ void end() {}
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    double* c = C + i * ldc + j;
    *c = beta == 0.0 ? alpha * acc : fma(beta, *c, alpha * acc);
  }
};

// Sweep product a3: X = -W T, written to H[lo + i, phys(j)] and H[phys(j), lo + i].
struct EpiSweepX {
  double* H; int64_t ldh; int64_t lo; GapMap nmap;
  __device__ void begin() {}
  __device__ void end() {}
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    int64_t jp = nmap(j), ip = lo + i;
    double x = -acc;
    H[ip * ldh + jp] = x;
    H[jp * ldh + ip] = x;
  }
};

// Sweep product a4: S = A_I^{-1} - X W^T into scratch S (m x m, ld m).
struct EpiSweepS {
  const double* Ainv; double* S; int64_t m;
  __device__ void begin() {}
  __device__ void end() {}
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    S[i * m + j] = Ainv[i * m + j] - acc;
  }
};

// Residual: accumulate (delta_ij - acc)^2 and write one partial per CTA.
struct EpiResidual {
  double* partials;
  double s;
  __device__ void begin() { s = 0.0; }
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    double r = (i == j ? 1.0 : 0.0) - acc;
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

// Newton-Schulz: R = I - acc (store).
struct EpiIdentityMinus {
  double* R; int64_t ldr;
  __device__ void begin() {}
  __device__ void end() {}
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    R[i * ldr + j] = (i == j ? 1.0 : 0.0) - acc;
  }
};

// Newton-Schulz: Xn = X + acc.
struct EpiAddTo {
  const double* X; int64_t ldx; double* Xn; int64_t ldn;
  __device__ void begin() {}
  __device__ void end() {}
  __device__ __forceinline__ void operator()(int64_t i, int64_t j, double acc) {
    Xn[i * ldn + j] = X[i * ldx + j] + acc;
  }
};

// A launch of fewer than about two rounds of 64 x 64 tiles is latency-bound:
// one tile's K = 32 update is ~130 K DFMA, tens of microseconds on one SM of
// GB300 (about two FP64 FMAs per clock).  Store epilogues then use 32 x 32
// tiles, a quarter of the work per CTA and four times the CTAs.
constexpr int64_t F64_SMALL_LAUNCH = 300;

template <bool A_KMAJOR, bool B_NMAJOR, class Epi>
inline cudaError_t launch_gemm_f64(const F64Operands& op, const Epi& epi, cudaStream_t st) {
  if (op.M <= 0 || op.N <= 0) return cudaSuccess;
  const int64_t tiles64 =
      ((op.N + F64_BN - 1) / F64_BN) * ((op.M + F64_BM - 1) / F64_BM) * (op.tile_batch > 0 ? op.tile_batch : op.batch);
  note_launch();
  if constexpr (std::is_same<Epi, EpiStore>::value) {
    // triangular K: a 64 x 64 tile at the start of the diagonal sums all of K
    // on one SM; 32 x 32 tiles quarter that critical path
    if (tiles64 < F64_SMALL_LAUNCH || op.tri_k) {
      dim3 grid((unsigned)((op.N + 31) / 32), (unsigned)((op.M + 31) / 32), (unsigned)op.batch);
      k_gemm_f64<A_KMAJOR, B_NMAJOR, Epi, 32><<<grid, f64_threads<32>(), 0, st>>>(op, epi);
      return cudaGetLastError();
    }
  }
  dim3 grid((unsigned)((op.N + F64_BN - 1) / F64_BN), (unsigned)((op.M + F64_BM - 1) / F64_BM), (unsigned)op.batch);
  static_assert(f64_threads<F64_BM>() == F64_THREADS, "EpiResidual reduces over F64_THREADS");
  k_gemm_f64<A_KMAJOR, B_NMAJOR, Epi><<<grid, F64_THREADS, 0, st>>>(op, epi);
  return cudaGetLastError();
}

inline int64_t gemm_f64_ctas(int64_t M, int64_t N) {
  return ((N + F64_BN - 1) / F64_BN) * ((M + F64_BM - 1) / F64_BM);
}

}  // namespace ibmi
