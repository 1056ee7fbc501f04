// Per-row digit slicing and the exact recombination of digit-group sums of
// the error-free sliced products (Ozaki scheme), shared by the single-matrix
// refinement (refine.cu) and the batched engine (batch_dev.cu).  Internal.
#pragma once
#include <cuda_bf16.h>

#include "oz_round.h"
#include "refine.cuh"

namespace ibmi {


// One CTA per row: exponent e with max|row| < 2^e, then the fixed-point value
// F = rint(x 2^{55-e}) (|F| < 2^55) is cut into signed digits of weight
// 2^{49-7s}: d_s = round(F_s / 2^{49-7s}), F_{s+1} = F_s - d_s 2^{49-7s}
// (round half up, so F_{s+1} in [-2^{48-7s}, 2^{48-7s})).  Digits 7..9 come
// from F' = F_7 2^14 + rint((x 2^{55-e} - F) 2^14), the exact FP64 remainder
// of the 55-bit scaling carried 14 bits further.  All |d_s| <= 64.
struct SlicePtrs {
  __nv_bfloat16* s[OZ_S];
};

// The nslices digits of column c of a row whose maximum is below 2^e (zero
// outside [c0, c0 + ncols)): F = rint(x 2^{55-e}) and Flo = the remainder
// carried 14 bits further, from the bit pattern of x with integer operations
// only (no FP64 ALU), cut as described above; with `sq_on`, (x 2^-e)^2 is
// added to sq.
__device__ __forceinline__ void oz_elem_digits(const double* row, int64_t c, int64_t c0, int64_t ncols, int e,
                                               bool nonfinite, int nslices, bool sq_on, int (&d)[OZ_S], float& sq) {
  long long F = 0, Flo = 0;
  if (c >= c0 && c < c0 + ncols) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(row[c - c0]);
    const int ex = (int)((bits >> 52) & 0x7ff);
    const bool neg = (bits >> 63) != 0;
    if (ex != 0 && !nonfinite) {   // zeros and subnormals are far below 2^(e-69)
      const unsigned long long m = (bits & 0xfffffffffffffull) | 0x10000000000000ull;   // 53-bit significand
      const int sh = ex - 1075 + 55 - e;   // x 2^{55-e} = m 2^sh, sh <= 2 because |x| < 2^e
      if (sq_on) {   // |x| 2^-e ~ (m >> 29) 2^(ex - 1046 - e), 24 bits
        const float xs = ldexpf((float)(m >> 29), ex - 1046 - e);
        sq += xs * xs;
      }
      long long qq = 0, lo14 = 0;
      if (sh >= 0) {
        qq = (long long)(m << sh);
      } else if (sh > -68) {
        const int rs = -sh;
        if (rs >= 54) {   // |x 2^{55-e}| < 1/2: remainder only
          lo14 = (long long)(m >> (rs - 14));
        } else {
          const unsigned long long q = m >> rs;
          const unsigned long long rem = m - (q << rs);   // 0 <= rem < 2^rs
          const unsigned long long half = 1ull << (rs - 1);
          const bool up = rem >= half;                      // round half away from zero
          qq = (long long)q + (up ? 1 : 0);
          if (rs > 14)
            lo14 = up ? -(long long)(((half << 1) - rem) >> (rs - 14)) : (long long)(rem >> (rs - 14));
          else
            lo14 = up ? -(long long)(((half << 1) - rem) << (14 - rs)) : (long long)(rem << (14 - rs));
        }
      }
      F = neg ? -qq : qq;
      Flo = neg ? -lo14 : lo14;
    }
  }
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    const int sh = 49 - 7 * s;
    const long long dd = (F + (1ll << (sh - 1))) >> sh;
    F -= dd * (1ll << sh);
    d[s] = (int)dd;
  }
  if (nslices > 7) {
    long long G = F * 16384 + Flo;   // F = F_7 in [-64, 64)
#pragma unroll
    for (int s = 7; s < OZ_S; ++s) {
      const int sh = 14 - 7 * (s - 7);
      long long dd;
      if (s == OZ_S - 1 || sh == 0) {
        dd = G;
      } else {
        dd = (G + (1ll << (sh - 1))) >> sh;
        G -= dd * (1ll << sh);
      }
      d[s] = (int)dd;
    }
  }
}

// rowsq (optional): sum over the row of (x 2^-e)^2 in float, so that the
// row's squared norm is rowsq 2^(2e) (integer and float operations only).
// Called by all threads of a CTA for one row: `row` (ncols values, placed at
// columns [c0, c0 + ncols) of an ldp-wide output row, zero elsewhere), output
// row i of the planes, its exponent to expo[i] and its sum to rowsq[i].
__device__ __forceinline__ void oz_slice_row(const double* row, int64_t i, int64_t ncols, int64_t c0, int64_t ldp,
                                             const SlicePtrs& out, int nslices, int* expo, float* rowsq) {
  // row maximum of |x| on the bit patterns (integer order = order of |x|)
  unsigned long long mx = 0;
  for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) mx = max(mx, (unsigned long long)ozr_abs_bits(row[c]));
  __shared__ unsigned long long red[32];
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) v = max(v, (unsigned long long)__shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  int e = 0;   // max = f 2^e, f in [0.5, 1)
  const bool nonfinite = (red[0] >> 52) == 0x7ff;   // an Inf or NaN in the row
  if (red[0] != 0 && !nonfinite) {
    const int ef = (int)(red[0] >> 52);
    if (ef != 0) e = ef - 1022;
    else frexp(ozr_bits_to_double(red[0]), &e);   // subnormal maximum
  }
  if (threadIdx.x == 0) expo[i] = nonfinite ? OZ_NONFINITE_EXP : e;
  // Two adjacent columns per thread (ldp is even), stored as BF16 pairs.
  float sq = 0.f;
  for (int64_t c = 2 * (int64_t)threadIdx.x; c < ldp; c += 2 * (int64_t)blockDim.x) {
    int d0[OZ_S], d1[OZ_S];
    oz_elem_digits(row, c, c0, ncols, e, nonfinite, nslices, rowsq != nullptr, d0, sq);
    oz_elem_digits(row, c + 1, c0, ncols, e, nonfinite, nslices, rowsq != nullptr, d1, sq);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      if (s >= nslices) break;
      *reinterpret_cast<__nv_bfloat162*>(out.s[s] + i * ldp + c) =
          __halves2bfloat162(__int2bfloat16_rn(d0[s]), __int2bfloat16_rn(d1[s]));
    }
  }
  if (rowsq) {   // the same for every thread of the block
    __shared__ float sred[32];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sred[w];
      rowsq[i] = t;
    }
  }
}


// 2^k for integer k in the normal range, built from the exponent field.
__device__ __forceinline__ double pow2i(int k) {
  k = k < -1022 ? -1022 : (k > 1023 ? 1023 : k);
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// 2^e * sum_{qmin <= q <= qmax} T_q 2^{-7q} for the int32 group sums at
// `idx` of planes `plane` apart.  The sum is formed exactly in two int64
// halves (groups 0..4 and 5..qmax, each below 2^59), so only the final
// conversion and scaling round.
__device__ __forceinline__ double oz_groups_value(const int (&t)[10], int e);
__device__ __forceinline__ double oz_value(const int* T, int64_t plane, int64_t idx, int qmax, int e, int qmin = 0) {
  // all group loads issued together (predicated, no early exit)
  int t[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) t[q] = (q >= qmin && q <= qmax) ? T[(int64_t)q * plane + idx] : 0;
  return oz_groups_value(t, e);
}

// 2^e * sum_q t[q] 2^{-7q} (groups left out given as 0), as oz_value.
__device__ __forceinline__ double oz_groups_value(const int (&t)[10], int e) {
  long long hi = 0, lo = 0;
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    if (q < 5) hi += (long long)t[q] * (1ll << (7 * (4 - q)));
    else lo += (long long)t[q] * (1ll << (7 * (9 - q)));
  }
  if (e >= OZ_NONFINITE_EXP / 2) return __longlong_as_double(0x7ff8000000000000ll);   // a non-finite operand row
  // sum = (hi 2^35 + lo) 2^(e-63), rounded once, with integer operations
  bool ok;
  const double v = ozr_round(hi, lo, e - 63, &ok);
  return ok ? v : (double)hi * pow2i(e - 28) + (double)lo * pow2i(e - 63);
}


// x (FP32) ~ s0 + s1 + s2 with BF16 slices taken in turn from the remainder;
// the first two are the classic hi/lo pair (the operands of the BF16x3 sweep
// products).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  c = __float2bfloat16_rn(r - __bfloat162float(b));
}

}  // namespace ibmi
