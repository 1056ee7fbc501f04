// Integer-only conversions for the sliced products (internal).  GB300 runs
// FP64 arithmetic and conversions at a small fraction of its integer rate, so
// the elementwise kernels that recombine digit groups build their FP64 results
// from integers directly.  Host-compilable (no CUDA types) for exhaustive
// checks on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OZR_HD __host__ __device__ __forceinline__
#else
#define OZR_HD inline
#endif

namespace ibmi {

OZR_HD int ozr_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

OZR_HD double ozr_bits_to_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

OZR_HD uint64_t ozr_double_to_bits(double d) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}

// The double nearest to (hi * 2^35 + lo) * 2^s (ties to even), for signed
// |hi|, |lo| < 2^62, with integer operations only.  Results that would be
// subnormal or overflow are flagged through *exact_ok = false (the caller then
// takes an FP64 path); they do not occur for the scales of a residual.
OZR_HD double ozr_round(int64_t hi, int64_t lo, int s, bool* exact_ok) {
  // 128-bit two's complement value (H:L) = hi * 2^35 + lo
  uint64_t L = (uint64_t)hi << 35;
  int64_t H = hi >> 29;
  const uint64_t L2 = L + (uint64_t)lo;
  H += (lo < 0 ? -1 : 0) + (L2 < L ? 1 : 0);
  L = L2;
  const bool neg = H < 0;
  uint64_t uH = (uint64_t)H;
  if (neg) {   // magnitude
    L = ~L + 1;
    uH = ~uH + (L == 0 ? 1 : 0);
  }
  *exact_ok = true;
  if (uH == 0 && L == 0) return neg ? -0.0 : 0.0;
  int msb = uH ? 127 - ozr_clz64(uH) : 63 - ozr_clz64(L);   // highest set bit
  const int sh = msb - 52;                                   // bits below the 53-bit significand
  uint64_t m;
  bool up = false;
  if (sh <= 0) {
    m = L << (-sh);   // msb <= 52 < 64: all of it in L, exact
  } else if (sh < 64) {
    m = (L >> sh) | (sh ? uH << (64 - sh) : 0);
    const bool guard = (L >> (sh - 1)) & 1;
    const bool sticky = (L & ((1ull << (sh - 1)) - 1)) != 0;
    up = guard && (sticky || (m & 1));
  } else if (sh == 64) {
    m = uH;
    const bool guard = L >> 63;
    const bool sticky = (L << 1) != 0;
    up = guard && (sticky || (m & 1));
  } else {
    const int t = sh - 64;   // 1 .. 63
    m = uH >> t;
    const bool guard = (uH >> (t - 1)) & 1;
    const bool sticky = (uH & ((1ull << (t - 1)) - 1)) != 0 || L != 0;
    up = guard && (sticky || (m & 1));
  }
  m += up ? 1 : 0;
  if (m >> 53) {   // rounding carried into a new leading bit
    m >>= 1;
    ++msb;
  }
  const int ex = msb + s + 1023;   // biased exponent of the leading bit
  if (ex <= 0 || ex >= 2047) {
    *exact_ok = false;
    return 0.0;
  }
  const uint64_t bits = ((uint64_t)(neg ? 1 : 0) << 63) | ((uint64_t)ex << 52) | (m & ((1ull << 52) - 1));
  return ozr_bits_to_double(bits);
}

// Nearest float (ties to even) of a finite double, with integer operations;
// below the float normal range it returns a signed zero, above it +-inf.
OZR_HD float ozr_to_float(double x) {
  const uint64_t b = ozr_double_to_bits(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);   // 53-bit significand (normal x)
  uint32_t out;
  if (((b >> 52) & 0x7ff) == 0 || e <= 0) {
    out = sign;
  } else {
    const bool guard = (m >> 28) & 1;
    const bool sticky = (m & ((1ull << 28) - 1)) != 0;
    uint64_t r = m >> 29;                                  // 24-bit significand
    r += (guard && (sticky || (r & 1))) ? 1 : 0;
    int ee = e;
    if (r >> 24) {
      r >>= 1;
      ++ee;
    }
    out = ee >= 255 ? (sign | 0x7f800000u) : (sign | ((uint32_t)ee << 23) | (uint32_t)(r & 0x7fffff));
  }
  float f;
#if defined(__CUDA_ARCH__)
  f = __uint_as_float(out);
#else
  memcpy(&f, &out, 4);
#endif
  return f;
}

// |x| as an unsigned integer with the order of |x| (finite x).
OZR_HD uint64_t ozr_abs_bits(double x) { return ozr_double_to_bits(x) & 0x7fffffffffffffffull; }

}  // namespace ibmi
