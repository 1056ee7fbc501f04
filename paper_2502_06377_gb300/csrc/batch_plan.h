// Host-side choices of the batched executor and the server: size buckets,
// the partitions (K, h) a bucket may use, and the Newton-Schulz hand-over.
// Plain C++ (no CUDA), so that the CPU tests compile it on its own.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <tuple>
#include <vector>

namespace ibmi {

struct Shape {
  int64_t p;   // padded order of the bucket
  int32_t K;   // sets
  int64_t h;   // half-overlap: end sets m + h, interior sets m + 2h (m = p / K)
  bool operator<(const Shape& o) const { return std::tie(p, K, h) < std::tie(o.p, o.K, o.h); }
};

// Padded order of a bucket: multiples of 64 up to 1024, of 128 up to 4096,
// of 256 beyond.
inline int64_t bucket_of(int64_t p) {
  const int64_t g = p <= 1024 ? 64 : (p <= 4096 ? 128 : 256);
  return (p + g - 1) / g * g;
}

// Default partition of a bucket when not tuned: ~256-row cores, 2..4 sets,
// overlap 2h = 20% of the core.
inline Shape default_shape(int64_t pb) {
  int32_t K = (int32_t)std::min<int64_t>(4, std::max<int64_t>(2, (pb + 255) / 256));
  int64_t h = std::max<int64_t>(8, (int64_t)std::llround(0.1 * (double)pb / K));
  return Shape{pb, K, h};
}

// The partition used when the tuned one does not converge for a matrix:
// cores of about 256 rows (2 to 8 sets), overlap 2h = 30% of the core.
// Smaller blocks keep the mixed-precision floor of the sweeps low.
inline Shape robust_shape(int64_t pb) {
  const int32_t K = (int32_t)std::min<int64_t>(8, std::max<int64_t>(2, pb / 256));
  const int64_t m = pb / K;
  return Shape{pb, K, std::max<int64_t>(4, (int64_t)std::llround(0.15 * (double)m))};
}

// Candidates the bucket tuner times: K in {2, 3, 4}, 2h in {10%, 20%, 30%}
// of the core width (overlaps below the core only).
inline std::vector<Shape> tune_candidates(int64_t pb) {
  std::vector<Shape> c;
  for (int32_t K = 2; K <= 4; ++K) {
    for (double f : {0.1, 0.2, 0.3}) {
      const int64_t m = pb / K;
      const int64_t h = std::max<int64_t>(4, (int64_t)std::llround(0.5 * f * (double)m));
      if (K * m < pb / 2 || 2 * h >= m) continue;
      c.push_back(Shape{pb, K, h});
    }
  }
  return c;
}

// Newton-Schulz hand-over threshold on ||I - A H||_F (mixed precision only):
// the caller's value if set; else 3 up to order 1024, where a sweep costs
// about as much as a tail step (both launch-latency bound) so the tail starts
// earlier, and 0.9 above.
inline double handover_theta(int64_t pb, bool mixed, double requested) {
  if (!mixed) return 0.0;
  return requested > 0.0 ? requested : (pb <= 1024 ? 3.0 : 0.9);
}

}  // namespace ibmi
