// Stop-test cadence of the sweeps (Algorithm 1 tests after every sweep; here
// the test, as costly as a sweep, is spaced by the contraction seen so far).
// Plain C++ (no CUDA), so that the CPU tests compile it on its own.
#pragma once
#include <algorithm>
#include <cmath>

namespace ibmi {

// Stop-test cadence (a6 is as costly as a sweep): after a check, the
// per-sweep contraction f seen since the previous check predicts how many
// sweeps the residual needs to reach `target`; the next check comes after
// about half of them (at least `gmin`, at most 8 sweeps).
struct CheckCadence {
  int gmin = 1;
  int next = 1;
  int last_r = 0;
  double last_rho = 0.0;
  double f = 0.0;   // contraction per sweep between the last two tests (0: unknown)
  void after(int r, double rho, double target) {
    int gap = gmin;
    if (last_r > 0 && rho > 0.0 && last_rho > rho) f = std::pow(rho / last_rho, 1.0 / (double)(r - last_r));
    else f = 0.0;
    if (f > 0.0 && target > 0.0 && rho > target) {
      const double need = std::log(target / rho) / std::log(f);
      gap = (int)std::max<double>(gmin, std::min<double>(8.0, std::floor(0.5 * need)));
    }
    last_r = r;
    last_rho = rho;
    next = r + gap;
  }
  // Sweeps predicted to take rho down to target (infinity if unknown).
  double sweeps_to(double rho, double target) const {
    if (!(f > 0.0 && f < 1.0) || rho <= target) return f > 0.0 && f < 1.0 ? 0.0 : INFINITY;
    return std::log(target / rho) / std::log(f);
  }
};

}  // namespace ibmi
