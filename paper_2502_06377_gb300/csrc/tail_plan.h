// Host-side plan of the Newton-Schulz tail (eq. newton) of the mixed path:
// how many digit groups each digit-sliced residual and update keeps.  Plain
// C++ (no CUDA), so that the CPU tests compile it on its own.
//
// With Q = I - X A exact, a step leaves E' = E^2 (E = I - A X).  A residual
// that keeps digit groups q <= qc carries the truncation error D of the
// groups left out, about 2^-7 of the norm g of group qc's part (each group's
// part is about 2^-7 of the one before; g is measured with the residual).
// The step X + X (Q + D)^T, made symmetric, leaves
// E' = E^2 - (D^T + A D X) / 2: for an unstructured D the second term is
// about amp = ||A||_F ||X||_F / p times D (also measured; 60 to 8000 on the
// benchmark's matrices, and this is what the measured floors follow).  The
// update's own truncation D_U enters E' as A D_U.  Each error only has to
// stay below what the steps still to come square away.
#pragma once
#include <cmath>

namespace ibmi {
namespace tail {

constexpr double kGrowth = 16.0;         // pessimistic rho_{k+1} / rho_k^2 of a step
constexpr int kCorrectionGroups = 5;     // digit groups of a first correction Q - (X - Xprev) A (21 pairs)
constexpr double kExactFraction = 1e-2;  // a correction counts as exact while its floor is below this share of tol
constexpr double kUpdateFloor = 512.0;   // update error constant (measured 75..260, doubled)

// pair products (s, u), s < sx digits of X and u < sa of the other operand,
// of digit groups s + u <= q
inline int pairs(int q, int sx, int sa) {
  int n = 0;
  for (int g = 0; g <= q; ++g)
    for (int s = 0; s <= g; ++s)
      if (s < sx && g - s < sa) ++n;
  return n;
}

// error (in rho) a step takes from a residual of groups <= q, from g measured
// at group qc and amp, with a factor 2 of margin
inline double residual_floor(int q, double g, int qc, double amp) {
  return 2.0 * g * std::ldexp(1.0, -7 * (q + 1 - qc)) * (1.0 + 0.5 * amp);
}

// error (in rho) of an update from a residual rho that keeps digit groups
// <= qu of the product X Q^T: measured at c amp rho 2^(-7 (qu + 1)) with
// c = 75..260 on five large matrices (row-scaled digits make it far larger
// than the naive estimate); kUpdateFloor doubles the largest
inline double update_floor(int qu, double rho, double amp) {
  return kUpdateFloor * amp * rho * std::ldexp(1.0, -7 * (qu + 1));
}

// steps from rho to rho <= tol / 4 if each one squares it (the optimistic
// count; at least 1, at most 12)
inline int steps(double rho, double tol) {
  int n = 0;
  for (double r = rho; r > 0.25 * tol && n < 12; r *= r) ++n;
  return n < 1 ? 1 : n;
}

// largest rho from which k steps reach tol / 4 when each multiplies rho^2 by kGrowth
inline double bound(int k, double tol) {
  double b = 0.25 * tol;
  for (int i = 0; i < k; ++i) b = std::sqrt(b / kGrowth);
  return b;
}

// error allowed in what feeds the step from rho: half of the bound for the
// steps that follow it
inline double target(double rho, double tol) { return 0.5 * bound(steps(rho, tol) - 1, tol); }

// fewest groups in [qlo, qhi) whose residual floor is within `t`, else qhi
// (a NaN or infinite estimate gives qhi)
inline int residual_groups(double t, double g, int qc, double amp, int qlo, int qhi) {
  for (int q = qlo; q < qhi; ++q)
    if (residual_floor(q, g, qc, amp) <= t) return q;
  return qhi;
}

// digit groups of a correction Q - (X - Xprev) A after an exact residual of
// rho, for a schedule without measured group norms (the batched tail): the
// fewest, at least kCorrectionGroups and at most qmax, whose truncation,
// about rho 2^(-7 (q + 1)) a c with a = ||A|| ||X|| / p up to 1e4 and c up
// to ~300 (the row-scaling constant measured for the update's product), is
// below kExactFraction of tol (tol = 1e-10: 5 groups, 21 pairs, up to
// rho = 1e-6; 6 up to 1e-4)
inline int correction_groups(double rho, double tol, int qmax) {
  int q = kCorrectionGroups;
  while (q < qmax && rho * std::ldexp(1.0, -7 * (q + 1)) * 3e6 > kExactFraction * tol) ++q;
  return q;
}

// groups of the update from a residual rho: qfull - 1 where its floor fits the
// step's target, else qfull
inline int update_groups(double rho, double amp, double tol, int qfull) {
  return update_floor(qfull - 1, rho, amp) <= target(rho, tol) ? qfull - 1 : qfull;
}

}  // namespace tail
}  // namespace ibmi
