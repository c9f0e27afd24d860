// The explicit update forms of the Mitigation Strategies section, for the
// ablation against the exactly monotone d-bar (2D): Algorithm 1 with the
// classical root d-tilde (form 1, "no mitigation"), the rearranged root d-hat
// (form 2), or d-hat refined by Newton's method on the root problem (form 3,
// the variant of the Achieving Exact Monotonicity section) in place of Eq.
// difference_as_root.
#pragma once

#include <cstdint>

namespace eik {
namespace forms {

constexpr unsigned long long kInf = 0x7ff0000000000000ull;
constexpr int kNewtonIters = 4;   // at most this many Newton steps (form 3)

__device__ __forceinline__ double as_d(unsigned long long u) {
  return __longlong_as_double(static_cast<long long>(u));
}
__device__ __forceinline__ unsigned long long as_u(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

// One-sided when |tH - tV| >= r or one minimum is +inf: min + r; +inf when
// both are +inf.  r = fl(h/v).  Every operation is an explicit round-to-nearest
// intrinsic, in the order the formulas are written.  Neither root is monotone
// in finite precision (Tables 1 and 2).
__device__ __forceinline__ unsigned long long explicit_update(int form, unsigned long long ab,
                                                              unsigned long long bb, double r) {
  const unsigned long long lo = ab < bb ? ab : bb;
  if (lo >= kInf) return kInf;
  if (ab >= kInf || bb >= kInf) return as_u(__dadd_rn(as_d(lo), r));
  const double tH = as_d(ab), tV = as_d(bb);
  const double d = __dsub_rn(tH, tV);
  if (fabs(d) >= r) return as_u(__dadd_rn(as_d(lo), r));
  const double c = __dmul_rn(r, r);
  double out;
  if (form == 1) {
    const double sum = __dadd_rn(tH, tV);
    const double q = __dadd_rn(__dmul_rn(tH, tH), __dmul_rn(tV, tV));
    const double disc = __dsub_rn(__dmul_rn(sum, sum), __dmul_rn(2.0, __dsub_rn(q, c)));
    out = __dmul_rn(0.5, __dadd_rn(sum, __dsqrt_rn(disc)));
  } else {
    const double disc = __dsub_rn(__dmul_rn(2.0, c), __dmul_rn(d, d));
    out = __dmul_rn(0.5, __dadd_rn(__dadd_rn(tH, tV), __dsqrt_rn(disc)));
    if (form == 3) {
      // Newton on alpha(tau) = (tau - tH)^2 + (tau - tV)^2 - c.  The paper
      // gives no stopping rule: stop when an iterate repeats, when the slope
      // 2 (mH + mV) is not positive, or after kNewtonIters steps.
#pragma unroll 1
      for (int k = 0; k < kNewtonIters; ++k) {
        const double mH = __dsub_rn(out, tH), mV = __dsub_rn(out, tV);
        const double alpha = __dsub_rn(__dadd_rn(__dmul_rn(mH, mH), __dmul_rn(mV, mV)), c);
        const double slope = __dmul_rn(2.0, __dadd_rn(mH, mV));
        if (!(slope > 0.0)) break;
        const double next = __dsub_rn(out, __ddiv_rn(alpha, slope));
        if (next == out) break;
        out = next;
      }
    }
  }
  return as_u(out);
}

}  // namespace forms
}  // namespace eik
