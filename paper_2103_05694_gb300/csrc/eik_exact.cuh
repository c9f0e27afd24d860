// Exact binary64 round-to-nearest-even arithmetic on the integer pipes, for the
// operations the exactly monotone update d-bar needs (section "Achieving Exact
// Monotonicity with Finite Precision Arithmetic"): x - y for x > y >= 0, m * m
// for m >= 0, x + y for x, y >= 0, and comparisons of non-negative values as
// bit patterns.
//
// Why: on GB300 an FP64 warp instruction occupies its sub-partition's FP64
// pipe for ~80 cycles (1.6 FP64 lanes per clock per SM) with 64-cycle latency,
// while 32-bit integer instructions issue every 1-2 cycles.  The operations
// below use 15-25 integer instructions each.
//
// Each function is the IEEE-754 definition written out: align the significands
// with guard bits and a sticky bit, add or subtract (or multiply to 128 bits),
// normalise, round to nearest with ties to even.  Operands outside a safe
// exponent window (subnormals, results near overflow or underflow) are passed
// to the hardware intrinsics instead, so every result is the correctly rounded
// IEEE result for every input.  A self-test kernel (eik_selftest) compares
// these functions with the hardware FP64 unit on random and tie-heavy inputs.
#pragma once

#include <cstdint>

namespace eik {
namespace xf {

constexpr unsigned long long kFrac = (1ull << 52) - 1;
constexpr unsigned long long kHidden = 1ull << 52;
constexpr unsigned long long kInf = 0x7ff0000000000000ull;

__device__ __forceinline__ double as_d(unsigned long long u) {
  return __longlong_as_double(static_cast<long long>(u));
}
__device__ __forceinline__ unsigned long long as_u(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

// Round to nearest, ties to even, and pack.  The exact value is z + f with
// 0 <= f < 1 in units of z's last bit (f > 0 exactly when `sticky`), its
// leading 1 at bit `top` (63 or 62).  The significand is bits top..top-52;
// the bits below decide the rounding: above half rounds up, exactly half
// (rest == half and f == 0) rounds to even.  e is the biased exponent that
// goes with a significand whose leading 1 sits at bit 52.
__device__ __forceinline__ unsigned long long round_pack(unsigned long long z, int top, bool sticky,
                                                         int e) {
  const int sh = top - 52;                       // 11 or 10
  unsigned long long m = z >> sh;
  const unsigned long long rest = z & ((1ull << sh) - 1ull);
  const unsigned long long half = 1ull << (sh - 1);
  if (rest > half || (rest == half && (sticky || (m & 1ull)))) m += 1ull;
  if (m >> 53) {
    m >>= 1;
    ++e;
  }
  if (e >= 2047) return kInf;
  return (static_cast<unsigned long long>(e) << 52) | (m & kFrac);
}

// fl(x - y) for bit patterns with x > y >= 0, x finite.
__device__ __forceinline__ unsigned long long sub_pos(unsigned long long x, unsigned long long y) {
  if (y == 0ull) return x;
  const int ex = static_cast<int>(x >> 52), ey = static_cast<int>(y >> 52);
  if (ex < 64 || ey == 0 || ex > 2045) return as_u(__dsub_rn(as_d(x), as_d(y)));
  const unsigned long long X = ((x & kFrac) | kHidden) << 10;
  const unsigned long long Ys = ((y & kFrac) | kHidden) << 10;
  const int d = ex - ey;
  unsigned long long Y;
  bool sticky;
  if (d >= 63) {
    Y = 0ull;
    sticky = true;
  } else {
    Y = Ys >> d;
    sticky = (Y << d) != Ys;
  }
  // exact difference = (X - Y) - f with 0 < f < 1 when sticky: Z + (1 - f)
  const unsigned long long Z = X - Y - (sticky ? 1ull : 0ull);
  const int lz = __clzll(static_cast<long long>(Z));
  return round_pack(Z << lz, 63, sticky, ex + 1 - lz);
}

// fl(m * m) for a bit pattern m >= 0.
__device__ __forceinline__ unsigned long long sq(unsigned long long m) {
  if (m == 0ull) return 0ull;
  const int e = static_cast<int>(m >> 52);
  if (e < 600 || e > 1500) return as_u(__dmul_rn(as_d(m), as_d(m)));
  const unsigned long long P = ((m & kFrac) | kHidden) << 11;   // bit 63 set
  const unsigned long long hi = __umul64hi(P, P);
  const unsigned long long lo = P * P;
  const int top = static_cast<int>(hi >> 63);
  const unsigned long long H = top ? hi : ((hi << 1) | (lo >> 63));
  const unsigned long long L = top ? lo : (lo << 1);
  return round_pack(H, 63, L != 0ull, 2 * e - 1023 + top);
}

// fl(x + y) for bit patterns x, y >= 0.
__device__ __forceinline__ unsigned long long add_pos(unsigned long long x, unsigned long long y) {
  if (y > x) {
    const unsigned long long t = x;
    x = y;
    y = t;
  }
  if (y == 0ull) return x;
  const int ex = static_cast<int>(x >> 52), ey = static_cast<int>(y >> 52);
  if (ey == 0 || ex > 2045) return as_u(__dadd_rn(as_d(x), as_d(y)));
  const unsigned long long X = ((x & kFrac) | kHidden) << 10;
  const unsigned long long Ys = ((y & kFrac) | kHidden) << 10;
  const int d = ex - ey;
  unsigned long long Y;
  bool sticky;
  if (d >= 63) {
    Y = 0ull;
    sticky = true;
  } else {
    Y = Ys >> d;
    sticky = (Y << d) != Ys;
  }
  const unsigned long long Z = X + Y;            // exact value: Z + f, 0 <= f < 1
  if (Z >> 63) return round_pack(Z, 63, sticky, ex + 1);
  return round_pack(Z, 62, sticky, ex);
}

// m = max(fl(tau - a), +0) for tau, a >= 0 (a may be +inf).
__device__ __forceinline__ unsigned long long upwind_diff(unsigned long long tau, unsigned long long a) {
  return tau > a ? sub_pos(tau, a) : 0ull;
}

// Approximate conversions by bit manipulation (no FP64-pipe conversion
// instructions).  Used only for the starting guess and Newton steps, whose
// accuracy does not affect the result.  to_f: truncates to fp32 (flushes
// values below the fp32 normal range to 0, saturates above it to +inf).
__device__ __forceinline__ float to_f(unsigned long long u) {
  const int e = static_cast<int>((u >> 52) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __int_as_float(0x7f800000);
  return __int_as_float((e << 23) | static_cast<int>((u >> 29) & 0x7fffffu));
}
// fp32 (>= 0, finite) to the bit pattern of the equal double (exact).
__device__ __forceinline__ unsigned long long from_f(float f) {
  const unsigned b = __float_as_uint(f) & 0x7fffffffu;
  const unsigned e = b >> 23;
  if (e == 0u) return 0ull;                       // zero or fp32 subnormal: 0 is fine here
  return (static_cast<unsigned long long>(e - 127u + 1023u) << 52) |
         (static_cast<unsigned long long>(b & 0x7fffffu) << 29);
}

// fp32 (finite, either sign) to the bit pattern of the equal double (exact).
__device__ __forceinline__ unsigned long long from_f_signed(float f) {
  return from_f(f) | (static_cast<unsigned long long>(__float_as_uint(f) >> 31) << 63);
}

__device__ __forceinline__ unsigned long long umin(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}
__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) {
  return a < b ? b : a;
}

// G(tau) = fl(fl(q_x + q_y) + q_z), q_k = fl(m_k * m_k), m_k = max(fl(tau - a_k), 0),
// terms in axis order; all arguments and the result are bit patterns (>= 0).
template <int D>
__device__ __forceinline__ unsigned long long G(unsigned long long tau, const unsigned long long (&a)[D]) {
  unsigned long long g = sq(upwind_diff(tau, a[0]));
#pragma unroll
  for (int k = 1; k < D; ++k) g = add_pos(g, sq(upwind_diff(tau, a[k])));
  return g;
}

// G(tau) and, in fp32, the sum of the upwind differences (G' / 2) for Newton.
template <int D>
__device__ __forceinline__ unsigned long long G_slope(unsigned long long tau,
                                                      const unsigned long long (&a)[D], float &msum) {
  unsigned long long m = upwind_diff(tau, a[0]);
  msum = to_f(m);
  unsigned long long g = sq(m);
#pragma unroll
  for (int k = 1; k < D; ++k) {
    m = upwind_diff(tau, a[k]);
    msum += to_f(m);
    g = add_pos(g, sq(m));
  }
  return g;
}

// ulp of a positive normal double, as fp32 (0 when below the fp32 range).
__device__ __forceinline__ float ulp_f(unsigned long long tau) {
  const int e = static_cast<int>(tau >> 52) - 1075 + 127;
  return e > 0 && e < 255 ? __int_as_float(e << 23) : 0.0f;
}

// d-bar: the smallest double tau with G(tau) >= c, for axis minima a (bit
// patterns, at least one finite) and c = fl(r*r) > 0.  Starting point: the
// one-sided root a_0 + r, else the quadratic root of the two (three) smallest
// minima, in fp32; refined by Newton steps on G(tau) - c with the exact G (G
// is convex and continuously differentiable above a_0); finished by the exact
// test G(tau) >= c > G(prev(tau)) with at most a few ulp steps; bisection over
// bit patterns if the walk does not end there.  Only the finish decides the
// result, so the guess and the Newton steps only affect speed.
template <int D>
__device__ unsigned long long dbar(const unsigned long long (&a)[D], unsigned long long cb) {
  unsigned long long s0 = a[0];
  unsigned long long s1 = D > 1 ? a[1] : kInf;
  unsigned long long s2 = D > 2 ? a[2] : kInf;
  {
    const unsigned long long lo = umin(s0, s1), hi = umax(s0, s1);
    s0 = lo;
    s1 = hi;
    if (D > 2) {
      const unsigned long long l2 = umin(s1, s2), h2 = umax(s1, s2);
      s2 = h2;
      s1 = umax(s0, l2);
      s0 = umin(s0, l2);
    }
  }
  const float cf = to_f(cb);
  const float rf = sqrtf(cf);
  float w = rf;
  if (s1 != kInf) {
    const float u1 = to_f(upwind_diff(s1, s0));
    if (u1 < rf) {
      w = 0.5f * (u1 + sqrtf(fmaxf(2.0f * cf - u1 * u1, 0.0f)));
      if (D > 2 && s2 != kInf) {
        const float u2 = to_f(upwind_diff(s2, s0));
        if (w > u2) {
          const float s = u1 + u2;
          const float disc = s * s - 3.0f * (u1 * u1 + u2 * u2 - cf);
          if (disc >= 0.0f) w = (s + sqrtf(disc)) * (1.0f / 3.0f);
        }
      }
    }
  }
  unsigned long long tau = add_pos(s0, from_f(w));
  if (tau <= s0) tau = s0 + 1ull;
  unsigned long long g = kInf;
  bool have_g = false;
#pragma unroll 1
  for (int it = 0; it < 3; ++it) {
    float msum;
    g = G_slope<D>(tau, a, msum);
    have_g = true;
    if (!(msum > 0.0f) || g >= kInf) break;
    const float alpha = g >= cb ? to_f(upwind_diff(g, cb)) : -to_f(sub_pos(cb, g));
    const float step = __fdividef(alpha, 2.0f * msum);
    if (fabsf(step) <= 0.25f * ulp_f(tau)) break;   // the root is within this ulp
    const unsigned long long sb = from_f(fabsf(step));
    unsigned long long nt = step > 0.0f ? (tau > sb ? sub_pos(tau, sb) : s0 + 1ull) : add_pos(tau, sb);
    if (nt <= s0) nt = s0 + 1ull;
    if (nt == tau) break;
    tau = nt;
    have_g = false;
  }
  if (!have_g) g = G<D>(tau, a);
  unsigned long long lo, hi;
  if (g >= cb) {
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      if (tau - 1ull <= s0) return tau;                  // G(a_0) = 0 < c
      if (G<D>(tau - 1ull, a) < cb) return tau;
      --tau;
    }
    hi = tau;
    lo = s0;
  } else {
    lo = tau;
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
      ++tau;
      if (G<D>(tau, a) >= cb) return tau;
      lo = tau;
    }
    unsigned long long step = 1ull;
    hi = lo + 1ull;
#pragma unroll 1
    while (hi < kInf && G<D>(hi, a) < cb) {
      lo = hi;
      step <<= 1;
      hi = umin(lo + step, kInf);
    }
  }
#pragma unroll 1
  while (hi - lo > 1ull) {       // G(lo) < c <= G(hi)
    const unsigned long long mid = lo + (hi - lo) / 2ull;
    if (G<D>(mid, a) >= cb) hi = mid; else lo = mid;
  }
  return hi;
}

// One application of the update operator to a non-source cell whose best
// known value is `best`: true and the new value if it decreases.  A decrease
// needs a finite neighbour below best (d-bar > min a_k) and G(prev(best)) >= c
// (then d-bar <= prev(best)).
template <int D>
__device__ __forceinline__ bool relax(unsigned long long best, const unsigned long long (&a)[D],
                                      unsigned long long cb, unsigned long long &out) {
  unsigned long long amin = a[0];
#pragma unroll
  for (int k = 1; k < D; ++k) amin = umin(amin, a[k]);
  if (amin >= kInf || best <= amin) return false;
  if (best < kInf && G<D>(best - 1ull, a) < cb) return false;
  out = dbar<D>(a, cb);
  return true;
}

}  // namespace xf
}  // namespace eik

namespace eik {
// Float-float ("double-single") arithmetic on the FP32 pipe: a value is an
// unevaluated sum hi + lo of two floats, about 48 bits.  Error-free
// transformations: Knuth's TwoSum, Dekker's FastTwoSum (|a| >= |b|) and the
// FMA-based TwoProduct; square root by one Newton correction of sqrtf
// (Karp and Markstein).  Used only for starting points of d-bar, whose exact
// test decides the result.
namespace ffa {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return F2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return F2{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F2 add(F2 x, F2 y) {
  const F2 s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ F2 neg(F2 x) { return F2{-x.hi, -x.lo}; }
__device__ __forceinline__ F2 mul(F2 x, F2 y) {
  const F2 p = two_prod(x.hi, y.hi);
  return fast_two_sum(p.hi, __fadd_rn(p.lo, __fadd_rn(__fmul_rn(x.hi, y.lo), __fmul_rn(x.lo, y.hi))));
}
// sqrt(x.hi + x.lo) from the hardware's approximate reciprocal square root:
// one Newton-Raphson step in fp32 (y + (x - y^2) r / 2, r ~ 1/sqrt(x)), then one
// float-float correction with the same r / 2 in place of 1 / (2y) (the
// coupled iteration of Karp and Markstein, "High-precision division and
// square root", ACM TOMS 23(4), 1997).  About 2^-46 relative for normal x.hi;
// no IEEE special-case path.
__device__ __forceinline__ F2 sqrt_nr(F2 x) {
  if (!(x.hi > 0.0f)) return F2{0.0f, 0.0f};
  const float r = rsqrtf(x.hi);
  const float h = __fmul_rn(0.5f, r);
  float y = __fmul_rn(x.hi, r);
  y = __fmaf_rn(__fmaf_rn(-y, y, x.hi), h, y);
  const F2 p = two_prod(y, y);
  const float e = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);   // x - y^2
  return fast_two_sum(y, __fmul_rn(e, h));
}
// fp32 estimate of sqrt(x) for x > 0 (active-set decisions only).
__device__ __forceinline__ float sqrt_est(float x) { return __fmul_rn(x, rsqrtf(x)); }
// A non-negative finite double (bit pattern) as hi + lo without the FP64
// pipe: hi keeps the leading 24 bits of the significand (xf::to_f truncates),
// lo the remaining 29 bits rounded to a float.
__device__ __forceinline__ F2 split(unsigned long long u) {
  const float hi = xf::to_f(u);
  const int se = static_cast<int>((u >> 52) & 0x7ffu) - 1075 + 127;   // 2^(E - 1075) as a float
  const unsigned rem = static_cast<unsigned>(u & ((1ull << 29) - 1ull));
  float lo = 0.0f;
  if (se > 0 && se < 255) lo = __fmul_rn(__uint2float_rn(rem), __int_as_float(se << 23));
  return F2{hi, lo};
}

}  // namespace ffa

namespace hw {

// Starting point of d-bar from float-float arithmetic: u = tau - s0 is the
// root of the active-set quadratic over the sorted minima s0 <= s1 (<= s2)
// (one-sided: u = sqrt(c); two axes: u = (b1 + sqrt(2c - b1^2)) / 2, the
// rearranged root d-hat of the Mitigation Strategies section; three axes:
// u = (S + sqrt(S^2 - 3 (Q - c))) / 3), with b_k = s_k - s0 (exact FP64
// differences of close values).  About 3 (2D) / 4 (3D) FP64 instructions;
// u carries about 46 bits, so tau = s0 + u lands within an ulp of d-bar when
// u is small against tau (cells farther than a few dozen cells from a
// source), else within a few.  Only speed depends on this.
template <int D>
__device__ __forceinline__ unsigned long long ffguess(const unsigned long long (&a)[D],
                                                      unsigned long long cb) {
  // One float-float root for the active set, which fp32 estimates of the one-
  // and two-axis roots pick (the root is continuous where the active set
  // changes, so an estimate that errs near a boundary costs nothing): with k
  // active axes and B_j = b_j for j < k, else 0,
  //   u = (S + sqrt(S^2 - k (Q - c))) / k,   S = B_1 + B_2,   Q = B_1^2 + B_2^2,
  // which is sqrt(c) for k = 1, the d-hat form for k = 2 and the three-axis
  // root for k = 3.
  unsigned long long s0 = a[0], s1 = D > 1 ? a[1] : xf::kInf, s2 = D > 2 ? a[2] : xf::kInf;
  {
    const unsigned long long lo = xf::umin(s0, s1), hi = xf::umax(s0, s1);
    s0 = lo;
    s1 = hi;
    if (D > 2) {
      const unsigned long long l2 = xf::umin(s1, s2), h2 = xf::umax(s1, s2);
      s2 = h2;
      s1 = xf::umax(s0, l2);
      s0 = xf::umin(s0, l2);
    }
  }
  const ffa::F2 c = ffa::split(cb);
  // b_j = s_j - s0 (+inf when s_j is): exact FP64 differences of close values
  const ffa::F2 b1 = ffa::split(xf::as_u(__dsub_rn(xf::as_d(s1), xf::as_d(s0))));
  const ffa::F2 b2 = D > 2 ? ffa::split(xf::as_u(__dsub_rn(xf::as_d(s2), xf::as_d(s0))))
                           : ffa::F2{__int_as_float(0x7f800000), 0.0f};
  const float cf = c.hi;
  const bool two = b1.hi < ffa::sqrt_est(cf);
  bool three = false;
  if (D > 2) {
    const float u2f = __fmul_rn(0.5f, __fadd_rn(b1.hi, ffa::sqrt_est(__fmaf_rn(-b1.hi, b1.hi, __fmul_rn(2.0f, cf)))));
    const float sf = __fadd_rn(b1.hi, b2.hi);
    const float qf = __fmaf_rn(b1.hi, b1.hi, __fmul_rn(b2.hi, b2.hi));
    const float d3 = __fmaf_rn(sf, sf, __fmul_rn(-3.0f, __fsub_rn(qf, cf)));
    three = two && b2.hi < u2f && d3 > 0.0f;
  }
  const ffa::F2 B1 = two ? b1 : ffa::F2{0.0f, 0.0f};
  const ffa::F2 B2 = three ? b2 : ffa::F2{0.0f, 0.0f};
  const ffa::F2 S = ffa::add(B1, B2);
  const ffa::F2 Q = ffa::add(ffa::mul(B1, B1), ffa::mul(B2, B2));
  const float kf = three ? -3.0f : two ? -2.0f : -1.0f;
  const ffa::F2 disc = ffa::add(ffa::mul(S, S), ffa::mul(ffa::F2{kf, 0.0f}, ffa::add(Q, ffa::neg(c))));
  const ffa::F2 inv = three ? ffa::F2{__int_as_float(0x3eaaaaab), __int_as_float(static_cast<int>(0xb22aaaabu))}
                            : ffa::F2{two ? 0.5f : 1.0f, 0.0f};
  const ffa::F2 u = ffa::mul(ffa::add(S, ffa::sqrt_nr(disc)), inv);
  const double ud = __dadd_rn(xf::as_d(xf::from_f(u.hi)), xf::as_d(xf::from_f_signed(u.lo)));
  unsigned long long tau = xf::as_u(__dadd_ru(xf::as_d(s0), ud));
  if (!(tau > s0) || tau >= xf::kInf) tau = s0 + 1ull;
  return tau;
}

}  // namespace hw

namespace hw {

// The same update on the hardware FP64 unit: every operation of G an explicit
// round-to-nearest intrinsic (never contracted into an FMA); the starting
// point is ffguess (float-float, the d-hat form of the quadratic root for two
// axes); the finish is the exact ulp test.  Same interface as xf::relax (bit
// patterns in and out).
using xf::as_d;
using xf::as_u;
using xf::kInf;

template <int D>
__device__ __forceinline__ unsigned long long G(unsigned long long tau, const unsigned long long (&a)[D]) {
  double m = __dsub_rn(as_d(tau), as_d(a[0]));
  m = (__double_as_longlong(m) < 0) ? 0.0 : m;
  double g = __dmul_rn(m, m);
#pragma unroll
  for (int k = 1; k < D; ++k) {
    double mk = __dsub_rn(as_d(tau), as_d(a[k]));
    mk = (__double_as_longlong(mk) < 0) ? 0.0 : mk;
    g = __dadd_rn(g, __dmul_rn(mk, mk));
  }
  return as_u(g);
}

// G(tau) on the FP64 unit and, in fp32 (bit conversions, no FP64 pipe), the
// sum of the upwind differences.
template <int D>
__device__ __forceinline__ unsigned long long G_slope(unsigned long long tau,
                                                      const unsigned long long (&a)[D], float &msum) {
  double m = __dsub_rn(as_d(tau), as_d(a[0]));
  m = (__double_as_longlong(m) < 0) ? 0.0 : m;
  msum = xf::to_f(as_u(m));
  double g = __dmul_rn(m, m);
#pragma unroll
  for (int k = 1; k < D; ++k) {
    double mk = __dsub_rn(as_d(tau), as_d(a[k]));
    mk = (__double_as_longlong(mk) < 0) ? 0.0 : mk;
    msum += xf::to_f(as_u(mk));
    g = __dadd_rn(g, __dmul_rn(mk, mk));
  }
  return as_u(g);
}

// Is G(tau - 1) < c (ge: G(tau) >= c) or G(tau + 1) >= c (!ge: G(tau) < c)
// certain without evaluating it?  Rounding-error argument, 3D, for non-negative
// doubles a_k and c > 0:
//   each of the five roundings in G (difference, square, two sums) is within
//   2^-53 relative (underflow is far below the slack), so with
//   T(x) = sum_k ((x - a_k)^+)^2 exactly, (1 - 2^-53)^5 T <= G <= (1 + 2^-53)^5 T;
//   with d = tau - prev(tau) (ge) or next(tau) - tau (!ge) and
//   M = sum_{a_k < tau} (tau - a_k):
//     T(prev tau) <= T(tau) - 2 d M + 3 d^2,   T(next tau) >= T(tau) + 2 d M,
//   hence (rho = ((1 + 2^-53) / (1 - 2^-53))^5 <= 1 + 11 * 2^-53)
//     |G(tau) - c| + 11 * 2^-53 G(tau) < 2 d M - 3 d^2
//   implies G(prev tau) < c (ge), resp. G(next tau) >= c (!ge).
// The test runs in fp32 with margins that cover its own roundings: |G - c| in
// ulps of c rounded up, M from the truncated m_k (msum <= sum m_k), 3 d^2 below
// 2^-19 of 2 d M (checked), and a 1e-4 relative margin on both sides.  Outside
// the exponent ranges where these fp32 quantities stay normal it answers no.
__device__ __forceinline__ bool neighbour_certified(unsigned long long tau, unsigned long long g,
                                                    unsigned long long cb, float msum, bool ge) {
  const int et = static_cast<int>(tau >> 52), ec = static_cast<int>(cb >> 52);
  if (static_cast<int>(g >> 52) != ec || ec < 960 || ec > 1150 || et < 960 || et > 1150) return false;
  // |G - c| = k ulps of c (same binade), ulp(c) = 2^(ec - 1075): exact power of two
  const unsigned long long k = ge ? g - cb : cb - g;
  const float diff = __ull2float_ru(k) * __int_as_float((ec - 948) << 23);
  // d: ulp(tau), halved below tau when tau is a power of two
  const int ed = (ge && (tau & xf::kFrac) == 0ull) ? et - 949 : et - 948;
  const float d = __int_as_float(ed << 23);
  if (!(msum >= d * 1048576.0f)) return false;                   // 3 d^2 <= 2^-19 (2 d M)
  const float slack = xf::to_f(g) * 1.33226763e-15f;              // >= 11 * 2^-53 G
  const float lhs = __fadd_rn(diff, slack);
  const float rhs = __fmul_rn(2.0f * d, msum);   // exact (2 d a power of two) unless not normal
  if (!(rhs >= 1.17549435e-38f)) return false;
  return __fmul_rn(lhs, 1.0001f) < __fmul_rn(rhs, 0.9999f);
}

// The search that finishes d-bar from a point tau and the side of G(tau)
// (above: G(tau) >= c): walk a few ulps; if the root is farther (float-float
// carries ~46 bits, too few when tau - s0 is large against tau), one Newton
// step on G(tau) - c on the FP64 unit, walk again, then bracket and bisect.
template <int D>
__device__ unsigned long long dbar_search(const unsigned long long (&a)[D], unsigned long long cb,
                                          unsigned long long tau, bool above, unsigned *path) {
  unsigned long long s0 = a[0];
#pragma unroll
  for (int k = 1; k < D; ++k) s0 = xf::umin(s0, a[k]);
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    if (above) {
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        if (path) atomicAdd(&path[1], 1u);
        if (tau - 1ull <= s0) return tau;                  // G(a_0) = 0 < c
        if (G<D>(tau - 1ull, a) < cb) return tau;
        --tau;
      }
    } else {
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        if (path) atomicAdd(&path[1], 1u);
        ++tau;
        if (G<D>(tau, a) >= cb) return tau;
      }
    }
    if (pass == 1) break;
    if (path) atomicAdd(&path[0], 1u);
    float msum;
    const unsigned long long gs = G_slope<D>(tau, a, msum);
    if (!(msum > 0.0f) || gs >= kInf) break;
    const float alpha = gs >= cb ? xf::to_f(as_u(__dsub_rn(as_d(gs), as_d(cb))))
                                 : -xf::to_f(as_u(__dsub_rn(as_d(cb), as_d(gs))));
    const float step = __fdividef(alpha, 2.0f * msum);
    unsigned long long sb = xf::from_f(fabsf(step));
    if (step < 0.0f) sb |= 1ull << 63;                   // tau - step, sign set on the bits
    unsigned long long nt = as_u(__dsub_rn(as_d(tau), as_d(sb)));
    if (nt <= s0 || nt >= kInf) nt = s0 + 1ull;
    tau = nt;
    above = G<D>(tau, a) >= cb;
  }
  unsigned long long lo, hi;
  if (above) {
    hi = tau;
    lo = s0;
  } else {
    lo = tau;
    unsigned long long step = 1ull;
    hi = lo + 1ull;
#pragma unroll 1
    while (hi < kInf && G<D>(hi, a) < cb) {
      lo = hi;
      step <<= 1;
      hi = xf::umin(lo + step, kInf);
    }
  }
  if (path) atomicAdd(&path[2], 1u);
#pragma unroll 1
  while (hi - lo > 1ull) {
    const unsigned long long mid = lo + (hi - lo) / 2ull;
    if (G<D>(mid, a) >= cb) hi = mid; else lo = mid;
  }
  return hi;
}

// First stage of the two-stage d-bar: G at the starting point t, and the
// rounding-error bound on t's neighbour on the other side of c.  Returns true
// with d-bar in `out` when that settles it (t, or t + 1 when G(t) < c);
// otherwise t and the side of G(t) (ge: G(t) >= c) for dbar_second.  The bound
// counts five roundings on any term's path, as in 3D; 2D has fewer.
template <int D>
__device__ __forceinline__ bool dbar_first(const unsigned long long (&a)[D], unsigned long long cb,
                                           unsigned long long &out, unsigned long long &tau, bool &ge) {
  tau = ffguess<D>(a, cb);
  float msum;
  const unsigned long long g_here = G_slope<D>(tau, a, msum);
  ge = g_here >= cb;
  if (neighbour_certified(tau, g_here, cb, msum, ge)) {
    out = ge ? tau : tau + 1ull;
    return true;
  }
  return false;
}

// Second stage: G at the second point, t - 1 when G(t) >= c (is t the
// smallest?), t + 1 when G(t) < c (then G(t + 1) >= c makes t + 1 the
// smallest); the float-float starting point is most often one ulp low in 3D,
// which this settles without a walk.  Else the search.
template <int D>
__device__ __forceinline__ unsigned long long dbar_second(const unsigned long long (&a)[D],
                                                          unsigned long long cb, unsigned long long tau,
                                                          bool ge, unsigned *path) {
  const unsigned long long p2 = ge ? tau - 1ull : tau + 1ull;
  const bool ge2 = G<D>(p2, a) >= cb;
  if (ge && !ge2) return tau;
  if (!ge && ge2) return p2;
  return dbar_search<D>(a, cb, p2, ge2, path);
}

// d-bar with the exact G on the FP64 unit: float-float starting point
// (ffguess), then the exact test G(tau) >= c > G(prev(tau)) in two stages: G
// at the starting point and the rounding-error bound first, G at a second
// point only when the bound leaves it open; then a few ulp steps, Newton and
// bisection as the last resort.  About 4 + 8 (3D) / 3 + 5 (2D) FP64
// instructions when the bound settles it.
template <int D>
__device__ unsigned long long dbar(const unsigned long long (&a)[D], unsigned long long cb,
                                   unsigned *path = nullptr) {
  unsigned long long out, tau;
  bool ge;
  if (dbar_first<D>(a, cb, out, tau, ge)) return out;
  return dbar_second<D>(a, cb, tau, ge, path);
}

template <int D>
__device__ __forceinline__ bool relax(unsigned long long best, const unsigned long long (&a)[D],
                                      unsigned long long cb, unsigned long long &out,
                                      unsigned *path = nullptr) {
  unsigned long long amin = a[0];
#pragma unroll
  for (int k = 1; k < D; ++k) amin = xf::umin(amin, a[k]);
  if (amin >= kInf || best <= amin) return false;
  if (path) atomicAdd(&path[3], 1u);
  // d-bar directly (no separate G(prev(best)) test): a decrease iff d-bar < best
  out = dbar<D>(a, cb, path);
  return out < best;
}

}  // namespace hw
}  // namespace eik

namespace eik {
namespace hw {

// The update for one cell, evaluated by a group of L lanes (L = 4 or 8,
// aligned within the warp).  Every lane computes the same starting point;
// lane 0 of the group evaluates G(prev(best)) (is a decrease possible?), the
// other lanes G at the L-1 consecutive doubles centred on the guess, in one
// G pass.  d-bar is the first of those points with G >= c whose predecessor
// fails; if the window does not contain it, lane 0 runs the full search.
// Returns (in every lane of the group) true and the new value if the cell
// decreases.  All lanes of the warp must call this together.
template <int D, int L>
__device__ __forceinline__ bool relax_group(unsigned long long best, const unsigned long long (&a)[D],
                                            unsigned long long cb, bool valid,
                                            unsigned long long &out) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned j = lane & (L - 1u);
  const unsigned long long tg = valid ? ffguess<D>(a, cb) : 1ull;
  unsigned long long amin = a[0];
#pragma unroll
  for (int k = 1; k < D; ++k) amin = xf::umin(amin, a[k]);
  unsigned long long pt;
  if (j == 0) {
    pt = best < kInf ? best - 1ull : tg;
  } else {
    const long long off = static_cast<long long>(j) - static_cast<long long>(L / 2);
    pt = static_cast<unsigned long long>(static_cast<long long>(tg) + off);
    if (pt < amin) pt = amin;                          // G(a_min) = 0 < c
  }
  const bool ge = valid && G<D>(pt, a) >= cb;
  const unsigned bal = __ballot_sync(0xffffffffu, ge);
  const unsigned bits = (bal >> (lane & ~(L - 1u))) & ((1u << L) - 1u);
  bool dec = false;
  unsigned long long res = kInf;
  if (valid) {
    const bool possible = best >= kInf || (bits & 1u);
    if (possible) {
      const unsigned w = bits >> 1;                    // points 1..L-1
      const int first = w ? __ffs(static_cast<int>(w)) : 0;   // 1-based index within the window
      if (first >= 2) {
        res = static_cast<unsigned long long>(static_cast<long long>(tg) + (first - static_cast<int>(L / 2)));
      } else if (j == 0) {
        res = dbar<D>(a, cb);                          // window missed: full exact search
      }
      dec = true;
    }
  }
  // lane 0 of the group may have run the fallback: share its result
  const unsigned long long r0 = __shfl_sync(0xffffffffu, res, lane & ~(L - 1u));
  if (dec && res >= kInf) res = r0;
  out = res;
  return dec && res < best;
}

}  // namespace hw
}  // namespace eik
