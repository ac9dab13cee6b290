// Float-float ("double-single") arithmetic: a value is hi + lo with two
// FP32 numbers, |lo| <= ulp(hi) / 2, about 48 bits of significand.
//
// GB300 issues one FP64 warp instruction per ~80 cycles on each SM
// sub-partition whatever the number of active lanes (measured), so a serial
// FP64 chain such as one Gauss-Newton solve is ~20x slower than the same
// chain of FP32 instructions.  The refinement and the adjoint need more than
// FP32 (points to ~1e-13 of the scene size) but not FP64's 53 bits, so they
// run on this type.  The error-free transformations are the classic ones:
// Knuth's TwoSum, the FMA form of Dekker's TwoProduct, and Newton's
// iteration for 1/sqrt.
#pragma once

#include "mpt_math.cuh"

namespace mpt {

struct ff {
  float hi, lo;
  ff() = default;
  MPT_HD constexpr ff(float h) : hi(h), lo(0.f) {}
  MPT_HD constexpr ff(float h, float l) : hi(h), lo(l) {}
  MPT_HD constexpr ff(int i) : hi((float)i), lo(0.f) {}
  // Literal constants only (folded at compile time); runtime doubles go
  // through ff_from_double.
  MPT_HD constexpr ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

MPT_HD ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff(s, (a - (s - bb)) + (b - bb));
}
MPT_HD ff quick_two_sum(float a, float b) {
  const float s = a + b;
  return ff(s, b - (s - a));
}
MPT_HD ff operator+(const ff& a, const ff& b) {
  const ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  const ff u = quick_two_sum(s.hi, s.lo + t.hi);
  return quick_two_sum(u.hi, u.lo + t.lo);
}
MPT_HD ff operator-(const ff& a) { return ff(-a.hi, -a.lo); }
MPT_HD ff operator-(const ff& a, const ff& b) { return a + (-b); }
MPT_HD ff operator*(const ff& a, const ff& b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
MPT_HD ff fma_(const ff& a, const ff& b, const ff& c) { return a * b + c; }
MPT_HD bool operator<(const ff& a, const ff& b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
MPT_HD bool operator>(const ff& a, const ff& b) { return b < a; }
MPT_HD bool operator<=(const ff& a, const ff& b) { return !(b < a); }
MPT_HD bool operator>=(const ff& a, const ff& b) { return !(a < b); }

// 1/sqrt(x): the FP32 estimate refined by two Newton steps in ff,
// y <- y + y (1 - x y^2) / 2 (each step squares the relative error).
MPT_HD ff rsq(const ff& x) {
  ff y(rsq(x.hi));
  const ff half(0.5f);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const ff r = ff(1.0f) - x * (y * y);
    y = y + y * (r * half);
  }
  return y;
}

// sin and cos through FP64 (arc edges only, never in a hot loop).
MPT_HD ff ff_from_double(double d);
MPT_HD double to_double(const ff& a);
MPT_HD void sincos_(const ff& x, ff& s, ff& c) {
  double sd, cd;
  sincos_(to_double(x), sd, cd);
  s = ff_from_double(sd);
  c = ff_from_double(cd);
}

// double -> ff on the integer units: hi = the top 24 significand bits
// (truncated), lo = the next 29 bits rounded to 24 (exact for |d| > 2^-96).
MPT_HD ff ff_from_double(double d) {
#if defined(__CUDA_ARCH__)
  const float hi = d2f_bits(d);
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((u >> 52) & 0x7FFu);
  const unsigned rem = (unsigned)(u & 0x1FFFFFFFull);  // low 29 significand bits
  float lo = 0.f;
  const int e = ex - 1075 + 127;  // biased exponent of 2^(ex - 1075), one unit of rem
  if (rem != 0u && e > 0 && e < 255) {
    lo = __uint2float_rn(rem) * __uint_as_float((unsigned)e << 23);
    if (u >> 63) lo = -lo;
  }
  return ff(hi, lo);
#else
  const float hi = (float)d;
  return ff(hi, (float)(d - (double)hi));
#endif
}
MPT_HD double to_double(const ff& a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

template <>
struct Conv<float, ff> {
  MPT_HD static float go(const ff& x) { return x.hi; }
};
template <>
struct Conv<ff, float> {
  MPT_HD static ff go(float x) { return ff(x); }
};

MPT_HD bool finite_ff(const ff& a) { return isfinite(a.hi); }

}  // namespace mpt
