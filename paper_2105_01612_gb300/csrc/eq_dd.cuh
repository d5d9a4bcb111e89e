// eq_dd.cuh - double-float arithmetic: a value held as the unevaluated sum hi + lo of two FP32
// numbers (|lo| <= half an ulp of hi), about 48 significant bits, worked by FP32 instructions.
//
// The operations are the classical error-free transformations: Knuth's two-sum (the exact
// rounding error of a + b from six additions), the fast two-sum for |a| >= |b| (three), and the
// product's rounding error from one fused multiply-add, a * b - fl(a * b) = fma(a, b, -fl(a * b)).
// Sums add the two low parts to the high parts' rounding error and renormalise ("sloppy" sum:
// an error of a few units of 2^-48 relative to |a| + |b|); products add the cross terms
// hi_a lo_b + lo_a hi_b to the high product's error. Exponents are those of FP32, which holds the
// stresses, spectra and sums of squares met here by a wide margin.
//
// Conversions to and from FP64 are done on the bits with integer instructions (the GPU's FP64
// rate is a small fraction of its FP32 and integer rates): a double's 53-bit significand splits
// into its leading 24 bits (hi) and the remaining 29 bits rounded to 24 (lo); the way back adds
// the two significands exactly in a 64-bit integer and rounds once to 53 bits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace eqk {

template <typename T> struct V2;    // complex type of a real type (eq_fft.cuh)

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float dd_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float dd_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dd_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dd_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float dd_add(float a, float b) { volatile float s = a + b; return s; }
inline float dd_sub(float a, float b) { volatile float s = a - b; return s; }
inline float dd_mul(float a, float b) { volatile float s = a * b; return s; }
inline float dd_fma(float a, float b, float c) { return std::fma(a, b, c); }
#endif

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // from a constant or a rarely converted double (FP64 instructions; hot loads use dd_from_bits)
  __host__ __device__ constexpr explicit dd(double d)
      : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
  __host__ __device__ constexpr explicit dd(int i) : dd(static_cast<double>(i)) {}
  __host__ __device__ explicit operator double() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
  // found by argument-dependent lookup only, so that they hide no FP32 / FP64 overloads
  friend __host__ __device__ __forceinline__ dd fabs(dd a) { return a.hi < 0.f ? dd(-a.hi, -a.lo) : a; }
  friend __host__ __device__ __forceinline__ dd fmax(dd a, dd b) {
    return (a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo)) ? a : b;
  }
  friend __host__ __device__ __forceinline__ bool isfinite(dd a) {
#if defined(__CUDA_ARCH__)
    return ::isfinite(a.hi) && ::isfinite(a.lo);
#else
    return std::isfinite(a.hi) && std::isfinite(a.lo);
#endif
  }
};

__host__ __device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = dd_add(a, b);
  return dd(s, dd_sub(b, dd_sub(s, a)));
}
__host__ __device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = dd_add(a, b);
  const float v = dd_sub(s, a);
  return dd(s, dd_add(dd_sub(a, dd_sub(s, v)), dd_sub(b, v)));
}

__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, dd_add(s.lo, dd_add(a.lo, b.lo)));
}
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = dd_mul(a.hi, b.hi);
  float e = dd_fma(a.hi, b.hi, -p);
  e = dd_fma(a.hi, b.lo, e);
  e = dd_fma(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__host__ __device__ __forceinline__ dd& operator-=(dd& a, dd b) { return a = a - b; }
__host__ __device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }
// comparisons of normalised values: the high parts decide unless equal
__host__ __device__ __forceinline__ bool operator>(dd a, dd b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__host__ __device__ __forceinline__ bool operator<(dd a, dd b) { return b > a; }


// 1 / sqrt(x) for x > 0: the FP32 estimate refined by one Newton step in FP32 and one in
// double-float (each step doubles the correct bits: 2^-22 -> 2^-44 -> below the format's 2^-48)
__device__ __forceinline__ dd rsqrt_t(dd x) {
  float r = rsqrtf(x.hi);
  r = dd_mul(r, dd_fma(dd_mul(-0.5f * x.hi, r), r, 1.5f));
  const dd rr(r, 0.f);
  const dd e = dd(1.0) - x * (rr * rr);                    // 1 - x r^2, small
  return rr + rr * (dd(0.5) * e);
}

// ---- conversions on the bits -------------------------------------------------------------

// double -> double-float: hi = the leading 24 significand bits (truncated), lo = the remaining 29
// bits rounded to 24, renormalised.  Zeros, doubles below FP32's normal range and non-finite
// values map to (float(d), 0); values beyond FP32's range to infinities.
__host__ __device__ __forceinline__ dd dd_from_bits(double d) {
#if defined(__CUDA_ARCH__)
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
#else
  unsigned long long u;
  static_assert(sizeof(u) == sizeof(d), "64-bit double");
  __builtin_memcpy(&u, &d, sizeof(u));
#endif
  const unsigned sign = static_cast<unsigned>(u >> 32) & 0x80000000u;
  const int e = static_cast<int>((u >> 52) & 0x7ff) - 1023;
  auto f_of = [](unsigned bits) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(bits);
#else
    float f;
    __builtin_memcpy(&f, &bits, sizeof(f));
    return f;
#endif
  };
  if (e < -126) return dd(f_of(sign), 0.f);                         // zero / tiny: signed zero
  if (e > 127) {                                                    // beyond FP32, inf or nan
    const bool nan = e == 1024 && (u & 0xfffffffffffffull) != 0;
    return dd(f_of(sign | (nan ? 0x7fc00000u : 0x7f800000u)), 0.f);
  }
  const unsigned long long m = u & 0xfffffffffffffull;              // 52 stored bits
  const float hi = f_of(sign | (static_cast<unsigned>(e + 127) << 23) | static_cast<unsigned>(m >> 29));
  const unsigned r = static_cast<unsigned>(m & 0x1fffffffull);      // the remaining 29 bits
  // lo = r 2^(e - 52) = (r 2^-29) 2^(e - 23); r 2^-29 < 1 is exact in FP32 up to rounding of r
  float lo = dd_mul(static_cast<float>(r), 1.862645149230957e-09f);  // 2^-29
  const int sh = e - 23;                                            // in [-149, 104]
  if (sh >= -126) {
    lo = dd_mul(lo, f_of(static_cast<unsigned>(sh + 127) << 23));
  } else {
    lo = dd_mul(dd_mul(lo, f_of(static_cast<unsigned>(sh + 24 + 127) << 23)), 5.9604644775390625e-08f);  // 2^-24
  }
  if (sign) lo = -lo;
  return fast_two_sum(hi, lo);
}

// double-float -> double, rounded to nearest (ties away from zero) from the exact sum of the
// two parts' significands.  Non-finite parts give hi's value.
__host__ __device__ __forceinline__ double dd_to_bits(dd x) {
  auto bits_of = [](float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    unsigned b;
    __builtin_memcpy(&b, &f, sizeof(b));
    return b;
#endif
  };
  auto d_of = [](unsigned long long b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(static_cast<long long>(b));
#else
    double d;
    __builtin_memcpy(&d, &b, sizeof(d));
    return d;
#endif
  };
  const unsigned bh = bits_of(x.hi), bl = bits_of(x.lo);
  const int eh = static_cast<int>((bh >> 23) & 0xff), el = static_cast<int>((bl >> 23) & 0xff);
  const unsigned long long sgn = static_cast<unsigned long long>(bh & 0x80000000u) << 32;
  if (eh == 0xff || eh == 0) {
    // non-finite, zero or FP32-subnormal hi: its own value (exact in FP64) plus nothing
    if (eh == 0xff) return d_of(sgn | (0x7ffull << 52) | (static_cast<unsigned long long>(bh & 0x7fffff) << 29));
    return static_cast<double>(x.hi);                              // exact; rare (|x| < 2^-126)
  }
  // hi = Mh 2^(eh - 150), Mh in [2^23, 2^24); the sum as S 2^(eh - 150 - 40), S = Mh 2^40 +- L
  unsigned long long S = static_cast<unsigned long long>((bh & 0x7fffff) | 0x800000u) << 40;
  if ((bl & 0x7fffffffu) != 0) {                                    // lo nonzero (normal or not)
    const unsigned long long Ml = el ? ((bl & 0x7fffff) | 0x800000u) : (bl & 0x7fffff);
    const int sh = (el ? el : 1) - eh + 40;                         // lo's weight against S's unit
    unsigned long long L = sh >= 0 ? (sh < 40 ? Ml << sh : 0ull) : (sh > -24 ? Ml >> (-sh) : 0ull);
    if ((bl ^ bh) & 0x80000000u) S -= L; else S += L;
  }
  // S in (2^62, 2^64): normalise to [2^63, 2^64) keeping the exponent, then round to 53 bits
  int ex = eh - 127;                                                // unbiased exponent of 2^63 in S
  if (S >> 63 == 0) { S <<= 1; ex -= 1; }
  // S now has its leading bit at 63; keep bits 63..11 (53), round on bit 10
  unsigned long long mant = S >> 11;
  if ((S >> 10) & 1ull) mant += 1;
  if (mant >> 53) { mant >>= 1; ex += 1; }
  return d_of(sgn | (static_cast<unsigned long long>(ex + 1023) << 52) | (mant & 0xfffffffffffffull));
}

// The same conversions with FP64 instructions (the FP64 units are otherwise idle in the
// double-float passes, while the integer forms take FP32 / integer issue slots): hi = the double
// rounded to FP32, lo = the exact remainder d - hi rounded to FP32; the way back one FP64 add of
// the exact widenings.  Beyond FP32's range: infinities with lo = 0.
__host__ __device__ __forceinline__ dd dd_from_f64(double d) {
#if defined(__CUDA_ARCH__)
  const float hi = __double2float_rn(d);
  const float lo = ::isfinite(hi) ? __double2float_rn(d - static_cast<double>(hi)) : 0.f;
#else
  const float hi = static_cast<float>(d);
  const float lo = std::isfinite(hi) ? static_cast<float>(d - static_cast<double>(hi)) : 0.f;
#endif
  return dd(hi, lo);
}
__host__ __device__ __forceinline__ double dd_to_f64(dd x) {
#if defined(__CUDA_ARCH__)
  return __dadd_rn(static_cast<double>(x.hi), static_cast<double>(x.lo));
#else
  return static_cast<double>(x.hi) + static_cast<double>(x.lo);
#endif
}

// complex double-float (the register and shared-memory type of the FP64 transforms that run in
// double-float arithmetic)
struct dd2 {
  dd x, y;
};
template <> struct V2<dd> { using t = dd2; };

}  // namespace eqk
