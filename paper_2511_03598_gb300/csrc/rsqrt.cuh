// 1/sqrt(y) in FP64 without the FP64 square root and division (each a chain of dependent FP64
// operations on this part, whose FP64 unit issues a warp instruction every 64 cycles).
#pragma once

namespace ttr {

static __device__ __noinline__ double rsqrt_slow(double y) { return 1.0 / sqrt(y); }

// 1/sqrt(y) for positive, finite y to full double precision: y = m 2^(2h) with m in [1, 4), a
// binary32 seed for 1/sqrt(m) (MUFU, ~22 bits; the bit patterns are moved by integer operations),
// then one third-order Newton-Householder correction r (1 + e/2 + 3e^2/8), e = 1 - m r^2: the
// truncated binomial series of (1 - e)^(-1/2), whose relative error is about (5/16) e^3 < 2^-60
// for a 22-bit seed, so the result lies within about 1 ulp of 1/sqrt(y) (ttr_selftest_rsqrt).
static __device__ __forceinline__ double rsqrt_full(double y) {
  const long long yb = __double_as_longlong(y);
  const int ef = (int)((yb >> 52) & 0x7FF);
  if (ef == 0) return rsqrt_slow(y);                        // subnormal: rare, slow path
  const int h = (ef - 1023) >> 1;                           // floor((e) / 2)
  const double m = __longlong_as_double(yb - (long long)(2 * h) * (1LL << 52));        // in [1, 4)
  const long long mb = __double_as_longlong(m);
  const int mf = (int)(((((mb >> 52) & 0x7FF) - 1023 + 127) << 23) | (int)((mb >> 29) & 0x7FFFFF));
  const float r0f = rsqrtf(__int_as_float(mf));             // in (0.5, 1]
  const int rb = __float_as_int(r0f);
  const double r0 = __longlong_as_double(((long long)(((rb >> 23) & 0xFF) - 127 + 1023) << 52) |
                                         ((long long)(rb & 0x7FFFFF) << 29));
  const double e = fma(-m * r0, r0, 1.0);
  const double r1 = fma(r0 * e, fma(e, 0.375, 0.5), r0);
  return __longlong_as_double(__double_as_longlong(r1) - (long long)h * (1LL << 52));
}

}  // namespace ttr
