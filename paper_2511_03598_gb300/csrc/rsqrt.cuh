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

// Rotation (cs, sn) of one-sided Jacobi for a column pair with squared norms A2, B2 and inner product
// G: none (cs = 1, sn = 0) when |G| <= 1e-15 sqrt(A2 B2) or both columns lie below `tiny`; else
// zeta = (B2 - A2) / (2 G), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), cs = 1 / sqrt(1 + t^2),
// sn = cs t.  The square roots and reciprocals come from rsqrt_full (1 / x = rsqrt(x)^2, sqrt(x) =
// x rsqrt(x)), a few dependent FP64 operations each instead of the FP64 square root and division;
// cs^2 + sn^2 = 1 to a few ulps, as with them.  Inputs whose products leave the normal range take
// the library square root and division.
static __device__ __forceinline__ void jacobi_rotation(double A2, double B2, double G, double tiny, double& cs,
                                                       double& sn) {
  cs = 1.0;
  sn = 0.0;
  if (G == 0.0 || (A2 <= tiny && B2 <= tiny)) return;
  const double ab = A2 * B2, g2 = 2.0 * G;
  if (!(ab > 2.3e-308) || !(ab < 1.7e308) || !(fabs(g2) > 2.3e-308)) {
    if (!(fabs(G) > 1e-15 * sqrt(A2) * sqrt(B2))) return;
    const double zeta = (B2 - A2) / g2;
    const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
    cs = 1.0 / sqrt(1.0 + t * t);
    sn = cs * t;
    return;
  }
  if (!(fabs(G) > 1e-15 * (ab * rsqrt_full(ab)))) return;
  const double rg = rsqrt_full(fabs(g2));
  const double zeta = (B2 - A2) * copysign(rg * rg, g2);     // (B2 - A2) / (2 G)
  const double az = fabs(zeta);
  double t;
  if (az < 0x1p500) {
    const double y = fma(zeta, zeta, 1.0);
    const double rd = rsqrt_full(az + y * rsqrt_full(y));
    t = copysign(rd * rd, zeta);
  } else {
    const double rz = rsqrt_full(az);
    t = copysign(0.5 * rz * rz, zeta);
  }
  cs = rsqrt_full(fma(t, t, 1.0));
  sn = cs * t;
}

}  // namespace ttr
