// Counter-based Gaussian sketch entries (Sec. 3.1: Omega_k with iid N(0,1) entries).
//
// Omega_k(i, j) = rint(2^20 * sqrt(-2 ln u1) * cos(2 pi u2)) / 2^20, where (u1, u2) are two
// 53-bit uniforms from one Philox4x32-10 block (Salmon et al., SC'11) with counter
// (j, i, k, 0) and key (seed mod 2^32, seed div 2^32); u1 in (0, 1], u2 in [0, 1).
// ln and cos are evaluated here from their series (atanh series after an exact binary
// exponent split; Taylor series after an exact octant reduction) with explicitly rounded
// IEEE operations (__dadd_rn & co. are never fused), so the values are reproducible bit for
// bit by any IEEE-754 implementation that performs the same operations in the same order.
#pragma once

#include <stdint.h>

#include "series_constants.cuh"

namespace ttr {

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
}

// ln u for u in (0, 1] (u is always a normal number here: u >= 2^-53).
__device__ __forceinline__ double series_log(double u) {
  const long long bits = __double_as_longlong(u);
  double e = (double)(int)(((bits >> 52) & 0x7ff) - 1022);
  double m = __longlong_as_double((bits & 0x800fffffffffffffLL) | (1022LL << 52));   // [0.5, 1)
  if (m < TTR_SQRT_HALF) {
    m = __dmul_rn(m, 2.0);
    e = __dsub_rn(e, 1.0);
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double p = kTtrAtanh[13];
#pragma unroll
  for (int t = 12; t >= 0; --t) p = __dadd_rn(__dmul_rn(p, s2), kTtrAtanh[t]);
  const double logm = __dmul_rn(__dadd_rn(s, s), p);
  return __dadd_rn(__dmul_rn(e, TTR_LN2_HI), __dadd_rn(__dmul_rn(e, TTR_LN2_LO), logm));
}

// cos(2 pi t) for t in [0, 1).
__device__ __forceinline__ double series_cos2pi(double t) {
  t = fabs(__dsub_rn(t, rint(t)));
  const bool neg = t > 0.25;
  if (neg) t = __dsub_rn(0.5, t);
  const bool swap = t > 0.125;
  if (swap) t = __dsub_rn(0.25, t);
  const double x = __dadd_rn(__dmul_rn(t, TTR_TWO_PI_HI), __dmul_rn(t, TTR_TWO_PI_LO));
  const double x2 = __dmul_rn(x, x);
  double r;
  if (swap) {
    double p = kTtrSin[10];
#pragma unroll
    for (int k = 9; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, x2), kTtrSin[k]);
    r = __dmul_rn(x, p);
  } else {
    double p = kTtrCos[10];
#pragma unroll
    for (int k = 9; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, x2), kTtrCos[k]);
    r = p;
  }
  return neg ? -r : r;
}

__device__ __forceinline__ double gaussian_f64(uint64_t seed, uint32_t k, uint32_t i, uint32_t j) {
  uint32_t c0 = j, c1 = i, c2 = k, c3 = 0u;
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t m1 = ((uint64_t)c0 << 21) | (uint64_t)(c1 >> 11);
  const uint64_t m2 = ((uint64_t)c2 << 21) | (uint64_t)(c3 >> 11);
  const double u1 = __dmul_rn(__ull2double_rn(m1 + 1ull), 0x1p-53);
  const double u2 = __dmul_rn(__ull2double_rn(m2), 0x1p-53);
  const double rad = __dsqrt_rn(__dmul_rn(-2.0, series_log(u1)));
  return __dmul_rn(rad, series_cos2pi(u2));
}

// The sketch entry: the Gaussian rounded (half to even) to the fixed-point grid 2^-20, so that
// entry * 2^20 is an integer of magnitude below 2^24 (|g| <= sqrt(2*53*ln 2) < 8.6).  The
// integer is what the tensor-core partial-contraction epilogue multiplies by.
constexpr double kOmegaScale = 1048576.0;   // 2^20
__device__ __forceinline__ int32_t omega_int(uint64_t seed, uint32_t k, uint32_t i, uint32_t j) {
  return (int32_t)rint(__dmul_rn(gaussian_f64(seed, k, i, j), kOmegaScale));
}
__device__ __forceinline__ double omega_entry(uint64_t seed, uint32_t k, uint32_t i, uint32_t j) {
  return (double)omega_int(seed, k, i, j) * (1.0 / kOmegaScale);
}

}  // namespace ttr
