// Device pieces of the sliced FP64 products on the BF16 tensor cores (tcgen05), shared by the
// contraction kernels (ozaki_tc.cu) and the block loop (adaptive_core.cu): the UMMA shared-memory
// descriptor, bounded mbarrier waits, the cut of FP64 values into base-128 digits exact in BF16,
// the digit layout of B operands, and the integer-only conversion of the recombined results.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace ttr {
namespace tc {

constexpr int TM = 128;               // rows per tile = UMMA M
constexpr int KC = 32;                // K per shared-memory chunk (two UMMA K-steps of 16)
constexpr int MAXS = kMaxSlices;      // slices per operand
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  const long long t0 = clock64();
  uint32_t done = 0;
  while (true) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (done) return true;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(err, 1);
      return false;
    }
  }
}

// s base-128 digits (BF16 bit patterns, sign attached) of 8 values sharing the biased exponent
// scale E: each value becomes the 7s-bit integer floor(|v| 2^(7s - E + 1022)), cut into s digits,
// most significant first.
// The slice count is fixed at compile time (constant digit offsets).  The two digits d0, d1 < 128 of
// a pair of values are packed as the BF16 bit patterns of 128 + d0 and 128 + d1 (0x4300 | d), and
// one packed BF16 subtraction of (128, 128) leaves d0 and d1 exactly; the signs are then ORed in.
template <int S>
__device__ __forceinline__ void slice8_t(const double* v, int E, uint32_t (&w)[S][4]) {
  const __nv_bfloat162 c128 = __floats2bfloat162_rn(128.f, 128.f);
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    uint64_t fx[2];
    uint32_t sg[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t bits = (uint64_t)__double_as_longlong(v[2 * h + u]);
      sg[u] = (uint32_t)(bits >> 32) & 0x80000000u;
      const int ef = (int)((bits >> 52) & 0x7FF);
      const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
      const int sh = 53 - 7 * S + (E - (ef ? ef : 1));
      fx[u] = (sh >= 64) ? 0ull : (sh >= 0 ? (mant >> sh) : (mant << (-sh)));
    }
    const uint32_t sgn = (sg[0] >> 16) | sg[1];               // sign bits of the low and high halves
#pragma unroll
    for (int p = 0; p < S; ++p) {
      const int off = 7 * (S - 1 - p);
      const uint32_t d0 = (uint32_t)(fx[0] >> off) & 127u, d1 = (uint32_t)(fx[1] >> off) & 127u;
      const uint32_t packed = __byte_perm(d0, d1, 0x5410) | 0x43004300u;
      __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&packed);
      b = __hsub2(b, c128);
      w[p][h] = *reinterpret_cast<const uint32_t*>(&b) | sgn;
    }
  }
}

// The s digit planes of 8 values (one 16-byte store per plane at bf16 index idx of each plane).
template <int S>
__device__ __forceinline__ void store_digits(const double* v, int E, uint16_t* planes, size_t plane_stride, int idx) {
  uint32_t w[S][4];
  slice8_t<S>(v, E, w);
#pragma unroll
  for (int p = 0; p < S; ++p)
    *reinterpret_cast<uint4*>(planes + (size_t)p * plane_stride + idx) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// V * 2^X as a double for |V| < 2^63 (round to nearest even; underflow to zero); integer only.
__device__ __forceinline__ double i64_to_double(long long V, int X) {
  if (V == 0) return 0.0;
  const uint64_t sign = V < 0 ? (1ull << 63) : 0ull;
  uint64_t u = V < 0 ? (uint64_t)(-V) : (uint64_t)V;
  const int lz = __clzll((long long)u);
  u <<= lz;                                                  // top bit at position 63
  uint64_t mant = u >> 11;                                   // 53 bits
  const uint64_t rest = u & 0x7FFull;
  int e = 63 - lz + X;
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++e;
    }
  }
  const int field = e + 1023;
  if (field <= 0) return __longlong_as_double((long long)sign);
  if (field >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((uint64_t)field << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// V * 2^X as a double (round to nearest even; underflow to zero).
__device__ __forceinline__ double i128_to_double(__int128 V, int X) {
  if (V == 0) return 0.0;
  const uint64_t sign = V < 0 ? (1ull << 63) : 0ull;
  unsigned __int128 u = V < 0 ? (unsigned __int128)(-V) : (unsigned __int128)V;
  const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  u <<= lz;                                                  // top bit at position 127
  uint64_t mant = (uint64_t)(u >> 75);                       // 53 bits
  const unsigned __int128 rest = u & (((unsigned __int128)1 << 75) - 1);
  const unsigned __int128 half = (unsigned __int128)1 << 74;
  int e = 127 - lz + X;                                      // value = mant/2^52 * 2^e
  if (rest > half || (rest == half && (mant & 1ull))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++e;
    }
  }
  const int field = e + 1023;
  if (field <= 0) return __longlong_as_double((long long)sign);
  if (field >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((uint64_t)field << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ int exp_field(double x) {
  return (int)(((uint64_t)__double_as_longlong(x) >> 52) & 0x7FF);
}

// B digit layout of one (column chunk, K-chunk) block, in BF16 elements: the 8x16-byte core
// matrices are ordered (k block, digit plane, row group), so that for each 8-deep k block the row
// groups of all s planes follow each other at a 128-byte stride.  One UMMA descriptor (row-group
// stride 128 B, k-block stride s (tn / 8) 128 B) then spans several planes along N, and one MMA
// accumulates several digit diagonals into adjacent TMEM columns.  Digit plane p of (k group grp,
// column j) is at b_digit_index(grp, j, s, tn) + p * tn * 8.
__host__ __device__ __forceinline__ int b_digit_index(int grp, int j, int s, int tn) {
  return ((grp * s * (tn / 8)) + (j >> 3)) * 64 + (j & 7) * 8;
}

}  // namespace tc
}  // namespace ttr
