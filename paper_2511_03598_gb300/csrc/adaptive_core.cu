// The adaptive block loop of one core (Algorithm 6 with Algorithm 5's residual sketch) as one
// persistent cooperative kernel.
//
// Given the sketch S_all = V(Y_k) W_{k+1}(:, 0:width) (computed on the tensor cores), the loop
//   Q = qr(S_all(:, 0:b_init))
//   repeat: S = S_all(:, c:c+b_e) - Q (Q^T S_all(:, c:c+b_e))              (Eqs. (3.4)-(3.5))
//           est = ||S||_F / sqrt(b_e); stop if est <= tau or c = rbar
//           Q_new = qr(S(:, 1:bb)); Q_new = qr(Q_new - Q (Q^T Q_new)); Q = [Q, Q_new]
// with b_e = max(b_inc, est_min) estimator columns and bb = min(b_inc, rbar - c) appended ones
// (b_e = b_inc in Algorithm 6 as printed).
// is a chain of small dependent FP64 steps.  On GB300 FP64 runs at ~1.2 TFLOP/s, so every step is
// spread over all SMs (each CTA owns a block of rows) and the steps are separated by a grid
// barrier instead of kernel launches; the stopping decision is taken on the device, and the
// host synchronizes once per core.
//
// Reductions over rows (Gram matrices, Q^T S, sums of squares) are FP64 atomic additions of
// per-CTA partials into one of three rotating accumulation buffers; after the barrier that
// completes reduction i, every CTA reads buffer i % 3 and CTA 0 zeroes buffer (i + 2) % 3, which
// no CTA touches again before the next barrier.  One barrier per reduction.
//
// The grid barrier is a counter/generation pair with a bounded spin: a wait that runs out sets
// the error flag and the kernel returns (the host reports TTR_ERR_TIMEOUT).
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "engine.cuh"
#include "rsqrt.cuh"
#include "sliced_mma.cuh"

namespace ttr {
namespace ac {

constexpr int NT = 256;
constexpr int BMAX = kBlockLoopMaxBlock;          // largest block handled here
constexpr long long BAR_CYCLES = 4000000000LL;   // ~2 s

enum Status { ST_DONE = 0, ST_EXTEND = 1, ST_BREAKDOWN = 2, ST_TIMEOUT = 3 };

struct Args {
  const double* Sall;   // m x width sketch, leading dimension lds
  int64_t lds;
  double* Q;            // m x qcap basis, leading dimension ldq
  int64_t ldq;
  double* S;            // m x bi work (leading dimension bi)
  double* acc;          // 3 accumulation buffers of acc_used doubles each (zero on entry)
  int acc_used;         // entries any reduction touches
  int64_t m;
  int64_t qcols;        // columns of Q kept per row in shared memory (>= rbar)
  int rpc;              // rows per CTA
  int b0, bi, rbar, width;
  int ba;               // columns appended per block (<= bi, the residual sketch's width)
  int cc0;              // columns of Q already final on entry (0: phase 1 still to do)
  double tau;
  unsigned* bar;        // [0] arrival counter, [1] generation
  int* err;
  // outputs
  double* est_out;      // estimates in order
  int* io;              // [0] status, [1] cc, [2] number of estimates
  unsigned long long* prof;   // optional: SM cycles per phase, seen by CTA 0 (null: off)
  int sshift;           // the sketch is held scaled by 2^sshift (double-float range; 0 in FP64)
  double* gwork;        // null: the CTA's rows live in shared memory; else in this global buffer,
  int64_t gstride;      //   gstride doubles per CTA (rows too wide for shared memory)
  int tc_off;           // tensor-core products: byte offset of their planes in dynamic shared memory
  int tc_cols;          //   and the TMEM columns they take (256 or 512)
};

// Phase timer of CTA 0 (launch-timeline profiling only): cycles since the previous mark are
// added to prof[phase]; prof[PH_BARRIER] collects the cycles spent waiting in grid barriers.
enum Phase { PH_STAGE = 0, PH_FIRST_QR, PH_COEFF, PH_RESIDUAL, PH_REDUCE_B, PH_QR1, PH_REORTH, PH_REDUCE_A,
             PH_FINISH, PH_BARRIER,
             // parts of the phases above (each mark closes the part before it)
             PH_B_LOCAL, PH_QR1_FACTOR, PH_RO_LOCAL, PH_RO_REDUCE, PH_RO_FIX, PH_QR2_FACTOR, PH_QR2_P, PH_COUNT };
struct Timer {
  unsigned long long* p;
  long long t;
  __device__ void mark(int phase) {
    if (p && blockIdx.x == 0 && threadIdx.x == 0) {
      const long long n = clock64();
      atomicAdd(p + phase, (unsigned long long)(n - t));
      t = n;
    }
  }
};
// the CTA's copy of Args::prof, for grid_sync
__shared__ unsigned long long* s_barrier_prof;

constexpr int ACC = 8192;                         // doubles per accumulation buffer allocated up front

// generation of the grid barrier this CTA last passed (thread 0; read once at the kernel's start,
// before any CTA can pass a barrier, then advanced by one per barrier)
__shared__ unsigned s_gen;

__device__ __forceinline__ void grid_sync_init(unsigned* bar) {
  if (threadIdx.x == 0) s_gen = *(volatile unsigned*)(bar + 1);
}

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    ok_s = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = s_gen;
    s_gen = gen + 1u;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > BAR_CYCLES) {
          atomicExch(err, 1);
          ok_s = 0;
          break;
        }
        __nanosleep(20);
      }
      if (s_barrier_prof) atomicAdd(s_barrier_prof + PH_BARRIER, (unsigned long long)(clock64() - t0));
    }
    __threadfence();
  }
  __syncthreads();
  return ok_s != 0;
}

__device__ __forceinline__ void my_rows(int64_t m, int64_t& lo, int64_t& hi) {
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  lo = min(m, (int64_t)blockIdx.x * per);
  hi = min(m, lo + per);
}

// Cross-CTA sums go through three rotating accumulation buffers in global memory: for reduction i
// every CTA adds its partial sums into buffer i%3 with FP64 atomics, passes the grid barrier and
// reads the totals (through L2).  On grids of at least RCOPY_FROM CTAs each buffer holds RCOPY
// copies, CTA c adding into copy c % RCOPY (fewer atomics per address: the barrier's fence waits
// for them to drain) and readers summing the copies; smaller grids use one copy.  Right after barrier i, the CTAs zero buffer (i+2)%3 between them: its last readers
// (reduction i-1) finished before barrier i, and its next writers (reduction i+2) start only after
// barrier i+1.  The totals are the same in every CTA, so all CTAs take the same branch.
constexpr int RCOPY = 4;
constexpr int RCOPY_FROM = 128;
__device__ __forceinline__ int red_copies() { return gridDim.x >= RCOPY_FROM ? RCOPY : 1; }
struct Red {
  double* base;     // 3 x RCOPY x used doubles, zero on entry
  int i;            // index of the next reduction
  int used;         // entries of one copy (the distance between copies)
};

// copy 0 of the current buffer (readers), and this CTA's copy (writers)
__device__ __forceinline__ double* red_buf(const Red& r) {
  return r.base + (int64_t)(r.i % 3) * red_copies() * r.used;
}
__device__ __forceinline__ double* red_out(const Red& r) {
  return red_buf(r) + (int64_t)(blockIdx.x % red_copies()) * r.used;
}

// the total at p (a location in copy 0) over the copies, `stride` doubles apart
__device__ __forceinline__ double rtot(const double* p, int stride) {
  double t = __ldcg(p);
  if (red_copies() > 1) {
#pragma unroll
    for (int q = 1; q < RCOPY; ++q) t += __ldcg(p + (int64_t)q * stride);
  }
  return t;
}

// after the barrier of the current reduction: clear the buffer two reductions ahead, advance
__device__ __forceinline__ void red_advance(Red& r) {
  double* z = r.base + (int64_t)((r.i + 2) % 3) * red_copies() * r.used;
  const int n = red_copies() * r.used;
  for (int o = blockIdx.x * NT + threadIdx.x; o < n; o += gridDim.x * NT) z[o] = 0.0;
  r.i++;
}

// ---- arithmetic of the block loop.  F64: native FP64.  DF: double-float (pairs of binary32,
// ~48 significant bits) on the FP32 pipe, which runs ~64x the FP64 rate of this part; used with the
// sliced precision form, whose contractions already carry errors of ~1e-12.  Both keep the
// cross-CTA sums in FP64 (atomic additions in L2) and the small factorizations as they are.
struct dfl {
  float h, l;
};
__device__ __forceinline__ dfl df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.h + (double)a.l; }
// c + a b
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = c.h + p;
  const float bb = s - c.h;
  const float err = (c.h - (s - bb)) + (p - bb);
  const float lo = err + (e + c.l);
  const float t = s + lo;
  return {t, lo - (t - s)};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float err = (a.h - (s - bb)) + (b.h - bb);
  const float lo = err + (a.l + b.l);
  const float t = s + lo;
  return {t, lo - (t - s)};
}

struct F64 {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T from(double x) { return x; }
  static __device__ __forceinline__ double to(T x) { return x; }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T shfl_xor(T a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
};
struct DF {
  using T = dfl;
  static __device__ __forceinline__ T zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ T from(double x) { return df_from(x); }
  static __device__ __forceinline__ double to(T x) { return df_to(x); }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return df_fma(a, b, c); }
  static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
  static __device__ __forceinline__ T neg(T a) { return {-a.h, -a.l}; }
  static __device__ __forceinline__ T shfl_xor(T a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
  }
};

// ---- tensor-core products of the block loop (sliced form).  The per-row products of a block --
// the coefficients and Gram matrices [Q, Q_new]^T [Q_new, S_next] and Q^T S, and the updates
// X <- X - Q P -- run on the BF16 tensor cores as 8-slice products (the error bound of an FP64
// product; FP64 retires two FMAs per clock per SM on this part).  Each CTA multiplies its own
// rows: K (the rows for a Gram product, the columns of Q for an update) is at most 256, so the
// low digit diagonals accumulate exactly in FP32; operands are cut into digits in shared memory
// one 16-deep K-chunk at a time, one thread issues the MMAs of the chunk into TMEM and waits on an
// mbarrier (bounded), and the epilogue recombines the diagonals in integers as the contraction
// kernels do.  C(m, n) = sum_k A(m, k) B(k, n) with m < M (tiles of 128), n < N <= 64, k < K.
constexpr int TKC = 16;                            // K per chunk: one UMMA K-step
constexpr int TSL = kMaxSlices;                    // slices per operand
constexpr int TNB = 64;                            // widest N
constexpr int TMAXK = 256;                         // K bound for exact low diagonals
constexpr int TROWS = 512;                         // largest M (row scales kept in shared memory)
constexpr int TPA = tc::TM * TKC;                  // bf16 per A digit plane
constexpr int TPB = TNB * TKC;                     // bf16 per B digit plane (widest)
constexpr size_t TC_BYTES = (size_t)TSL * (TPA + TPB) * 2;    // 48 KB of dynamic shared memory

struct Tc {
  uint16_t* ap;          // A digit planes (TSL x TPA), K-major UMMA layout
  uint16_t* bp;          // B digit planes, layout of b_digit_index
  uint32_t tmem;         // TMEM base: TSL diagonals x NB columns
  uint64_t* bar;         // MMA completion
  uint32_t* phase;       // parity of the next wait on bar (shared)
  int* rowE;             // biased exponent scale of each A row m (TROWS)
  int* colE;             // of each B column n (TNB)
  int* err;
};

// rowE[m] = max_k exponent field of A(m, k), colE[n] = that of B(k, n) (at least 1)
template <class FA, class FB>
__device__ __forceinline__ void tc_scales(const Tc& t, int M, int N, int K, FA a_at, FB b_at) {
  for (int m = threadIdx.x; m < M; m += NT) t.rowE[m] = 1;
  for (int n = threadIdx.x; n < N; n += NT) t.colE[n] = 1;
  __syncthreads();
  for (int e = threadIdx.x; e < M * K; e += NT) {
    const int m = e / K, k = e - m * K;
    atomicMax(&t.rowE[m], tc::exp_field(a_at(m, k)));
  }
  for (int e = threadIdx.x; e < K * N; e += NT) {
    const int k = e / N, n = e - k * N;
    atomicMax(&t.colE[n], tc::exp_field(b_at(k, n)));
  }
  __syncthreads();
}

// digits of the chunk k0 .. k0 + 15 of rows m0 .. m0 + 127 of A (rows below M; entries past K are 0)
// and of columns n < N of B, into the planes; the rows >= M and columns >= N of the planes are
// left as they are (they reach only outputs that are dropped)
template <class FA, class FB>
__device__ __forceinline__ void tc_slice(const Tc& t, int m0, int M, int N, int K, int k0, int NB, FA a_at, FB b_at) {
  for (int task = threadIdx.x; task < tc::TM * (TKC / 8); task += NT) {
    const int row = task >> 1, grp = task & 1, m = m0 + row;
    if (m >= M) continue;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + grp * 8 + q;
      v[q] = (k < K) ? a_at(m, k) : 0.0;
    }
    const int idx = ((grp * (tc::TM / 8)) + (row >> 3)) * 64 + (row & 7) * 8;
    tc::store_digits<TSL>(v, t.rowE[m], t.ap, TPA, idx);
  }
  for (int task = threadIdx.x; task < N * (TKC / 8); task += NT) {
    const int n = task % N, grp = task / N;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + grp * 8 + q;
      v[q] = (k < K) ? b_at(k, n) : 0.0;
    }
    tc::store_digits<TSL>(v, t.colE[n], t.bp, (size_t)NB * 8, tc::b_digit_index(grp, n, TSL, NB));
  }
}

// The MMAs of one chunk (one 16-deep K-step): for each A plane p, the B planes q = 0 .. TSL-1-p,
// adjacent along N in the b_digit_index layout, go to diagonals p + q in one MMA per group of
// floor(256 / NB) planes.  The first chunk's p = 0 MMAs write every diagonal first.
__device__ __forceinline__ void tc_issue(const Tc& t, int NB, bool first) {
  const uint64_t da0 = tc::umma_desc(tc::smem_u32(t.ap), (tc::TM / 8) * 128, 128);
  const uint64_t db0 = tc::umma_desc(tc::smem_u32(t.bp), TSL * (NB / 8) * 128, 128);
  constexpr uint32_t PA = (TPA * 2) >> 4;
  const uint32_t pb = (uint32_t)((NB / 8) * 128) >> 4;
  const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(tc::TM >> 4) << 24);
  const int G = 256 / NB;
#pragma unroll
  for (int p = 0; p < TSL; ++p) {
    const uint64_t da = da0 + (uint64_t)(p * PA);
    for (int q0 = 0; q0 < TSL - p; q0 += G) {
      const int nq = min(G, TSL - p - q0);
      const uint64_t db = db0 + (uint64_t)((uint32_t)q0 * pb);
      const uint32_t idesc = idesc0 | ((uint32_t)((nq * NB) >> 3) << 17);
      const uint32_t accum = (first && p == 0) ? 0u : 1u;
      asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                   "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(t.tmem + (uint32_t)((p + q0) * NB)),
                   "l"(da), "l"(db), "r"(idesc), "r"(accum));
    }
  }
}

// C = A B (see above), out(m, n, value) for m < M, n < N.  Returns false when a wait ran out (the
// error flag is set).  All threads of the CTA call it.
template <class FA, class FB, class FO>
__device__ bool tc_product(const Tc& t, int M, int N, int K, FA a_at, FB b_at, FO out) {
  __shared__ int ok_s;
  const int NB = N <= 32 ? 32 : 64;                 // TSL * NB TMEM columns (256 or 512)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  tc_scales(t, M, N, K, a_at, b_at);
  if (threadIdx.x == 0) ok_s = 1;
  for (int m0 = 0; m0 < M; m0 += tc::TM) {
    for (int k0 = 0; k0 < K; k0 += TKC) {
      tc_slice(t, m0, M, N, K, k0, NB, a_at, b_at);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        tc_issue(t, NB, k0 == 0);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            tc::smem_u32(t.bar)));
        if (!tc::mbar_wait(tc::smem_u32(t.bar), *t.phase, t.err)) ok_s = 0;
        *t.phase ^= 1u;
      }
      __syncthreads();
      if (!ok_s) return false;
    }
    // epilogue: warp w reads TMEM lane quarter w % 4 (rows), the two warps of a quarter take
    // alternate groups of 16 columns; V = sum_t acc_t 2^(7(TSL-1-t)) in integers (as in the
    // contraction kernels: Vh carries the shifts >= 35), then one rounding to FP64
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int quarter = warp & 3, half = warp >> 2, row = quarter * 32 + lane, m = m0 + row;
    for (int cg = half; cg < NB / 16; cg += NT / 128) {
      long long Vh[16], Vl[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) Vh[j] = Vl[j] = 0;
#pragma unroll 1
      for (int d = 0; d < TSL; ++d) {
        uint32_t r[16];
        const uint32_t taddr = t.tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(d * NB + cg * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int shift = 7 * (TSL - 1 - d);
        if (shift >= 35) {
#pragma unroll
          for (int j = 0; j < 16; ++j) Vh[j] += (long long)__float2int_rz(__uint_as_float(r[j])) << (shift - 35);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) Vl[j] += (long long)__float2int_rz(__uint_as_float(r[j])) << shift;
        }
      }
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = cg * 16 + j;
          if (n < N) {
            const __int128 V = (__int128)Vh[j] * ((__int128)1 << 35) + (__int128)Vl[j];
            out(m, n, tc::i128_to_double(V, t.rowE[m] + t.colE[n] - 2044 - 7 * TSL - 7));
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  return true;
}

// Each CTA keeps its own rows resident in shared memory (or, for rows too wide, in its own region
// of a global buffer, with the same layout):
//   Qs  [nr][ldq]  rows of Q,    Ss [nr][ldw] rows of the sketch S_all,   Rs [nr][bi] residual block.
// buf[i*b + j] += sum_{own rows} X(r, i) Y(r, j), i < a, j < b   (X, Y the CTA's own rows)
template <class A>
__device__ void gram_acc(const typename A::T* X, int ldx, const typename A::T* Y, int ldy, int a, int b, int nr,
                         double* buf) {
  using T = typename A::T;
  for (int o = threadIdx.x; o < a * b; o += NT) {
    const int i = o / b, j = o % b;
    T s0 = A::zero(), s1 = A::zero(), s2 = A::zero(), s3 = A::zero();      // four independent chains
    int r = 0;
    for (; r + 3 < nr; r += 4) {
      s0 = A::fma(X[r * ldx + i], Y[r * ldy + j], s0);
      s1 = A::fma(X[(r + 1) * ldx + i], Y[(r + 1) * ldy + j], s1);
      s2 = A::fma(X[(r + 2) * ldx + i], Y[(r + 2) * ldy + j], s2);
      s3 = A::fma(X[(r + 3) * ldx + i], Y[(r + 3) * ldy + j], s3);
    }
    for (; r < nr; ++r) s0 = A::fma(X[r * ldx + i], Y[r * ldy + j], s0);
    if (nr > 0) atomicAdd(buf + o, A::to(A::add(A::add(s0, s1), A::add(s2, s3))));
  }
}

// buf[i b + j] and buf[j b + i] += sum over the own rows of X(r, i) X(r, j) for i <= j < b: the
// upper triangle of a symmetric Gram matrix, the rows of each entry split over ks lanes (ks a power
// of two, at most 8, at least 4 rows a part) so that the few entries of a narrow block still spread
// over the warps; the ks partial sums meet by xor shuffles.  Warp-uniform trip counts.
template <class A>
__device__ void gram_sym_acc(const typename A::T* X, int ldx, int b, int nr, double* buf) {
  using T = typename A::T;
  const int nout = b * (b + 1) / 2;
  int ks = 1;
  while (ks < 8 && nout * ks * 2 <= NT && nr >= 8 * ks) ks *= 2;
  const int per = (nr + ks - 1) / ks;
  const int total = nout * ks;
  const int lane = threadIdx.x & 31;
  for (int base = threadIdx.x - lane; base < total; base += NT) {
    const int o = base + lane;
    const bool live = o < total;
    const int u = live ? o / ks : 0, p = o % ks;
    int i = 0, rem = u;                                     // u -> (i, j): triangle row i holds b - i entries
    while (rem >= b - i) {
      rem -= b - i;
      ++i;
    }
    const int j = i + rem;
    const int r0 = live ? p * per : 0, r1 = live ? min(nr, r0 + per) : 0;
    T s0 = A::zero(), s1 = A::zero();
    int r = r0;
    for (; r + 1 < r1; r += 2) {
      s0 = A::fma(X[r * ldx + i], X[r * ldx + j], s0);
      s1 = A::fma(X[(r + 1) * ldx + i], X[(r + 1) * ldx + j], s1);
    }
    if (r < r1) s0 = A::fma(X[r * ldx + i], X[r * ldx + j], s0);
    T t = A::add(s0, s1);
    for (int m = 1; m < ks; m <<= 1) t = A::add(t, A::shfl_xor(t, m));
    if (live && p == 0 && nr > 0) {
      const double v = A::to(t);
      atomicAdd(buf + i * b + j, v);
      if (i != j) atomicAdd(buf + j * b + i, v);
    }
  }
}

// buf[0] += sum of squares of the own rows of X (b columns, shared memory)
template <class A>
__device__ void sumsq_acc(const typename A::T* X, int ldx, int b, int nr, double* buf) {
  using T = typename A::T;
  __shared__ double red[NT / 32];
  T s = A::zero();
  for (int e = threadIdx.x; e < nr * b; e += NT) {
    const T v = X[(e / b) * ldx + e % b];
    s = A::fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s = A::add(s, A::shfl_xor(s, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = A::to(s);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    atomicAdd(buf, t);
  }
  __syncthreads();
}

// shared-memory copy of the first n totals of buf (written by other CTAs: read through L2)
__device__ void read_totals(const double* buf, int n, double* dst, int stride) {
  for (int o = threadIdx.x; o < n; o += NT) dst[o] = rtot(buf + o, stride);
  __syncthreads();
}
template <class A>
__device__ void read_totals_t(const double* buf, int n, typename A::T* dst, int stride) {
  for (int o = threadIdx.x; o < n; o += NT) dst[o] = A::from(rtot(buf + o, stride));
  __syncthreads();
}

// ---- small dense factorization, shaped for this part's FP64 unit: a dependent FP64 operation
// costs ~64 cycles whatever the number of active lanes, so the critical path is kept to two FP64
// operations per column and every scaling by a power of two is done on the exponent bits.

// x * 2^k, exact; integer exponent arithmetic unless x is zero, subnormal, non-finite or the
// result leaves the normal range.
// The rare paths below stay out of line: on this part an FP64 instruction costs its ~64 pipe
// cycles even when its predicate is off, so if-converted slow paths would tax every call.
__device__ __noinline__ double mul_pow2_slow(double x, int k) { return ldexp(x, k); }

__device__ __forceinline__ double mul_pow2(double x, int k) {
  const long long xb = __double_as_longlong(x);
  const int ef = (int)((xb >> 52) & 0x7FF);
  if (ef != 0 && ef != 0x7FF && ef + k > 0 && ef + k < 0x7FF) return __longlong_as_double(xb + (long long)k * (1LL << 52));
  if ((xb << 1) == 0) return x;
  return mul_pow2_slow(x, k);
}

// G (b x b, shared, symmetric positive definite) -> Ri = R^{-1} (b x b upper, shared) with
// G = R^T R.  Gauss-Jordan elimination of [G | I] (LDL^T with L^{-1} built alongside) without
// divisions: step j replaces row p > j by d'_j row_p - G_pj 2^(-e_j) row_j, where the pivot
// d_j = d'_j 2^(e_j), d'_j in [1, 2).  Row p then holds s_p = prod_{j<p} d'_j times the row of the
// ordinary elimination, so with D the pivots and L^{-1} the right block,
//   R^{-1}(i, j) = L^{-1}(j, i) / sqrt(D_j) = M(j, b + i) / sqrt(M(j, j) s_j).
// Each thread keeps its elements of [G | I] in registers; only the pivot row and column of the
// next step go through shared memory (double-buffered, one barrier per step).  Critical path per
// column: one FP64 product and one FMA.  Scratch M: b x 2b, rowbuf: 2 x 2b, colbuf: 2 x b,
// sc: b + 1.  Every CTA computes the same factor from the same data, so all take the same branch.
constexpr int FKMAX = (BMAX * 2 * BMAX + NT - 1) / NT;    // elements of [G | I] per thread
__device__ bool factor_small(const double* G, int b, double* Ri, double* M, double* rowbuf, double* colbuf,
                             double* sc) {
  __shared__ int fail;
  const int w2 = 2 * b, tot = b * w2;
  double v[FKMAX];
  int pp[FKMAX], qq[FKMAX];
#pragma unroll
  for (int k = 0; k < FKMAX; ++k) {
    const int e = threadIdx.x + k * NT;
    pp[k] = -1;
    qq[k] = 0;
    v[k] = 0.0;
    if (e < tot) {
      pp[k] = e / w2;
      qq[k] = e % w2;
      v[k] = (qq[k] < b) ? G[pp[k] * b + qq[k]] : ((qq[k] - b == pp[k]) ? 1.0 : 0.0);
      if (pp[k] == 0) rowbuf[qq[k]] = v[k];
      if (qq[k] == 0) colbuf[pp[k]] = v[k];
    }
  }
  if (threadIdx.x == 0) {
    fail = 0;
    sc[0] = 1.0;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    const double* rb = rowbuf + (j & 1) * w2;
    const double* cb = colbuf + (j & 1) * b;
    double* rn = rowbuf + ((j + 1) & 1) * w2;
    double* cn = colbuf + ((j + 1) & 1) * b;
    const long long dbits = __double_as_longlong(rb[j]);
    const int ef = (int)((dbits >> 52) & 0x7FF);
    if (dbits <= 0 || ef == 0 || ef == 0x7FF) {               // not positive and normal (integer tests)
      if (threadIdx.x == 0) fail = 1;
      break;
    }
    const int ej = ef - 1023;
    const double dp = __longlong_as_double((dbits & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    if (threadIdx.x == 0) sc[j + 1] = sc[j] * dp;
#pragma unroll
    for (int k = 0; k < FKMAX; ++k) {
      if (k * NT >= tot) break;                              // same for the whole CTA
      const int p = pp[k], q = qq[k];
      // left block: columns > j; right block (L^{-1}, lower): columns <= j and the diagonal
      const bool act = p > j && (q < b ? q > j : (q - b <= j || q - b == p));
      if (__any_sync(0xffffffffu, act)) {                    // idle warps issue no FP64 work
        const double upd = fma(dp, v[k], -cb[p < 0 ? 0 : p] * mul_pow2(rb[q], -ej));
        if (act) v[k] = upd;
      }
      if (p == j + 1) rn[q] = v[k];
      if (q == j + 1 && p > j) cn[p] = v[k];
    }
    __syncthreads();
  }
  __syncthreads();
  if (fail) return false;
#pragma unroll
  for (int k = 0; k < FKMAX; ++k)
    if (pp[k] >= 0) M[pp[k] * w2 + qq[k]] = v[k];
  __syncthreads();
  for (int e = threadIdx.x; e < b * b; e += NT) {
    const int i = e / b, j = e % b;
    double r = 0.0;
    if (i <= j) {
      const double y = M[j * w2 + j] * sc[j];
      r = (y > 0.0 && isfinite(y)) ? M[j * w2 + b + i] * rsqrt_full(y) : 0.0;
    }
    Ri[e] = r;
  }
  __syncthreads();
  return true;
}

// ---- double-float (pairs of binary32, ~48 significant bits) for the first CholeskyQR pass, whose
// factor only has to bring the condition number of the block near 1 (the second pass restores full
// FP64 orthogonality).  Its dependent operations run on the FP32 pipe (~4 cycles each instead of
// ~64 for FP64 on this part).  Error-free transformations: Dekker / Knuth two-product and two-sum.
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = p + e;
  return {s, e - (s - p)};
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) {
  const float s = a.h - b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (-b.h - bb);
  e += a.l - b.l;
  const float t = s + e;
  return {t, e - (t - s)};
}
__device__ __forceinline__ dfl df_scale(dfl a, float p2) { return {a.h * p2, a.l * p2}; }   // p2 a power of two
// factor_small with the elimination in double-float: G is scaled by 2^(-2 sigma) (exact) so that
// its largest diagonal entry is near 1 and every intermediate stays in the binary32 range.  Same
// outputs and contract as factor_small; fails (false) on a non-positive pivot.
__device__ bool factor_small_df(const double* G, int b, double* Ri, double* M, dfl* rowbuf, dfl* colbuf, double* sc) {
  __shared__ int fail;
  __shared__ int sigma_s;
  const int w2 = 2 * b, tot = b * w2;
  if (threadIdx.x < 32) {
    int e = -1022;
    for (int j = threadIdx.x; j < b; j += 32) {
      const long long gb = __double_as_longlong(G[j * b + j]);
      e = max(e, (int)((gb >> 52) & 0x7FF) - 1023);
    }
    e = __reduce_max_sync(0xffffffffu, e);
    if (threadIdx.x == 0) {
      sigma_s = e >> 1;
      fail = 0;
      reinterpret_cast<dfl*>(sc)[0] = {1.f, 0.f};
    }
  }
  __syncthreads();
  const int sigma = sigma_s;
  dfl* scd = reinterpret_cast<dfl*>(sc);                     // s_j in double-float (8 bytes, as sc)
  dfl v[FKMAX];
  int pp[FKMAX], qq[FKMAX];
#pragma unroll
  for (int k = 0; k < FKMAX; ++k) {
    pp[k] = -1;
    qq[k] = 0;
    v[k] = {0.f, 0.f};
  }
  // the conversions only for the slots that hold elements (the bound is the same for the whole CTA:
  // FP64 instructions with all lanes masked off still take FP64 pipe time on this part)
#pragma unroll
  for (int k = 0; k < FKMAX; ++k) {
    if (k * NT >= tot) break;
    const int e = threadIdx.x + k * NT;
    if (e < tot) {
      pp[k] = e / w2;
      qq[k] = e % w2;
      v[k] = (qq[k] < b) ? df_from(mul_pow2(G[pp[k] * b + qq[k]], -2 * sigma))
                         : dfl{(qq[k] - b == pp[k]) ? 1.f : 0.f, 0.f};
      if (pp[k] == 0) rowbuf[qq[k]] = v[k];
      if (qq[k] == 0) colbuf[pp[k]] = v[k];
    }
  }
  __syncthreads();
  dfl scp = {1.f, 0.f};                                       // running product of the d'_j (thread 0)
  for (int j = 0; j < b; ++j) {
    const dfl* rb = rowbuf + (j & 1) * w2;
    const dfl* cb = colbuf + (j & 1) * b;
    dfl* rn = rowbuf + ((j + 1) & 1) * w2;
    dfl* cn = colbuf + ((j + 1) & 1) * b;
    const dfl d = rb[j];
    const int db = __float_as_int(d.h);
    const int ef = (db >> 23) & 0xFF;
    if (db <= 0 || ef == 0 || ef == 0xFF) {                  // not positive and normal
      if (threadIdx.x == 0) fail = 1;
      break;
    }
    const float inv2 = __int_as_float((254 - ef) << 23);      // 2^-(ef - 127)
    const dfl dp = df_scale(d, inv2);
    if (threadIdx.x == 0) {
      scp = df_mul(scp, dp);
      scd[j + 1] = scp;                                       // no FP64 operation on the critical path
    }
#pragma unroll
    for (int k = 0; k < FKMAX; ++k) {
      if (k * NT >= tot) break;
      const int p = pp[k], q = qq[k];
      const bool act = p > j && (q < b ? q > j : (q - b <= j || q - b == p));
      if (act) v[k] = df_sub(df_mul(dp, v[k]), df_mul(cb[p], df_scale(rb[q], inv2)));
      if (p == j + 1) rn[q] = v[k];
      if (q == j + 1 && p > j) cn[p] = v[k];
    }
    __syncthreads();
  }
  __syncthreads();
  if (fail) return false;
  dfl* Md = reinterpret_cast<dfl*>(M);                       // [G | I] after the elimination, double-float
#pragma unroll
  for (int k = 0; k < FKMAX; ++k)
    if (pp[k] >= 0 && (qq[k] == pp[k] || (qq[k] >= b && qq[k] - b <= pp[k]))) Md[pp[k] * w2 + qq[k]] = v[k];
  __syncthreads();
  // R^{-1}(i, j) = M(j, b + i) / sqrt(M(j, j) s_j) in double-float (the reciprocal square root from a
  // binary32 seed and one Newton step, ~2^-45 relative), one conversion to FP64 per entry
  for (int e = threadIdx.x; e < b * b; e += NT) {
    const int i = e / b, j = e % b;
    double r = 0.0;
    if (i <= j) {
      const dfl y = df_mul(Md[j * w2 + j], scd[j]);
      const int yb = __float_as_int(y.h), ye = (yb >> 23) & 0xFF;
      if (yb > 0 && ye != 0 && ye != 0xFF) {
        const float r0 = rsqrtf(y.h);
        const dfl t = df_sub(dfl{1.f, 0.f}, df_mul(df_mul(y, dfl{r0, 0.f}), dfl{r0, 0.f}));   // 1 - y r0^2
        const dfl rs = df_add(dfl{r0, 0.f}, dfl{0.5f * r0 * t.h, 0.f});
        r = mul_pow2(df_to(df_mul(Md[j * w2 + b + i], rs)), -sigma);
      }
    }
    Ri[e] = r;
  }
  __syncthreads();
  return true;
}

// R^{-1} for G = R^T R close to the identity (the second CholeskyQR pass): with E = G - I,
// N = triu(E) - diag(E)/2 and Z = triu(N^T N) - diag(N^T N)/2, R = I + N - Z + O(|E|^3), so
// R^{-1} = I - N + Z + N^2 + O(|E|^3).  Parallel products only (no dependent elimination).
// Returns false without touching Ri when b * max|E_ij| > 1e-6 (then the O(|E|^3) term could exceed
// 1e-18); the caller uses the elimination.  Scratch Nb: b x b.
__device__ bool rinv_near_identity(const double* G, int b, double* Ri, double* Nb) {
  __shared__ int too_far;
  if (threadIdx.x == 0) too_far = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < b * b; e += NT) {
    const int i = e / b, j = e % b;
    const double ev = G[e] - (i == j ? 1.0 : 0.0);
    if (!(fabs(ev) * b <= 1e-6)) too_far = 1;
    Nb[e] = (i < j) ? ev : (i == j ? 0.5 * ev : 0.0);
  }
  __syncthreads();
  if (too_far) return false;
  for (int e = threadIdx.x; e < b * b; e += NT) {
    const int i = e / b, j = e % b;
    double r = 0.0;
    if (i <= j) {
      double n2 = 0.0, z = 0.0;
      for (int k = i; k <= j; ++k) n2 = fma(Nb[i * b + k], Nb[k * b + j], n2);      // (N N)_ij, N upper
      for (int k = 0; k <= i; ++k) z = fma(Nb[k * b + i], Nb[k * b + j], z);        // (N^T N)_ij
      if (i == j) z *= 0.5;
      r = (i == j ? 1.0 : 0.0) - Nb[e] + z + n2;
    }
    Ri[e] = r;
  }
  __syncthreads();
  return true;
}

// own rows of X (b columns, shared memory) <- X R^{-1}, one thread per (row, column):
// out(r, j) = sum_{i <= j} X(r, i) Ri(i, j) in two interleaved partial sums, staged through T and
// written back after a barrier.
template <class A>
__device__ void apply_rinv(typename A::T* X, int ldx, int b, const typename A::T* Ri, int nr, typename A::T* T) {
  using V = typename A::T;
  // a task is row r and the column pair j, b - 1 - j (j < ceil(b / 2)): column j takes j + 1 terms
  // and column b - 1 - j takes b - j, so every task makes b + 1 multiply-adds in one loop.  A warp
  // issues each FP64 instruction for all its lanes, masked or not, so equal trip counts keep the
  // lanes of the triangular product busy.
  const int hb = (b + 1) / 2;
  for (int e = threadIdx.x; e < nr * hb; e += NT) {
    const int r = e / hb, j = e % hb, j2 = b - 1 - j;
    const V* xr = X + r * ldx;
    V v = A::zero(), w = A::zero();
    for (int t = 0; t <= b; ++t) {
      const bool first = t <= j;
      const int i = first ? t : t - j - 1;
      const V res = A::fma(xr[i], Ri[i * b + (first ? j : j2)], first ? v : w);
      if (first) v = res;
      else w = res;
    }
    T[r * b + j] = v;
    if (j2 != j) T[r * b + j2] = w;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * b; e += NT) X[(e / b) * ldx + e % b] = T[e];
  __syncthreads();
}

// dst[0:n] = the FP64 values src[0:n] in the block loop's arithmetic (shared memory)
template <class A>
__device__ void to_arith(const double* src, int n, typename A::T* dst) {
  for (int o = threadIdx.x; o < n; o += NT) dst[o] = A::from(src[o]);
  __syncthreads();
}

// own rows: X(:, 0:b) -= Q(:, 0:c) P, P (c x b, leading dimension ldp) in shared memory
template <class A>
__device__ void sub_qp(typename A::T* X, int ldx, const typename A::T* Q, int ldq, int c, const typename A::T* P,
                       int ldp, int b, int nr) {
  using V = typename A::T;
  if (c <= 0) return;
  for (int e = threadIdx.x; e < nr * b; e += NT) {
    const int r = e / b, j = e % b;
    const V* qr = Q + r * ldq;
    // two chains, the first starting from X(r, j): one FP64 addition per element to join them
    // (each FP64 warp instruction holds this part's FP64 unit for 64 cycles, so the joins count)
    V s0 = X[r * ldx + j], s1 = A::zero();
    int i = 0;
    for (; i + 1 < c; i += 2) {
      s0 = A::fma(A::neg(qr[i]), P[i * ldp + j], s0);
      s1 = A::fma(A::neg(qr[i + 1]), P[(i + 1) * ldp + j], s1);
    }
    if (i < c) s0 = A::fma(A::neg(qr[i]), P[i * ldp + j], s0);
    X[r * ldx + j] = A::add(s0, s1);
  }
  __syncthreads();
}

// out (b x n, ld n, shared) = Ri^T (b x b lower) C (b x n, ld n, global totals): the coefficients
// of the new basis block (X R^{-1})^T Y from X^T Y
template <class A>
__device__ void mul_rinv_t_left(const double* C, int b, int n, const double* Ri, typename A::T* out, int stride) {
  for (int e = threadIdx.x; e < b * n; e += NT) {
    const int i = e / n, j = e % n;
    double v = 0.0;
    for (int k = 0; k <= i; ++k) v = fma(Ri[k * b + i], rtot(C + k * n + j, stride), v);
    out[e] = A::from(v);
  }
  __syncthreads();
}

template <class A, bool TCP>
__global__ void __launch_bounds__(NT, 1) adaptive_core_kernel(Args a) {
  using T = typename A::T;
  extern __shared__ __align__(128) double sm[];
  __shared__ T RiT[BMAX * BMAX];
  __shared__ double G[BMAX * BMAX];
  __shared__ double Ri[BMAX * BMAX];
  __shared__ double M[BMAX * 2 * BMAX];
  __shared__ double rowbuf[2 * 2 * BMAX];
  __shared__ double colbuf[2 * BMAX];
  __shared__ dfl rowbuf_df[2 * 2 * BMAX];
  __shared__ dfl colbuf_df[2 * BMAX];
  __shared__ double sc[BMAX + 1];
  __shared__ double est_s;
  __shared__ double wred[NT / 32];
  __shared__ double c2_s;
  // first CholeskyQR pass: double-float elimination; second pass: near-identity series, else the
  // FP64 elimination
  auto factor1 = [&](int bb) { return factor_small_df(G, bb, Ri, M, rowbuf_df, colbuf_df, sc); };
  auto factor2 = [&](int bb) {
    return rinv_near_identity(G, bb, Ri, M) || factor_small(G, bb, Ri, M, rowbuf, colbuf, sc);
  };
  int64_t lo, hi;
  my_rows(a.m, lo, hi);
  const int nr = (int)(hi - lo);
  const int ldq = (int)a.qcols, ldw = a.width, bi = a.bi;
  static_assert(sizeof(T) == sizeof(double), "the shared-memory layout assumes 8-byte elements");
  double* base = a.gwork ? a.gwork + (int64_t)blockIdx.x * a.gstride : sm;
  T* Qs = reinterpret_cast<T*>(base);                // [rpc][ldq]   own rows of Q
  T* Ss = Qs + (size_t)a.rpc * ldq;                  // [rpc][ldw]   own rows of the sketch S_all (x 2^sshift)
  T* Rs = Ss + (size_t)a.rpc * ldw;                  // [rpc][bi]    residual block (x 2^sshift)
  T* Tb = Rs + (size_t)a.rpc * bi;                   // [rpc][BMAX]  staging for X R^{-1}
  T* Ps = Tb + (size_t)a.rpc * BMAX;                 // [qcols][max(b0, bi)] projection coefficients
  T* Cs = Ps + (size_t)a.qcols * max(a.b0, bi);      // [qcols][max(b0, bi)] Q^T Q_new of the current block
  const int ldp = bi;
  bool timeout = false;
  int cc = a.cc0;
  int nest = 0;
  Red rd{a.acc, 0, a.acc_used};
  Timer tmr{a.prof, clock64()};
  if (threadIdx.x == 0) s_barrier_prof = (blockIdx.x == 0) ? a.prof : nullptr;
  grid_sync_init(a.bar);
  // tensor-core products: TMEM, the completion barrier and the scales
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t tc_bar;
  __shared__ uint32_t tc_phase;
  __shared__ int tc_rowE[TROWS];
  __shared__ int tc_colE[TNB];
  Tc tcx{};
  if constexpr (TCP) {
    unsigned char* tb = reinterpret_cast<unsigned char*>(sm) + a.tc_off;
    tcx.ap = reinterpret_cast<uint16_t*>(tb);
    tcx.bp = reinterpret_cast<uint16_t*>(tb + (size_t)TSL * TPA * 2);
    tcx.bar = &tc_bar;
    tcx.phase = &tc_phase;
    tcx.rowE = tc_rowE;
    tcx.colE = tc_colE;
    tcx.err = a.err;
    if ((threadIdx.x >> 5) == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                   "r"(a.tc_cols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&tc_bar)));
      asm volatile("fence.mbarrier_init.release.cluster;");
      tc_phase = 0u;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    tcx.tmem = tmem_slot;
  }
  // stage the own rows: sketch columns, and the part of Q that is already final
  for (int e = threadIdx.x; e < nr * ldw; e += NT)
    Ss[e] = A::from(mul_pow2(a.Sall[(lo + e / ldw) * a.lds + e % ldw], a.sshift));
  for (int e = threadIdx.x; e < nr * cc; e += NT)
    Qs[(e / cc) * ldq + e % cc] = A::from(a.Q[(lo + e / cc) * a.ldq + e % cc]);
  __syncthreads();
  tmr.mark(PH_STAGE);
  auto finish = [&](int status) {
    // write back Q(:, 0:cc) (plus the residual block, which the host needs after a breakdown)
    for (int e = threadIdx.x; e < nr * cc; e += NT)
      a.Q[(lo + e / cc) * a.ldq + e % cc] = A::to(Qs[(e / cc) * ldq + e % cc]);
    for (int e = threadIdx.x; e < nr * bi; e += NT) a.S[(lo + e / bi) * bi + e % bi] = mul_pow2(A::to(Rs[e]), -a.sshift);
    tmr.mark(PH_FINISH);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.io[0] = timeout ? ST_TIMEOUT : status;
      a.io[1] = cc;
      a.io[2] = nest;
    }
    if constexpr (TCP) {
      // every MMA of this CTA has completed (each product waits for its own): release TMEM
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tcx.tmem), "r"(a.tc_cols));
    }
  };
  // one cross-CTA reduction: everything accumulated into red_buf(rd) before the call is summed
  auto reduce = [&]() -> double* {
    double* buf = red_buf(rd);
    if (!grid_sync(a.bar, a.err)) {
      timeout = true;
      return nullptr;
    }
    red_advance(rd);
    return buf;
  };
  // In the loop, P = Q^T S_all(:, cc:cc+bi) for the next block is carried over from the previous
  // iteration's second reduction whenever that block lies within the sketch (have_p).
  bool have_p = false;
  if (cc == 0) {
    // first block: Q(:, 0:b0) = qr(S_all(:, 0:b0)) by CholeskyQR2; the second pass's reduction also
    // sums Q1^T S_all(:, b0:b0+bi), the projection coefficients of the first residual block
    const int b0 = a.b0;
    for (int e = threadIdx.x; e < nr * b0; e += NT) Qs[(e / b0) * ldq + e % b0] = Ss[(e / b0) * ldw + e % b0];
    __syncthreads();
    gram_sym_acc<A>(Qs, ldq, b0, nr, red_out(rd));
    double* buf = reduce();
    if (!buf) return finish(ST_TIMEOUT);
    read_totals(buf, b0 * b0, G, rd.used);
    if (!factor1(b0)) return finish(ST_BREAKDOWN);
    to_arith<A>(Ri, b0 * b0, RiT);
    apply_rinv<A>(Qs, ldq, b0, RiT, nr, Tb);
    const bool want = b0 < a.rbar && b0 + bi <= a.width;
    gram_sym_acc<A>(Qs, ldq, b0, nr, red_out(rd));
    if (want) gram_acc<A>(Qs, ldq, Ss + b0, ldw, b0, bi, nr, red_out(rd) + b0 * b0);
    buf = reduce();
    if (!buf) return finish(ST_TIMEOUT);
    read_totals(buf, b0 * b0, G, rd.used);
    if (!factor2(b0)) return finish(ST_BREAKDOWN);
    to_arith<A>(Ri, b0 * b0, RiT);
    apply_rinv<A>(Qs, ldq, b0, RiT, nr, Tb);
    if (want) mul_rinv_t_left<A>(buf + b0 * b0, b0, bi, Ri, Ps, rd.used);      // (Q1 R2^{-1})^T S = R2^{-T} Q1^T S
    have_p = want;
    cc = b0;
    tmr.mark(PH_FIRST_QR);
  }
  while (cc < a.rbar) {
    if (cc + bi > a.width) return finish(ST_EXTEND);
    if (!have_p) {
      if (TCP && nr > 0) {
        double* eb = red_out(rd);
        const T* sc_ = Ss + cc;
        if (!tc_product(
                tcx, cc, bi, nr, [&](int m, int k) { return A::to(Qs[k * ldq + m]); },
                [&](int k, int n) { return A::to(sc_[k * ldw + n]); },
                [&](int m, int n, double v) { atomicAdd(eb + m * bi + n, v); })) {
          timeout = true;
          return finish(ST_TIMEOUT);
        }
      } else {
        gram_acc<A>(Qs, ldq, Ss + cc, ldw, cc, bi, nr, red_out(rd));
      }
      double* buf = reduce();
      if (!buf) return finish(ST_TIMEOUT);
      read_totals_t<A>(buf, cc * bi, Ps, rd.used);
    }
    tmr.mark(PH_COEFF);
    // residual sketch of the next block (Eqs. (3.4)-(3.5)): S = S_all(:, cc:cc+bi) - Q P
    for (int e = threadIdx.x; e < nr * bi; e += NT) Rs[e] = Ss[(e / bi) * ldw + cc + e % bi];
    __syncthreads();
    if (TCP && cc > 0 && cc <= TMAXK && nr > 0) {
      if (!tc_product(
              tcx, nr, bi, cc, [&](int m, int k) { return A::to(Qs[m * ldq + k]); },
              [&](int k, int n) { return A::to(Ps[k * ldp + n]); },
              [&](int m, int n, double v) { Rs[m * bi + n] = A::from(A::to(Rs[m * bi + n]) - v); })) {
        timeout = true;
        return finish(ST_TIMEOUT);
      }
    } else {
      sub_qp<A>(Rs, bi, Qs, ldq, cc, Ps, ldp, bi, nr);
    }
    tmr.mark(PH_RESIDUAL);
    // reduction B: ||S||_F^2 and the Gram matrix of the candidate block S(:, 0:bb)
    const int bb = min(a.ba, a.rbar - cc);
    {
      double* eb = red_out(rd);
      sumsq_acc<A>(Rs, bi, bi, nr, eb);
      gram_sym_acc<A>(Rs, bi, bb, nr, eb + 1);
    }
    tmr.mark(PH_B_LOCAL);
    double* bufB = reduce();
    if (!bufB) return finish(ST_TIMEOUT);
    if (threadIdx.x == 0) est_s = rtot(bufB, rd.used);
    __syncthreads();
    const double ss = est_s;                               // ||S||_F^2
    if (blockIdx.x == 0 && threadIdx.x == 0) a.est_out[nest] = mul_pow2(ss, -2 * a.sshift);   // host: sqrt(ss / b_e)
    ++nest;
    tmr.mark(PH_REDUCE_B);
    // est = sqrt(ss / b_e) > tau  <=>  ss > tau^2 b_e  (the square root is left to the host)
    const double tau_s = mul_pow2(a.tau, a.sshift);
    if (!(ss > tau_s * tau_s * (double)bi)) return finish(ST_DONE);
    // new directions (Algorithm 6): Q_new = qr(S(:, 0:bb)); Q_new -= Q (Q^T Q_new); Q_new = qr(Q_new).
    // Each qr is one CholeskyQR pass (CholeskyQR2 with the block Gram-Schmidt step in between:
    // the first pass leaves Q_new orthonormal to ~u cond(S)^2, the second to ~u).
    read_totals(bufB + 1, bb * bb, G, rd.used);
    if (!factor1(bb)) return finish(ST_BREAKDOWN);
    tmr.mark(PH_QR1_FACTOR);
    T* Qn = Qs + cc;
    for (int e = threadIdx.x; e < nr * bb; e += NT) Qn[(e / bb) * ldq + e % bb] = Rs[(e / bb) * bi + e % bb];
    __syncthreads();
    to_arith<A>(Ri, bb * bb, RiT);
    apply_rinv<A>(Qn, ldq, bb, RiT, nr, Tb);
    tmr.mark(PH_QR1);
    // One reduction for both the block Gram-Schmidt step and the second CholeskyQR pass, on the
    // Q_new just formed (so its rounding errors are seen): [Q, Q_new]^T Q_new gives C = Q^T Q_new and
    // G = Q_new^T Q_new, and when the next block lies within the sketch, [Q, Q_new]^T S_next.  After
    // Q_new <- Q_new - Q C, its Gram matrix is G - C^T C and its coefficients against S_next are
    // Q_new^T S_next - C^T Q^T S_next (Q^T Q = I to rounding; G is near I and C^T C tiny, so the
    // subtraction loses nothing).
    const int nxt = cc + bb;
    const bool want = nxt < a.rbar && nxt + bi <= a.width;
    {
      double* eb = red_out(rd);
      if (TCP && nr > 0) {
        const T* sn = Ss + nxt;
        const int nb = bb + (want ? bi : 0);
        if (!tc_product(
                tcx, nxt, nb, nr, [&](int m, int k) { return A::to(Qs[k * ldq + m]); },
                [&](int k, int n) { return n < bb ? A::to(Qn[k * ldq + n]) : A::to(sn[k * ldw + (n - bb)]); },
                [&](int m, int n, double v) {
                  if (n < bb) atomicAdd(eb + m * bb + n, v);
                  else atomicAdd(eb + nxt * bb + m * bi + (n - bb), v);
                })) {
          timeout = true;
          return finish(ST_TIMEOUT);
        }
      } else {
        gram_acc<A>(Qs, ldq, Qn, ldq, nxt, bb, nr, eb);                                  // (cc + bb) x bb
        if (want) gram_acc<A>(Qs, ldq, Ss + nxt, ldw, nxt, bi, nr, eb + nxt * bb);      // (cc + bb) x bi
      }
    }
    tmr.mark(PH_RO_LOCAL);
    double* bufA = reduce();
    if (!bufA) return finish(ST_TIMEOUT);
    // C = Q^T Q_new (cc x bb) and ||C||_F^2: when that is at most 2^-54, every entry of C^T C lies
    // below half an ulp of the unit diagonal of G (Q_new is orthonormal to ~u after the first pass)
    // and the correction G - C^T C is G to FP64 accuracy
    {
      double part = 0.0;
      for (int o = threadIdx.x; o < cc * bb; o += NT) {
        const double v = rtot(bufA + o, rd.used);
        Cs[o] = A::from(v);
        part = fma(v, v, part);
      }
      for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += wred[w];
        c2_s = t;
      }
      __syncthreads();
    }
    tmr.mark(PH_RO_REDUCE);
    const bool c_tiny = !(c2_s > 0x1p-54);
    // G - C^T C, two threads per output (each the sum over every other row of C)
    for (int base = 0; base < 2 * bb * bb; base += NT) {
      const int o2 = base + threadIdx.x, o = o2 >> 1, h = o2 & 1;
      const bool live = o < bb * bb;
      T t = A::zero();
      if (live && !c_tiny) {
        const int i = o / bb, j = o % bb;
        for (int k = h; k < cc; k += 2) t = A::fma(Cs[k * bb + i], Cs[k * bb + j], t);
      }
      t = A::add(t, A::shfl_xor(t, 1));
      if (live && h == 0) G[o] = rtot(bufA + (cc + o / bb) * bb + o % bb, rd.used) - A::to(t);
    }
    __syncthreads();
    tmr.mark(PH_RO_FIX);
    if (TCP && cc > 0 && cc <= TMAXK && nr > 0) {
      if (!tc_product(
              tcx, nr, bb, cc, [&](int m, int k) { return A::to(Qs[m * ldq + k]); },
              [&](int k, int n) { return A::to(Cs[k * bb + n]); },
              [&](int m, int n, double v) { Qn[m * ldq + n] = A::from(A::to(Qn[m * ldq + n]) - v); })) {
        timeout = true;
        return finish(ST_TIMEOUT);
      }
    } else if (cc > 0) {
      sub_qp<A>(Qn, ldq, Qs, ldq, cc, Cs, bb, bb, nr);
    }
    tmr.mark(PH_REORTH);
    if (!factor2(bb)) return finish(ST_BREAKDOWN);
    tmr.mark(PH_QR2_FACTOR);
    if (want) {
      // P = [Q^T S_next; R2^{-T} (Q_new^T S_next - C^T Q^T S_next)]; the middle term goes through M
      const double* pb = bufA + nxt * bb;
      read_totals_t<A>(pb, cc * bi, Ps, rd.used);
      for (int base = 0; base < 2 * bb * bi; base += NT) {
        const int o2 = base + threadIdx.x, o = o2 >> 1, h = o2 & 1;
        const bool live = o < bb * bi;
        T t = A::zero();
        if (live) {
          const int i = o / bi, j = o % bi;
          for (int k = h; k < cc; k += 2) t = A::fma(Cs[k * bb + i], Ps[k * bi + j], t);
        }
        t = A::add(t, A::shfl_xor(t, 1));
        if (live && h == 0) M[o] = rtot(pb + (cc + o / bi) * bi + o % bi, rd.used) - A::to(t);
      }
      __syncthreads();
      for (int o = threadIdx.x; o < bb * bi; o += NT) {
        const int i = o / bi, j = o % bi;
        double v = 0.0;
        for (int k = 0; k <= i; ++k) v = fma(Ri[k * bb + i], M[k * bi + j], v);
        Ps[cc * bi + o] = A::from(v);
      }
      __syncthreads();
    }
    tmr.mark(PH_QR2_P);
    to_arith<A>(Ri, bb * bb, RiT);
    apply_rinv<A>(Qn, ldq, bb, RiT, nr, Tb);
    have_p = want;
    cc = nxt;
    tmr.mark(PH_REDUCE_A);
  }
  finish(ST_DONE);
}

__global__ void rsqrt_selftest_kernel(const double* x, double* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rsqrt_full(x[i]);
}

__global__ void jacobi_rotation_selftest_kernel(const double* abg, double tiny, double* cs_sn, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double cs, sn;
    jacobi_rotation(abg[3 * i], abg[3 * i + 1], abg[3 * i + 2], tiny, cs, sn);
    cs_sn[2 * i] = cs;
    cs_sn[2 * i + 1] = sn;
  }
}

}  // namespace ac

int rsqrt_selftest(Ctx& c, const double* x, double* out, int64_t n) {
  if (n <= 0) return TTR_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  ac::rsqrt_selftest_kernel<<<blocks, 256, 0, c.stream>>>(x, out, n);
  return c.check_launch("rsqrt_selftest");
}

int jacobi_rotation_selftest(Ctx& c, const double* abg, double tiny, double* cs_sn, int64_t n) {
  if (n <= 0) return TTR_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  ac::jacobi_rotation_selftest_kernel<<<blocks, 256, 0, c.stream>>>(abg, tiny, cs_sn, n);
  return c.check_launch("jacobi_rotation_selftest");
}

// Whether the block loop's rows for these sizes fit in shared memory (else they would live in
// global memory); the same sizing as adaptive_core.
bool adaptive_core_rows_fit(int64_t m, int b0, int bi, int rbar, int width, int max_sms) {
  int dev = 0, nsm = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  const int sms = (max_sms > 0 && max_sms < nsm) ? max_sms : nsm;
  const int nblocks = (int)std::min<int64_t>(sms, m);
  if (nblocks < 1) return false;
  const int rpc = (int)((m + nblocks - 1) / nblocks);
  const int64_t qcols = std::min(rbar, width);
  const size_t dyn = sizeof(double) * ((size_t)rpc * (size_t)(qcols + width + bi + ac::BMAX) +
                                        2 * (size_t)qcols * (size_t)std::max(b0, bi));
  return dyn + 48 * 1024 <= (size_t)optin;
}

// Host side: runs the adaptive loop of one core on the device.  Returns TTR_OK with *status set
// (ST_DONE, ST_EXTEND: more sketch columns are needed, ST_BREAKDOWN: a CholeskyQR pivot failed
// at column *cc), or TTR_ERR_UNSUPPORTED when this path does not apply.
int adaptive_core(Ctx& c, const double* Sall, int64_t lds, double* Q, int64_t ldq, double* S, int64_t m, int b0,
                  int bi, int ba, int rbar, int width, int cc0, double tau, double* est_host, int est_cap, int* status,
                  int* cc, int* nest, bool double_float, double scale, int max_sms, bool host_if_global,
                  bool tensor_products) {
  if (b0 > ac::BMAX || bi > ac::BMAX || m <= 0) return TTR_ERR_UNSUPPORTED;
  if (ba < 1 || ba > bi) return set_error("adaptive loop: appended block wider than the residual sketch"), TTR_ERR_ARG;
  int dev = 0;
  TTR_CUDA(cudaGetDevice(&dev));
  // device properties and the kernel's shared-memory limit, looked up once per device
  constexpr int MAXDEV = 64;
  struct DevInfo {
    int nsm, coop, smem_optin, raised[3], static_bytes[3];
  };
  static DevInfo info[MAXDEV] = {};
  DevInfo local{};
  DevInfo& di = (dev >= 0 && dev < MAXDEV) ? info[dev] : local;
  if (di.nsm == 0) {
    TTR_CUDA(cudaDeviceGetAttribute(&di.coop, cudaDevAttrCooperativeLaunch, dev));
    TTR_CUDA(cudaDeviceGetAttribute(&di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    TTR_CUDA(cudaDeviceGetAttribute(&di.nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const int nsm = di.nsm, smem_optin = di.smem_optin;
  if (!di.coop) return TTR_ERR_UNSUPPORTED;
  // no more CTAs than rows; each CTA keeps its rows of Q, of the sketch and of the residual block.
  // One CTA per SM (a sweep of 38..152 CTAs on the 20-core workload: 152 is fastest), or the
  // caller's share of the SMs.
  const int sms = (max_sms > 0 && max_sms < nsm) ? max_sms : nsm;
  const int nblocks = (int)std::min<int64_t>(sms, m);
  const int rpc = (int)((m + nblocks - 1) / nblocks);
  const int64_t qcols = std::min(rbar, width);     // columns of Q never exceed the sketch width
  const size_t dyn = sizeof(double) * ((size_t)rpc * (size_t)(qcols + width + bi + ac::BMAX) +
                                        2 * (size_t)qcols * (size_t)std::max(b0, bi));
  // the kernels' static shared memory (G, R^{-1}, [G | I], pivot buffers, the product scales)
  const void* kerns[3] = {(const void*)ac::adaptive_core_kernel<ac::F64, false>,
                          (const void*)ac::adaptive_core_kernel<ac::DF, false>,
                          (const void*)ac::adaptive_core_kernel<ac::F64, true>};
  if (di.static_bytes[0] == 0) {
    for (int q = 0; q < 3; ++q) {
      cudaFuncAttributes fa{};
      TTR_CUDA(cudaFuncGetAttributes(&fa, kerns[q]));
      di.static_bytes[q] = (int)fa.sharedSizeBytes + 1024;
    }
  }
  // rows that do not fit in shared memory live in a global buffer, one region per CTA (same layout)
  const bool global_rows = dyn + (size_t)di.static_bytes[double_float ? 1 : 0] > (size_t)smem_optin;
  if (global_rows && host_if_global) return TTR_ERR_UNSUPPORTED;
  // tensor-core products (sliced form, FP64 arithmetic): K of every product within the exact bound,
  // the widths within the TMEM columns, and their digit planes beside the rows in shared memory
  const size_t tc_off = global_rows ? 0 : (dyn + 127) / 128 * 128;
  const bool use_tc = tensor_products && !double_float && rpc <= ac::TMAXK && rbar <= ac::TROWS &&
                      ba + bi <= ac::TNB &&
                      tc_off + ac::TC_BYTES + (size_t)di.static_bytes[2] <= (size_t)smem_optin;
  const int ki = use_tc ? 2 : (double_float ? 1 : 0);
  const void* kern = kerns[ki];
  size_t dyn_launch = use_tc ? tc_off + ac::TC_BYTES : (global_rows ? 0 : dyn);
  // a CTA that takes all 512 TMEM columns must have its SM to itself (a second one would wait for
  // them while the first waits for it at a grid barrier): ask for more than half the shared memory
  if (use_tc && ba + bi > 32) dyn_launch = std::max(dyn_launch, (size_t)smem_optin / 2 + 1024);
  double* gwork = nullptr;
  const int64_t gstride = (int64_t)((dyn / sizeof(double) + 31) / 32 * 32);
  if (global_rows) {
    const size_t need = sizeof(double) * (size_t)gstride * (size_t)nblocks;
    if (c.ac_gwork_bytes < need) {
      void* p = nullptr;
      TTR_CHECK(c.alloc(&p, need));
      c.ac_gwork = static_cast<double*>(p);
      c.ac_gwork_bytes = need;
    }
    gwork = c.ac_gwork;
  }
  if (dyn_launch > 0) {
    // the limit belongs to the kernel, shared by every thread that calls it: only ever raise it
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (di.raised[ki] < (int)dyn_launch) {
      TTR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_launch));
      int per_sm = 0;
      TTR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ac::NT, dyn_launch));
      if (per_sm < 1) return TTR_ERR_UNSUPPORTED;
      di.raised[ki] = (int)dyn_launch;
    }
  }
  // largest reduction: first block (b0^2 + b0 bi) or the second one of a block ((cc + bb)(bb + bi)
  // <= 2 rbar bi); the estimate's (1 + bi^2) and fresh coefficients (rbar bi) are smaller
  const int used = (std::max(b0 * b0 + b0 * bi, 1 + 2 * rbar * bi) + 1 + 31) / 32 * 32;
  if (!c.ac_bar) {
    TTR_CHECK(c.alloc_t(&c.ac_bar, 4));
    TTR_CUDA(cudaMemsetAsync(c.ac_bar, 0, 4 * sizeof(unsigned), c.stream));
  }
  if (c.ac_part_cap < used) {
    const int cap = std::max(used, ac::ACC + 64);
    TTR_CHECK(c.alloc_t(&c.ac_part, (size_t)3 * ac::RCOPY * cap));   // 3 rotating accumulation buffers
    c.ac_part_cap = cap;
  }
  // status words and the estimates share one device buffer, read back by a single copy:
  // [status, cc, count, -] ints, then up to est_cap doubles
  const int cap = std::max(est_cap, 8);
  if (c.ac_io_cap < cap) {
    void* mem = nullptr;
    TTR_CHECK(c.alloc(&mem, 16 + sizeof(double) * (size_t)cap));
    c.ac_io = static_cast<int*>(mem);
    c.ac_io_cap = cap;
  }
  if (!c.d_flags) {
    TTR_CHECK(c.alloc_t(&c.d_flags, 4));
    TTR_CUDA(cudaMemsetAsync(c.d_flags, 0, 4 * sizeof(int), c.stream));
  }
  TTR_CUDA(cudaMemsetAsync(c.ac_part, 0, sizeof(double) * 3 * ac::RCOPY * used, c.stream));
  ac::Args a{};
  a.Sall = Sall; a.lds = lds; a.Q = Q; a.ldq = ldq; a.S = S; a.acc = c.ac_part; a.acc_used = used;
  a.m = m; a.qcols = qcols; a.rpc = rpc; a.b0 = b0; a.bi = bi; a.ba = ba; a.rbar = rbar; a.width = width; a.cc0 = cc0;
  a.tau = tau;
  a.bar = c.ac_bar; a.err = c.d_flags; a.est_out = reinterpret_cast<double*>(c.ac_io + 4); a.io = c.ac_io;
  a.gwork = gwork; a.gstride = gstride;
  a.tc_off = (int)tc_off;
  a.tc_cols = (ba + bi <= 32) ? 256 : 512;
  // double-float keeps binary32 exponents: hold the sketch scaled so that ||X|| maps near 1
  a.sshift = 0;
  if (double_float && scale > 0.0 && isfinite(scale)) {
    int ex = 0;
    frexp(scale, &ex);
    a.sshift = -ex;
  }
  if (c.profiling) {
    if (!c.ac_prof) {
      TTR_CHECK(c.alloc_t(&c.ac_prof, ac::PH_COUNT));
      TTR_CUDA(cudaMemsetAsync(c.ac_prof, 0, sizeof(unsigned long long) * ac::PH_COUNT, c.stream));
    }
    a.prof = c.ac_prof;
  }
  void* params[] = {&a};
  c.time_begin(Ctx::KT_BLOCK_LOOP);
  TTR_CUDA(cudaLaunchCooperativeKernel(kern, dim3(nblocks), dim3(ac::NT), params, dyn_launch, c.stream));
  TTR_CHECK(c.check_launch("adaptive_core"));
  // one launch makes at most one estimate per block it runs
  const int est_max = std::min(cap, (rbar - cc0) / std::max(1, ba) + 3);
  std::vector<unsigned char> back(16 + sizeof(double) * (size_t)est_max);
  TTR_CUDA(cudaMemcpyAsync(back.data(), c.ac_io, back.size(), cudaMemcpyDeviceToHost, c.stream));
  TTR_CUDA(cudaStreamSynchronize(c.stream));
  int io[4];
  memcpy(io, back.data(), sizeof(io));
  if (io[0] == ac::ST_TIMEOUT) return set_error("adaptive loop: grid barrier wait ran out"), TTR_ERR_TIMEOUT;
  if (io[2] < 0 || io[2] > est_max || io[2] > est_cap) return set_error("adaptive loop: estimate count"), TTR_ERR_CUDA;
  *status = io[0];
  *cc = io[1];
  *nest = io[2];
  memcpy(est_host, back.data() + 16, sizeof(double) * (size_t)io[2]);
  if (c.timing) {
    // FP64 arithmetic of the blocks the kernel ran (2 flops per multiply-add), in its order:
    // first block (two CholeskyQR passes and the first coefficients), then per estimate the
    // residual, its norm and Gram matrix and, when the loop went on, the two passes with the block
    // Gram-Schmidt step between them and the next block's coefficients
    const double M = (double)m;
    double f = 0.0;
    int cur = cc0;
    if (cc0 == 0) {
      f += 2.0 * (2.0 * M * b0 * b0 + M * b0 * b0) + 2.0 * M * b0 * bi;
      cur = b0;
    } else {
      f += 2.0 * M * cur * bi;
    }
    for (int i = 0; i < *nest && cur < rbar; ++i) {
      const int bb = std::min(ba, rbar - cur);
      f += 2.0 * M * cur * bi + 2.0 * M * bi + 2.0 * M * bb * bb;
      if (i + 1 < *nest || *status != ac::ST_DONE) {
        f += M * bb * bb + 4.0 * M * cur * bb + 2.0 * M * bb * bb + 2.0 * M * (cur + bb) * bi + M * bb * bb;
        cur += bb;
      }
    }
    c.time_end(f);
  }
  return TTR_OK;
}

}  // namespace ttr
