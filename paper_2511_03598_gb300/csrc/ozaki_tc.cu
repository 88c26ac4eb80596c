// FP64-accurate contractions on the BF16 tensor cores (tcgen05, sm_103a).
//
// GB300 runs FP64 FMA at ~1.2 TFLOP/s but BF16 MMA at ~2 PFLOP/s, so the large contractions of
// the rounding (the right-to-left partial contractions of Algorithm 3, the sketches
// S_k = V(Y_k) W_{k+1} and the next-core projections M_k H(X_{k+1})) are computed from
// fixed-point slices of the FP64 operands, in the manner of the Ozaki splitting scheme
// (Ozaki, Ogita, Oishi, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 2012):
//
//  * every row m of A (or, for partial contractions, every mode slab X_k(a, :, :)) gets the
//    scale 2^(Emax_m - 1022) of its largest entry; each entry becomes a 7*s-bit integer
//    v = floor(|a| 2^(7s - Emax_m + 1022)) cut into s base-128 digits (sign attached), each
//    exactly representable in BF16; columns of B get digits the same way;
//  * digit products a_p b_q with p + q = t are accumulated on the tensor cores into one FP32
//    TMEM accumulator per "diagonal" t < s.  With |digit| <= 127 and at most 256 K-terms per
//    accumulation, diagonals t <= 3 stay below 2^24 (exact integers); higher diagonals carry
//    weights <= 2^-28 relative, so their FP32 rounding is below 2^-52 of the result;
//  * the epilogue converts the accumulators to integers and forms
//    V = sum_t acc_t 2^(7(s-1-t)) in 128-bit integer arithmetic, and only then scales to FP64
//    (or, for partial contractions, weights by the integer sketch entries 2^20*Omega and sums
//    over the mode index exactly before the single conversion).  No FP64 arithmetic runs per
//    element, which matters on this FP64-starved part.
//
// Truncating the digits and the diagonals at s leaves a relative error of about s*2^(1-7s)
// of the row/column scales: 8 slices reach FP64 accuracy, 5 slices ~1e-10.
//
// The same kernels also run the reduced-precision sketch forms (Args::flt): each operand value is
// stored as one BF16 plane (its BF16 rounding), or as two (the BF16 head and tail of its TF32
// rounding, so that head*head + head*tail + tail*head on two FP32 accumulators reproduces a TF32
// product with FP32 accumulation); no exponent scan, and the epilogue converts the FP32
// accumulators to FP64 and, for partial contractions, weights by the FP64 sketch entries and sums
// each slab in FP64.
//
// Operands are staged by the CTA's threads into shared memory in the canonical K-major,
// no-swizzle UMMA layout (8x16-byte core matrices; the leading byte offset steps along K,
// the stride byte offset along M/N), double-buffered across K-chunks of 32; one thread issues
// the tcgen05.mma instructions and commits them to an mbarrier; accumulators live in TMEM
// and come back through tcgen05.ld.  All device waits are bounded.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "engine.cuh"
#include "sliced_mma.cuh"

namespace ttr {
namespace tc {

constexpr int TNMAX = 256;            // largest UMMA N; the tile width tn is chosen per call
constexpr int PB = 64;                // partial-contraction epilogue: columns per staging block
constexpr int KSEG = 256;             // largest K per CTA: bound for exact FP32 accumulation
constexpr int PLANE_A = TM * KC;      // bf16 per A digit plane per chunk (8 KB)

constexpr int NP = 512;               // producer threads: slicing, then the epilogue (4 warps per TMEM lane quarter)
constexpr int NWP = NP / 32;          // producer warps
constexpr int MMA_WARP = NWP;         // one more warp issues the tensor-core instructions
constexpr int NT = NP + 32;           // threads per CTA

enum Mode { PLAIN = 0, ATOMIC = 1, RLM = 2 };

struct Args {
  const double* A;
  int64_t M, K, sam, sak;
  const uint4* Bp;                    // digit planes [nchunk][kchunk][s][tn*KC]
  const int* Fmax;                    // biased exponent scale of each B column [nchunks*tn]
  int tn;                             // tile width (UMMA N): multiple of 16, s*tn <= 512
  int64_t N;
  int kchunks;                        // ceil(K / KC)
  int s;
  double* C;
  int64_t scm, scn;
  // partial-contraction epilogue
  const int* Omint;                   // 2^20 * Omega(i, j), [i * ldo + j]
  int64_t ldo;
  int64_t nmode;                      // n_k: rows per slab
  int g;                              // slabs per tile
  int64_t slabs;                      // r_{k-1}
  double* W;
  int64_t ldw;
  int watomic;                        // partial contractions split over K: add into W atomically
  int kseg;                           // K per CTA (multiple of KC, <= KSEG); blockIdx.z selects the segment
  int* err;
  unsigned long long* prof;           // optional phase cycles of CTA (0, 0, 0) (launch-timeline profiling)
  // plain mode: output row m lands at row (m / rp) * rstride + m % rp of C (rp = 0: at row m), which
  // places the columns (i, c) of one summand's block of H(Y_{k+1}) inside the stacked right bond
  int64_t rp, rstride;
  int flt;                            // reduced-precision operands: s = 1 BF16, s = 2 TF32 (head, tail)
  const double* Omd;                  // flt partial contractions: Omega(i, j) [i * ldo + j]
};

// Up to MAXG independent products of one grouped launch (the summands of a sum of TTs): each
// group has its own A, K, rows and output, and its own rows koff .. koff + K - 1 of one stacked B
// operand.  A group reads the B chunks that hold its rows and places its A columns at the same
// positions (shifted by koff % KC); the rows of other groups in a shared boundary chunk meet zero
// A digits.
constexpr int MAXG = 8;
static_assert(MAXG == kMaxGroup, "group table size");
struct Groups {
  int n;                      // 0: one product, described by Args alone
  int tile0[MAXG + 1];        // first blockIdx.x of each group (tile0[n] = gridDim.x)
  const double* A[MAXG];
  int64_t M[MAXG];            // rows (plain mode; slabs * nmode in partial-contraction mode)
  int64_t K[MAXG];
  int64_t sam[MAXG], sak[MAXG];
  int64_t slabs[MAXG];        // partial-contraction mode: r_{k-1} of the group
  int64_t koff[MAXG];         // first row of the group in the stacked B
  double* C[MAXG];            // plain mode output (strides scm, scn of the group)
  int64_t scm[MAXG], scn[MAXG];
  double* W[MAXG];            // partial-contraction mode output rows (leading dimension Args::ldw)
  int64_t rp[MAXG];           // plain mode output row blocks (Args::rp), stride Args::rstride
};

// phases of one CTA, timed by thread 0 (setup, row scan, producers' chunk loop, waiting for the
// last MMAs, epilogue) and by the MMA thread (its chunk loop)
enum TcPhase { TP_SETUP = 0, TP_SCAN, TP_CHUNKS, TP_DRAIN, TP_EPILOGUE, TP_MMA_LOOP, TP_COUNT };

// Reduced-precision forms: the BF16 rounding of 8 values (s = 1), or the BF16 head and tail of
// their TF32 rounding (s = 2; TF32 keeps 11 significant bits, the head 8, so the tail is exact).
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float tf32_round(float x) {
  const uint32_t u = __float_as_uint(x);
  if (((u >> 23) & 0xFF) == 0xFF) return x;                  // inf / nan unchanged
  return __uint_as_float((u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu);
}
__device__ __forceinline__ void store_float_s(int s, const double* v, uint16_t* planes, size_t plane_stride, int idx) {
  uint16_t hbits[8], tbits[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float f = __double2float_rn(v[q]);
    if (s == 1) {
      hbits[q] = bf16_bits(f);
    } else {
      const float t = tf32_round(f);
      const __nv_bfloat16 h = __float2bfloat16_rn(t);
      hbits[q] = __bfloat16_as_ushort(h);
      tbits[q] = bf16_bits(t - __bfloat162float(h));
    }
  }
  uint4 hw, tw;
  hw.x = hbits[0] | ((uint32_t)hbits[1] << 16); hw.y = hbits[2] | ((uint32_t)hbits[3] << 16);
  hw.z = hbits[4] | ((uint32_t)hbits[5] << 16); hw.w = hbits[6] | ((uint32_t)hbits[7] << 16);
  *reinterpret_cast<uint4*>(planes + idx) = hw;
  if (s == 2) {
    tw.x = tbits[0] | ((uint32_t)tbits[1] << 16); tw.y = tbits[2] | ((uint32_t)tbits[3] << 16);
    tw.z = tbits[4] | ((uint32_t)tbits[5] << 16); tw.w = tbits[6] | ((uint32_t)tbits[7] << 16);
    *reinterpret_cast<uint4*>(planes + plane_stride + idx) = tw;
  }
}

__device__ __forceinline__ void store_digits_s(int s, const double* v, int E, uint16_t* planes, size_t plane_stride,
                                               int idx) {
  switch (s) {
    case 3: store_digits<3>(v, E, planes, plane_stride, idx); break;
    case 4: store_digits<4>(v, E, planes, plane_stride, idx); break;
    case 5: store_digits<5>(v, E, planes, plane_stride, idx); break;
    case 6: store_digits<6>(v, E, planes, plane_stride, idx); break;
    case 7: store_digits<7>(v, E, planes, plane_stride, idx); break;
    default: store_digits<8>(v, E, planes, plane_stride, idx); break;
  }
}

// The products of one K-chunk.  For each of the two 16-deep K-steps and each A digit plane p, the
// B planes q = 0 .. S-1-p go to the accumulators of diagonals p + q, TMEM columns [(p + q) tn, ..);
// with the B layout of b_digit_index those planes are adjacent along N, so one MMA covers up to
// floor(256 / tn) of them (N <= 256).  Descriptors are built once and advanced by constant offsets
// in their 14-bit start-address field (every operand lies inside this CTA's shared memory, so the
// field cannot overflow).  The first write of every accumulator comes from p = 0.
template <int S>
__device__ __forceinline__ void issue_chunk(uint64_t da0, uint64_t db0, uint32_t tmem, int tn, uint32_t idesc0,
                                            bool first) {
  constexpr uint32_t PA = (PLANE_A * 2) >> 4;            // one A digit plane
  constexpr uint32_t KSA = (2 * (TM / 8) * 128) >> 4;     // one 16-deep K-step of A
  const uint32_t pb = (uint32_t)((tn / 8) * 128) >> 4;   // one B digit plane (its row groups)
  const uint32_t ksb = (uint32_t)(2 * S * (tn / 8) * 128) >> 4;
  const int G = 256 / tn;                                 // B planes per MMA
#pragma unroll
  for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
    for (int p = 0; p < S; ++p) {
      const uint64_t da = da0 + (uint64_t)(p * PA + ks * KSA);
      for (int q0 = 0; q0 < S - p; q0 += G) {
        const int nq = min(G, S - p - q0);
        const uint64_t db = db0 + (uint64_t)((uint32_t)q0 * pb + (uint32_t)ks * ksb);
        const uint32_t idesc = idesc0 | ((uint32_t)((nq * tn) >> 3) << 17);
        const uint32_t accum = (first && ks == 0 && p == 0) ? 0u : 1u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)((p + q0) * tn)),
                     "l"(da), "l"(db), "r"(idesc), "r"(accum));
      }
    }
  }
}

// 17 warps: one SM sub-partition holds 5 of them, so its 16K registers cap a thread at 96.
template <int MODE, bool AKFAST, bool GROUPED, bool FLT>
__global__ void __launch_bounds__(NT, 1) sliced_kernel(const Args a0, const Groups gr) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // this CTA's product: the launch's, or that of its group (tiles numbered within the group)
  Args a = a0;
  int64_t bx = blockIdx.x;
  int kcb = 0;          // first B chunk of this CTA's product
  int ksh = 0;          // position of its first K column within that chunk
  if (GROUPED) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < MAXG; ++q)
      if (q < gr.n && (int)blockIdx.x >= gr.tile0[q]) g = q;
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
      if (q == g) {
        a.A = gr.A[q]; a.M = gr.M[q]; a.K = gr.K[q]; a.sam = gr.sam[q]; a.sak = gr.sak[q];
        a.slabs = gr.slabs[q]; a.C = gr.C[q]; a.scm = gr.scm[q]; a.scn = gr.scn[q]; a.W = gr.W[q]; a.rp = gr.rp[q];
        kcb = (int)(gr.koff[q] / KC);
        ksh = (int)(gr.koff[q] % KC);
        bx -= gr.tile0[q];
      }
    }
  }
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t full[2];    // digit buffer b filled (NP producer arrivals)
  __shared__ __align__(8) uint64_t empty[2];   // MMAs reading digit buffer b done (tcgen05.commit)
  __shared__ int rowE[TM];
  __shared__ int slabE[TM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = a.s;
  const int nc = blockIdx.y;
  const int64_t kseg0 = (int64_t)blockIdx.z * a.kseg;
  const int kseg_len = (int)(a.K - kseg0 < (int64_t)a.kseg ? a.K - kseg0 : (int64_t)a.kseg);
  const int nchunk = (ksh + kseg_len + KC - 1) / KC;
  const int kc0 = (int)(kseg0 / KC);
  // rows of this tile
  int64_t m0;
  int rows;
  if (MODE == RLM) {
    const int64_t s0 = bx * a.g;
    const int64_t na = (a.slabs - s0 < (int64_t)a.g) ? a.slabs - s0 : (int64_t)a.g;
    m0 = s0 * a.nmode;
    rows = (int)(na * a.nmode);
  } else {
    m0 = bx * TM;
    rows = (int)(a.M - m0 < (int64_t)TM ? a.M - m0 : (int64_t)TM);
  }
  const int tn = a.tn;
  const int plane_b = tn * KC;
  const uint32_t tcols = (s * tn <= 256) ? 256u : 512u;
  const size_t buf_bytes = (size_t)s * (PLANE_A + plane_b) * 2;
  unsigned char* bufs[2] = {smem, smem + buf_bytes};

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(NP));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < TM) {
    slabE[tid] = 1;
    rowE[tid] = 1;
  }
  const bool timed = a.prof && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
  const int pslot = TP_COUNT * MODE;
  long long t_prev = clock64();
  auto mark = [&](int ph) {
    if (timed && tid == 0) {
      const long long t = clock64();
      atomicAdd(a.prof + pslot + ph, (unsigned long long)(t - t_prev));
      t_prev = t;
    }
  };
  __syncthreads();
  mark(TP_SETUP);

  // ---- pass 1: exponent scale of every row over this K segment (many loads in flight)
  if (warp >= NWP || FLT) {
    // the MMA warp takes no part in the scan; the reduced-precision forms need no scale
  } else if (AKFAST) {
    // row-major A: a warp scans 8 rows; each step loads one value of each row per lane
    constexpr int RPW = TM / NWP;
    int em[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) em[r] = 1;
    for (int k = lane; k < kseg_len; k += 32) {
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int row = warp * RPW + r;
        if (row < rows) em[r] = max(em[r], exp_field(__ldcg(a.A + (m0 + row) * a.sam + kseg0 + k)));
      }
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int e = __reduce_max_sync(0xffffffffu, em[r]);
      if (lane == 0) rowE[warp * RPW + r] = e;
    }
  } else {
    // column-major A: lanes take 32 consecutive rows (coalesced), the four warps of a row group
    // interleave over k, 16 loads in flight per lane
    const int row = (warp & 3) * 32 + lane, kp = warp >> 2;
    constexpr int KP = NWP / 4;
    int e = 1;
    if (row < rows) {
      const double* colp = a.A + (m0 + row) * a.sam + kseg0 * a.sak;
#pragma unroll 1
      for (int k0 = kp; k0 < kseg_len; k0 += 16 * KP) {
        double x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int k = k0 + KP * j;
          x[j] = (k < kseg_len) ? __ldcg(colp + (int64_t)k * a.sak) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) e = max(e, exp_field(x[j]));
      }
    }
    atomicMax(&rowE[row], e);
  }
  __syncthreads();
  if (MODE == RLM) {
    if (tid < rows) atomicMax(&slabE[tid / a.nmode], rowE[tid]);
    __syncthreads();
    if (tid < rows) rowE[tid] = slabE[tid / a.nmode];
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  // instruction descriptor without N (set per MMA): FP32 accumulation, BF16 A and B, K-major, M = 128
  const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TM >> 4) << 24);
  bool ok = true;
  mark(TP_SCAN);

  // ---- K loop over chunks of 32: the producer warps slice chunk c into digit buffer c % 2 and
  // arrive on full[c % 2]; the MMA warp waits for it, issues the chunk's products and commits them
  // to empty[c % 2], which the producers wait for before refilling that buffer (chunk c + 2).
  // Every wait is bounded; a wait that runs out sets the error flag and the CTA winds down.
  if (warp == MMA_WARP) {
    if (lane == 0) {
      const long long tm0 = clock64();
      for (int c = 0; c < nchunk && ok; ++c) {
        const int b = c & 1;
        ok = mbar_wait(smem_u32(&full[b]), (uint32_t)((c >> 1) & 1), a.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t abase = smem_u32(bufs[b]), bbase = abase + (uint32_t)(s * PLANE_A * 2);
        const uint64_t da0 = umma_desc(abase, (TM / 8) * 128, 128);
        const uint64_t db0 = umma_desc(bbase, s * (tn / 8) * 128, 128);
        switch (s) {
          case 1: issue_chunk<1>(da0, db0, tmem, tn, idesc0, c == 0); break;
          case 2: issue_chunk<2>(da0, db0, tmem, tn, idesc0, c == 0); break;
          case 3: issue_chunk<3>(da0, db0, tmem, tn, idesc0, c == 0); break;
          case 4: issue_chunk<4>(da0, db0, tmem, tn, idesc0, c == 0); break;
          case 5: issue_chunk<5>(da0, db0, tmem, tn, idesc0, c == 0); break;
          case 6: issue_chunk<6>(da0, db0, tmem, tn, idesc0, c == 0); break;
          case 7: issue_chunk<7>(da0, db0, tmem, tn, idesc0, c == 0); break;
          default: issue_chunk<8>(da0, db0, tmem, tn, idesc0, c == 0); break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empty[b])));
      }
      if (timed) atomicAdd(a.prof + pslot + TP_MMA_LOOP, (unsigned long long)(clock64() - tm0));
    }
    __syncwarp();
  } else {
    // A digits: 128 rows x 4 groups of 8 consecutive k = 512 tasks, TASKS per thread; the values of
    // chunk c + 1 are loaded into registers while chunk c is being sliced.  Row-major A: a warp
    // takes 8 rows x 4 groups (its loads cover 32 consecutive k of each row), lane l row l % 8 and
    // group l / 8, so that the 8 lanes of each quarter-warp store phase write 8 different rows:
    // 8 different 16-byte bank groups of the digit plane.  Column-major A: lanes take consecutive
    // rows of one group (coalesced loads, and stores 16 bytes apart).
    constexpr int TASKS = (TM * (KC / 8)) / NP;
    int trow[TASKS], tgrp[TASKS];
#pragma unroll
    for (int i = 0; i < TASKS; ++i) {
      const int u = tid + NP * i;
      trow[i] = AKFAST ? ((u >> 5) * 8 + (u & 7)) : (u % TM);
      tgrp[i] = AKFAST ? ((u & 31) >> 3) : (u / TM);
    }
    auto load_chunk = [&](int c, double (&v)[TASKS][8]) {
#pragma unroll
      for (int i = 0; i < TASKS; ++i) {
        const int kb = c * KC + tgrp[i] * 8 - ksh;        // K column of the task's first value (< 0 only
                                                          // in a grouped launch's first chunk)
        const double* src = a.A + (m0 + trow[i]) * a.sam + (kseg0 + kb) * a.sak;
        const int klim = kseg_len - kb;
        const bool rok = trow[i] < rows;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          v[i][q] = (rok && q < klim && (!GROUPED || q >= -kb)) ? __ldcg(src + q * a.sak) : 0.0;
      }
    };
    double vc[TASKS][8];
    if (nchunk > 0) load_chunk(0, vc);
    for (int c = 0; c < nchunk && ok; ++c) {
      const int b = c & 1;
      if (c >= 2) ok = mbar_wait(smem_u32(&empty[b]), (uint32_t)(((c - 2) >> 1) & 1), a.err);
      if (!ok) break;
      uint16_t* Ap = (uint16_t*)bufs[b];
      uint16_t* Bpl = Ap + (size_t)s * PLANE_A;
      if (tid == 0) {
        // B digit planes of this chunk (s * tn * 64 contiguous bytes, 16-byte aligned at both ends):
        // one bulk async copy that completes on full[b]
        const uint4* src = a.Bp + ((size_t)nc * a.kchunks + (kcb + kc0 + c)) * (size_t)s * (plane_b / 8);
        const uint32_t bytes = (uint32_t)(s * plane_b * 2);
        asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])), "r"(bytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(Bpl)),
                     "l"(src), "r"(bytes), "r"(smem_u32(&full[b]))
                     : "memory");
      }
      double vn[TASKS][8];
      if (c + 1 < nchunk) load_chunk(c + 1, vn);
#pragma unroll
      for (int i = 0; i < TASKS; ++i) {
        const int row = trow[i], grp = tgrp[i];
        // From the third chunk on, tasks with no data (padding rows, k beyond the segment) keep
        // the digits this buffer held two chunks ago: those meet zero B digits (k >= K) or land in
        // accumulator rows the epilogue drops.  Chunks 0 and 1 write every position, so no
        // uninitialised shared memory ever reaches the tensor cores.
        // (A grouped launch writes every position: its B chunks may hold other groups' rows.)
        if (!GROUPED && c >= 2 && (row >= rows || c * KC + grp * 8 >= kseg_len)) continue;
        const int idx = ((grp * (TM / 8)) + (row >> 3)) * 64 + (row & 7) * 8;   // bf16 index in a plane
        if (FLT) store_float_s(s, vc[i], Ap, PLANE_A, idx);
        else store_digits_s(s, vc[i], rowE[row], Ap, PLANE_A, idx);
      }
#pragma unroll
      for (int i = 0; i < TASKS; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) vc[i][q] = vn[i][q];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[b])) : "memory");
    }
  }
  mark(TP_CHUNKS);
  if (ok && nchunk > 0) {
    const int c = nchunk - 1;
    ok = mbar_wait(smem_u32(&empty[c & 1]), (uint32_t)((c >> 1) & 1), a.err);
  }
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;");
  mark(TP_DRAIN);

  // ---- epilogue: warp w reads TMEM lane quarter (w % 4); the two warps of a quarter take
  // alternate 16-column groups.  Partial contractions stage int128 products per 64-column block.
  if (ok && nchunk > 0) {
    // [TM][PB] int128 staging for the slab sums; column index XOR (row % 8) spreads the 16-byte
    // stores of 32 consecutive rows over all banks
    __int128* P = reinterpret_cast<__int128*>(smem);
    const int quarter = warp & 3, half = warp >> 2;          // NWP / 4 warps share a lane quarter
    const int row = quarter * 32 + lane;
    const int ngroups = tn / 16;
    for (int blk0 = 0; blk0 < ngroups; blk0 += PB / 16) {
      const int blk1 = min(ngroups, blk0 + PB / 16);
      for (int cg = blk0 + half; warp < NWP && cg < blk1; cg += NWP / 4) {
        // V = sum_t acc_t 2^(7(s-1-t)) = Vh 2^35 + Vl, both parts in 64 bits: |acc_t| < 2^25, so
        // Vl (shifts 0..28) < 2^56 and Vh (shifts 35..49, less 35) < 2^41.  The accumulators are
        // integer-valued binary32 values, so the float-to-int32 conversion is exact.
        long long Vh[16], Vl[16];
        double Vd[FLT ? 16 : 1];              // reduced-precision forms: sum of the FP32 accumulators
#pragma unroll
        for (int j = 0; j < 16; ++j) Vh[j] = Vl[j] = 0;
#pragma unroll
        for (int j = 0; j < (FLT ? 16 : 1); ++j) Vd[j] = 0.0;
#pragma unroll 1
        for (int t = 0; t < s; ++t) {
          uint32_t r[16];
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * tn + cg * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (FLT) {
#pragma unroll
            for (int j = 0; j < (FLT ? 16 : 1); ++j) Vd[j] += (double)__uint_as_float(r[j]);
            continue;
          }
          const int shift = 7 * (s - 1 - t);
          if (shift >= 35) {
            const long long mul = 1LL << (shift - 35);
#pragma unroll
            for (int j = 0; j < 16; ++j) Vh[j] += (long long)__float2int_rz(__uint_as_float(r[j])) * mul;
          } else {
            const long long mul = 1LL << shift;
#pragma unroll
            for (int j = 0; j < 16; ++j) Vl[j] += (long long)__float2int_rz(__uint_as_float(r[j])) * mul;
          }
        }
        // with s <= 6, Vh is the top diagonal alone (|Vh| < 2^25), so V < 2^61 fits in 64 bits
        const bool v64 = s <= 6;
        __int128 V[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) V[j] = (__int128)Vh[j] * ((__int128)1 << 35) + (__int128)Vl[j];
        const int64_t n0 = (int64_t)nc * tn + cg * 16;
        if (MODE != RLM) {
          if (row < rows) {
            const int e_row = rowE[row];
            const int64_t mrow = m0 + row;
            int64_t maddr = mrow;
            if (GROUPED && a.rp > 0) {   // rows < 2^31 (checked by the host)
              const uint32_t q = (uint32_t)mrow / (uint32_t)a.rp;
              maddr = (int64_t)q * a.rstride + ((uint32_t)mrow - q * (uint32_t)a.rp);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int64_t n = n0 + j;
              if (n < a.N) {
                double out;
                if (FLT) {
                  out = Vd[FLT ? j : 0];
                } else {
                  const int X = e_row + max(1, a.Fmax[n]) - 2044 - 7 * s - 7;
                  out = v64 ? i64_to_double(Vh[j] * (1LL << 35) + Vl[j], X) : i128_to_double(V[j], X);
                }
                double* cp = a.C + maddr * a.scm + n * a.scn;
                if (MODE == ATOMIC) atomicAdd(cp, out);
                else *cp = out;
              }
            }
          }
        } else {
          // weight by the integer sketch entry 2^20 Omega(i, n); summed over i below (the
          // reduced-precision forms: by Omega(i, n) in FP64, into the same slots as doubles)
          const int i = row % (int)a.nmode;
          if (FLT) {
            double* PD = reinterpret_cast<double*>(P);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int64_t n = n0 + j;
              const double om = (row < rows && n < a.N) ? a.Omd[i * a.ldo + n] : 0.0;
              PD[row * PB + (((cg - blk0) * 16 + j) ^ (row & 7))] = Vd[FLT ? j : 0] * om;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int64_t n = n0 + j;
              const int om = (row < rows && n < a.N) ? a.Omint[i * a.ldo + n] : 0;
              P[row * PB + (((cg - blk0) * 16 + j) ^ (row & 7))] = V[j] * (__int128)om;
            }
          }
        }
      }
      if (MODE == RLM) {
        __syncthreads();
        const int nslab = rows / (int)a.nmode;
        const int bcols = (blk1 - blk0) * 16;
        for (int task = tid; task < nslab * bcols; task += NT) {
          const int sl = task / bcols, j = task % bcols;
          const int64_t n = (int64_t)nc * tn + blk0 * 16 + j;
          if (n >= a.N) continue;
          const int64_t aidx = bx * a.g + sl;
          double out;
          if (FLT) {
            const double* PD = reinterpret_cast<const double*>(P);
            double accd = 0.0;
            for (int ii = 0; ii < (int)a.nmode; ++ii) {
              const int r = sl * (int)a.nmode + ii;
              accd += PD[r * PB + (j ^ (r & 7))];
            }
            out = accd;
          } else {
            __int128 acc = 0;
            for (int ii = 0; ii < (int)a.nmode; ++ii) {
              const int r = sl * (int)a.nmode + ii;
              acc += P[r * PB + (j ^ (r & 7))];
            }
            const int e_slab = rowE[sl * (int)a.nmode];
            out = i128_to_double(acc, e_slab + max(1, a.Fmax[n]) - 2044 - 7 * s - 7 - 20);
          }
          if (a.watomic) atomicAdd(a.W + aidx * a.ldw + n, out);
          else a.W[aidx * a.ldw + n] = out;
        }
        __syncthreads();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  mark(TP_EPILOGUE);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}


// ---- B operand preparation: column exponent scales, then digit planes in the shared-memory
// image.  B(k, n) = B[k*sbk + n*sbn], K x N.
// Pass 1: grid (N-chunks, up to 128 CTAs along K); each CTA takes the largest exponent of each of
// its tn columns over the K-chunks of 32 rows y, y + gridDim.y, ... and folds it into Fmax[column]
// with one integer atomic maximum per column (Fmax is zeroed before the launch; every exponent
// field is at least 1).
__global__ void __launch_bounds__(256) colmax_b_kernel(const double* B, int64_t sbk, int64_t sbn, int64_t K, int64_t N,
                                                       int tn, int* Fmax) {
  __shared__ int cm[TNMAX];
  const int nc = blockIdx.x;
  for (int j = threadIdx.x; j < tn; j += blockDim.x) cm[j] = 1;
  __syncthreads();
  const int64_t kchunks = (K + KC - 1) / KC;
  // a task reads 8 rows of one column (all loads in flight)
  for (int64_t y = blockIdx.y; y < kchunks; y += gridDim.y) {
    for (int u = threadIdx.x; u < tn * (KC / 8); u += blockDim.x) {
      const int j = u % tn, grp = u / tn;
      const int64_t n = (int64_t)nc * tn + j;
      if (n >= N) continue;
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t k = y * KC + grp * 8 + q;
        v[q] = (k < K) ? B[k * sbk + n * sbn] : 0.0;
      }
      int e = 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) e = max(e, exp_field(v[q]));
      atomicMax(&cm[j], e);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < tn; j += blockDim.x) atomicMax(Fmax + (int64_t)nc * tn + j, cm[j]);
}

// Pass 2: one CTA per (tn-column chunk, 32-row K chunk), after pass 1 has completed Fmax (the
// column scales); tasks (column, group of 8 k) write the s digit planes.
__global__ void __launch_bounds__(256) slice_b_kernel(const double* B, int64_t sbk, int64_t sbn, int64_t K, int64_t N,
                                                      int s, int tn, int kchunks, const int* Fmax, uint4* planes) {
  __shared__ int E[TNMAX];
  const int nc = blockIdx.x, kcn = blockIdx.y;
  for (int j = threadIdx.x; j < tn; j += blockDim.x) E[j] = max(1, __ldg(Fmax + (int64_t)nc * tn + j));
  __syncthreads();
  const int plane_b = tn * KC;
  uint4* blk = planes + ((size_t)nc * kchunks + kcn) * (size_t)s * (plane_b / 8);
  for (int u = threadIdx.x; u < tn * (KC / 8); u += blockDim.x) {
    const int j = u % tn, grp = u / tn;
    const int64_t n = (int64_t)nc * tn + j;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)kcn * KC + grp * 8 + q;
      v[q] = (n < N && k < K) ? B[k * sbk + n * sbn] : 0.0;
    }
    store_digits_s(s, v, E[j], reinterpret_cast<uint16_t*>(blk), tn * 8, b_digit_index(grp, j, s, tn));
  }
}

// Both passes in one cooperative launch: each CTA keeps its B values in registers across a bounded
// grid barrier (counter and generation in bar[0], bar[1], left at counter 0 for the next use), so B
// is read once and one launch replaces two.
constexpr int PREP_TASKS = (TNMAX * (KC / 8) + 255) / 256;
__global__ void __launch_bounds__(256) prep_b_fused_kernel(const double* B, int64_t sbk, int64_t sbn, int64_t K,
                                                           int64_t N, int s, int tn, int kchunks, int64_t npad,
                                                           int* Fpart, int* Fmax, uint4* planes, unsigned* bar,
                                                           int* err) {
  __shared__ int cm[TNMAX];
  __shared__ int ok_s;
  const int nc = blockIdx.x, kcn = blockIdx.y;
  for (int j = threadIdx.x; j < tn; j += blockDim.x) cm[j] = 1;
  __syncthreads();
  double v[PREP_TASKS][8];
#pragma unroll
  for (int t = 0; t < PREP_TASKS; ++t) {
    const int u = threadIdx.x + 256 * t;
    const int j = u % tn, grp = u / tn;
    const int64_t n = (int64_t)nc * tn + j;
    const bool live = u < tn * (KC / 8) && n < N;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)kcn * KC + grp * 8 + q;
      v[t][q] = (live && k < K) ? B[k * sbk + n * sbn] : 0.0;
    }
    if (live) {
      int e = 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) e = max(e, exp_field(v[t][q]));
      atomicMax(&cm[j], e);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < tn; j += blockDim.x) Fpart[(int64_t)kcn * npad + (int64_t)nc * tn + j] = cm[j];
  // grid barrier
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    ok_s = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    if (atomicAdd(bar, 1u) == total - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > WAIT_CYCLES) {
          atomicExch(err, 1);
          ok_s = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (!ok_s) return;
  for (int j = threadIdx.x; j < tn; j += blockDim.x) {
    int e = 1;
    const int* fp = Fpart + (int64_t)nc * tn + j;
    for (int q = 0; q < kchunks; ++q) e = max(e, __ldcg(fp + (int64_t)q * npad));
    cm[j] = e;
    if (kcn == 0) Fmax[(int64_t)nc * tn + j] = e;
  }
  __syncthreads();
  const int plane_b = tn * KC;
  uint4* blk = planes + ((size_t)nc * kchunks + kcn) * (size_t)s * (plane_b / 8);
#pragma unroll
  for (int t = 0; t < PREP_TASKS; ++t) {
    const int u = threadIdx.x + 256 * t;
    if (u >= tn * (KC / 8)) continue;
    const int j = u % tn, grp = u / tn;
    store_digits_s(s, v[t], cm[j], reinterpret_cast<uint16_t*>(blk), tn * 8, b_digit_index(grp, j, s, tn));
  }
}

// Reduced-precision forms: B(k, n) as s = 1 (BF16) or 2 (TF32 head and tail) planes in the layout of
// b_digit_index; no column scales.
__global__ void __launch_bounds__(256) slice_b_float_kernel(const double* B, int64_t sbk, int64_t sbn, int64_t K,
                                                            int64_t N, int s, int tn, int kchunks, uint4* planes) {
  const int nc = blockIdx.x, kcn = blockIdx.y;
  const int plane_b = tn * KC;
  uint4* blk = planes + ((size_t)nc * kchunks + kcn) * (size_t)s * (plane_b / 8);
  for (int u = threadIdx.x; u < tn * (KC / 8); u += blockDim.x) {
    const int j = u % tn, grp = u / tn;
    const int64_t n = (int64_t)nc * tn + j;
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int64_t k = (int64_t)kcn * KC + grp * 8 + q;
      v[q] = (n < N && k < K) ? B[k * sbk + n * sbn] : 0.0;
    }
    store_float_s(s, v, reinterpret_cast<uint16_t*>(blk), tn * 8, b_digit_index(grp, j, s, tn));
  }
}

static size_t smem_bytes(int s, int tn, int mode) {
  size_t need = 2 * (size_t)s * (PLANE_A + tn * KC) * 2;
  if (mode == RLM) need = std::max(need, (size_t)TM * PB * sizeof(__int128));
  // TMEM: 2 CTAs per SM only when each takes 256 columns; otherwise shared memory keeps it at 1
  if (s * tn <= 256) need = std::max<size_t>(need, 100 * 1024);
  else need = std::max<size_t>(need, 118 * 1024);
  return need + 1024;
}

template <int MODE, bool AKFAST>
static int launch(Ctx& c, const Args& a_in, dim3 grid, const char* name, const Groups* groups = nullptr) {
  Args a = a_in;
  Groups gr{};
  if (groups) gr = *groups;
  if (c.profiling) {
    if (!c.tc_prof) {
      TTR_CHECK(c.alloc_t(&c.tc_prof, 3 * TP_COUNT));
      TTR_CUDA(cudaMemsetAsync(c.tc_prof, 0, sizeof(unsigned long long) * 3 * TP_COUNT, c.stream));
    }
    a.prof = c.tc_prof;
  }
  const size_t sm = smem_bytes(a.s, a.tn, MODE);
  if (groups && a.flt) return set_error("grouped reduced-precision products are not built"), TTR_ERR_UNSUPPORTED;
  auto kern = groups ? sliced_kernel<MODE, AKFAST, true, false>
                     : (a.flt ? sliced_kernel<MODE, AKFAST, false, true> : sliced_kernel<MODE, AKFAST, false, false>);
  // the shared-memory limit belongs to the kernel and every calling thread shares it: raise it per
  // device to the largest size requested so far, never lower it
  constexpr int MAXDEV = 64;
  static int raised[3][MAXDEV] = {};           // [plain, grouped, reduced-precision kernel][device]
  static std::mutex mu;
  int dev = 0;
  TTR_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    int* slot = (dev >= 0 && dev < MAXDEV) ? &raised[groups ? 1 : (a.flt ? 2 : 0)][dev] : nullptr;
    const int have = slot ? *slot : 0;
    if (have < (int)sm) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return set_error(std::string("sliced kernel attribute: ") + cudaGetErrorString(e)), TTR_ERR_CUDA;
      if (slot) *slot = (int)sm;
    }
  }
  kern<<<grid, NT, sm, c.stream>>>(a, gr);
  return c.check_launch(name);
}

}  // namespace tc
int tile_width(int s);
namespace tc {

struct BPrep {
  uint4* planes = nullptr;
  int* Fmax = nullptr;
  int nchunks = 0, kchunks = 0, tn = 0;
};

static int ensure_err(Ctx& c) {
  if (!c.d_flags) {
    TTR_CHECK(c.alloc_t(&c.d_flags, 4));
    TTR_CUDA(cudaMemsetAsync(c.d_flags, 0, 4 * sizeof(int), c.stream));
  }
  return TTR_OK;
}

static int prep_b(Ctx& c, const double* B, int64_t sbk, int64_t sbn, int64_t K, int64_t N, int s, BPrep& p,
                  BPlanes* keep = nullptr, int tmax_in = 0) {
  const int tmax = tmax_in > 0 ? std::min(tmax_in, tile_width(s)) : tile_width(s);
  p.nchunks = (int)((N + tmax - 1) / tmax);
  // balance the chunks: the narrowest multiple of 16 that still needs only nchunks tiles
  const int64_t per = (N + p.nchunks - 1) / p.nchunks;
  p.tn = (int)std::min<int64_t>(tmax, std::max<int64_t>(16, (per + 15) / 16 * 16));
  p.kchunks = (int)((K + KC - 1) / KC);
  const int64_t npad = (int64_t)p.nchunks * p.tn;
  // one workspace per call context, reused by every preparation: planes, then Fmax, then the
  // per-K-chunk partial maxima (calls are ordered on the context's stream)
  const size_t plane_bytes = ((size_t)p.nchunks * p.kchunks * s * p.tn * KC * 2 + 255) / 256 * 256;
  const size_t fmax_bytes = ((size_t)npad * sizeof(int) + 255) / 256 * 256;
  const size_t need = plane_bytes + fmax_bytes + (size_t)p.kchunks * npad * sizeof(int);
  unsigned char* base = nullptr;
  if (keep) {
    // planes kept for a later call on the same operand (an allocation of the call context)
    void* mem = nullptr;
    TTR_CHECK(c.alloc(&mem, need));
    base = static_cast<unsigned char*>(mem);
  } else {
    if (c.bprep_bytes < need) {
      void* ws = nullptr;
      TTR_CHECK(c.alloc(&ws, std::max(need, (size_t)2 * c.bprep_bytes)));
      c.bprep = ws;
      c.bprep_bytes = std::max(need, (size_t)2 * c.bprep_bytes);
    }
    base = static_cast<unsigned char*>(c.bprep);
  }
  p.planes = reinterpret_cast<uint4*>(base);
  p.Fmax = reinterpret_cast<int*>(base + plane_bytes);
  int* Fpart = reinterpret_cast<int*>(base + plane_bytes + fmax_bytes);
  const int64_t ctas = (int64_t)p.nchunks * p.kchunks;
  int nsm = 0;
  {
    int dev = 0;
    TTR_CUDA(cudaGetDevice(&dev));
    TTR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  if (ctas <= (int64_t)nsm) {
    // one cooperative launch (all CTAs co-resident: one per SM at most)
    TTR_CHECK(ensure_err(c));
    if (!c.prep_bar) {
      TTR_CHECK(c.alloc_t(&c.prep_bar, 4));
      TTR_CUDA(cudaMemsetAsync(c.prep_bar, 0, 4 * sizeof(unsigned), c.stream));
    }
    int kchunks = p.kchunks;
    int tn = p.tn;
    int sl = s;
    int* fmax = p.Fmax;
    uint4* planes = p.planes;
    unsigned* bar = c.prep_bar;
    int* err = c.d_flags;
    void* params[] = {(void*)&B, (void*)&sbk, (void*)&sbn, (void*)&K, (void*)&N, (void*)&sl, (void*)&tn,
                      (void*)&kchunks, (void*)&npad, (void*)&Fpart, (void*)&fmax, (void*)&planes, (void*)&bar,
                      (void*)&err};
    TTR_CUDA(cudaLaunchCooperativeKernel((const void*)prep_b_fused_kernel, dim3((unsigned)p.nchunks, (unsigned)p.kchunks),
                                         dim3(256), params, 0, c.stream));
    TTR_CHECK(c.check_launch("prep_b"));
  } else {
    TTR_CUDA(cudaMemsetAsync(p.Fmax, 0, sizeof(int) * (size_t)npad, c.stream));
    colmax_b_kernel<<<dim3((unsigned)p.nchunks, (unsigned)std::min(p.kchunks, 128)), 256, 0, c.stream>>>(
        B, sbk, sbn, K, N, p.tn, p.Fmax);
    TTR_CHECK(c.check_launch("colmax_b"));
    slice_b_kernel<<<dim3((unsigned)p.nchunks, (unsigned)p.kchunks), 256, 0, c.stream>>>(
        B, sbk, sbn, K, N, s, p.tn, p.kchunks, p.Fmax, p.planes);
    TTR_CHECK(c.check_launch("slice_b"));
  }
  if (keep) {
    keep->planes = p.planes;
    keep->Fmax = p.Fmax;
    keep->nchunks = p.nchunks;
    keep->kchunks = p.kchunks;
    keep->tn = p.tn;
    keep->s = s;
    keep->src = B;
    keep->ld = sbk;
    keep->K = K;
    keep->N = N;
  }
  return TTR_OK;
}

static int prep_b_float(Ctx& c, const double* B, int64_t sbk, int64_t sbn, int64_t K, int64_t N, int s, BPrep& p) {
  const int tmax = tile_width(s);
  p.nchunks = (int)((N + tmax - 1) / tmax);
  const int64_t per = (N + p.nchunks - 1) / p.nchunks;
  p.tn = (int)std::min<int64_t>(tmax, std::max<int64_t>(16, (per + 15) / 16 * 16));
  p.kchunks = (int)((K + KC - 1) / KC);
  const size_t need = ((size_t)p.nchunks * p.kchunks * s * p.tn * KC * 2 + 255) / 256 * 256;
  if (c.bprep_bytes < need) {
    void* ws = nullptr;
    TTR_CHECK(c.alloc(&ws, std::max(need, (size_t)2 * c.bprep_bytes)));
    c.bprep = ws;
    c.bprep_bytes = std::max(need, (size_t)2 * c.bprep_bytes);
  }
  p.planes = static_cast<uint4*>(c.bprep);
  p.Fmax = nullptr;
  slice_b_float_kernel<<<dim3((unsigned)p.nchunks, (unsigned)p.kchunks), 256, 0, c.stream>>>(B, sbk, sbn, K, N, s, p.tn,
                                                                                             p.kchunks, p.planes);
  return c.check_launch("prep_b_float");
}

// K per CTA for `tiles` output tiles: the fewest K-chunks per CTA that keep the grid within one
// wave (one CTA per SM: the shared memory and TMEM of a CTA fill an SM), at most KSEG.
// K per CTA: the fewest 32-deep chunks per CTA with which the tiles' K segments fit in one wave of
// the SMs the call is sized for (all of them, or its share ttr_options::max_sms when several calls
// share the GPU: fewer, longer CTAs then spend less SM time on the per-CTA exponent scans, TMEM
// set-up and the atomic epilogues of partial results).
static int kseg_for(const Ctx& c, int64_t tiles, int64_t K) {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (c.sm_share > 0 && c.sm_share < nsm) nsm = c.sm_share;
  const int64_t kch = (K + KC - 1) / KC;
  for (int cp = 1; cp < KSEG / KC; ++cp)
    if (cp >= kch || tiles * ((kch + cp - 1) / cp) <= nsm) return cp * KC;
  return KSEG;
}


// ---- tile-shape autotuner.  The tensor-core launches have three free parameters that change the
// work split but not the product's error bound: the widest tile (UMMA N) the B digit planes are cut
// for, the K per CTA (K-split CTAs add their partial results atomically in FP64, as the default
// split does), and, for the partial contractions, the mode slabs per 128-row tile.  With
// ttr_options::autotune set, the first call of each shape (kind of launch, slices, M, K, N, n_k, SM share)
// times every candidate on its stream (each run twice, the second timed between two events, the
// whole call: B preparation and product) and keeps the fastest for the rest of the process; every
// later call of that shape, tuned or not, uses the table.
struct TuneKey {
  int kind, s;
  int64_t M, K, N, n;
  int share = 0;   // the call's SM share (Ctx::sm_share): the default split and candidates depend on it
  bool operator<(const TuneKey& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (s != o.s) return s < o.s;
    if (share != o.share) return share < o.share;
    if (M != o.M) return M < o.M;
    if (K != o.K) return K < o.K;
    if (N != o.N) return N < o.N;
    return n < o.n;
  }
};
struct TuneVal {
  int tmax;   // widest tile the B planes are cut for (0: tile_width(s))
  int kseg;   // K per CTA (a multiple of KC, at most KSEG)
  int g;      // mode slabs per tile (partial contractions; 0 elsewhere)
};
enum TuneKind { TK_GEMM_TN = 0, TK_ROWMAJOR, TK_PROJECT, TK_RL };

static std::mutex tune_mu;
static std::map<TuneKey, TuneVal>& tune_table() {
  static std::map<TuneKey, TuneVal> t;
  return t;
}

// K-per-CTA candidates: the default first, then every power-of-two number of chunks up to KSEG
static std::vector<int> kseg_candidates(int dflt, int64_t K) {
  std::vector<int> v{dflt};
  for (int k = KC; k <= KSEG; k *= 2)
    if (k != dflt && (k < K || k == KC)) v.push_back(k);
  return v;
}

// Shapes share a table entry by bucket: 128-row tiles and K rounded up to powers of two, N to a
// multiple of 16 (the host-driven block loop grows its products by a few columns per block).
static int64_t pow2_at_least(int64_t x) {
  int64_t b = 1;
  while (b < x) b <<= 1;
  return b;
}
static TuneKey bucketed(const TuneKey& k) {
  TuneKey b = k;
  b.M = pow2_at_least((k.M + TM - 1) / TM);
  b.K = pow2_at_least(k.K);
  b.N = (k.N + 15) / 16;
  return b;
}

// the configuration for `key_exact`: from the table (by bucket), else (autotune) the fastest of
// `cands` measured with `run`, else cands[0]
template <class F>
static int tuned(Ctx& c, const TuneKey& key_exact, const std::vector<TuneVal>& cands, F run, TuneVal& out) {
  TuneKey key = bucketed(key_exact);
  key.share = c.sm_share;
  {
    std::lock_guard<std::mutex> lock(tune_mu);
    auto it = tune_table().find(key);
    if (it != tune_table().end()) {
      out = it->second;
      return TTR_OK;
    }
  }
  out = cands[0];
  if (!c.autotune || cands.size() < 2) return TTR_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TTR_CUDA(cudaEventCreate(&e0));
  TTR_CUDA(cudaEventCreate(&e1));
  float best = 3.0e38f;
  int st = TTR_OK;
  for (const TuneVal& v : cands) {
    if ((st = run(v)) != TTR_OK) break;
    cudaEventRecord(e0, c.stream);
    if ((st = run(v)) != TTR_OK) break;
    cudaEventRecord(e1, c.stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = (set_error("autotune: event wait failed"), TTR_ERR_CUDA);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      out = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TTR_OK) return st;
  std::lock_guard<std::mutex> lock(tune_mu);
  tune_table().emplace(key, out);
  return TTR_OK;
}

// Zero the a x b region C(i, j) = C[i*scm + j*scn] where one of the strides is 1.
static int zero_region(Ctx& c, double* C, int64_t a, int64_t b, int64_t scm, int64_t scn) {
  if (scn == 1) {
    TTR_CUDA(cudaMemset2DAsync(C, scm * sizeof(double), 0, b * sizeof(double), a, c.stream));
  } else {
    TTR_CUDA(cudaMemset2DAsync(C, scn * sizeof(double), 0, a * sizeof(double), b, c.stream));
  }
  return TTR_OK;
}

}  // namespace tc

using namespace tc;

// candidates of a plain product (M rows in 128-row tiles, K, N columns): the default split first,
// then the other K splits, then half-width tiles (two column chunks) with their default split
static void add_plain_candidates(const Ctx& c, std::vector<TuneVal>& cands, int s, int64_t M, int64_t K, int64_t N) {
  const int tw = tile_width(s);
  auto tiles_for = [&](int tmax) {
    const int64_t nch = (N + tmax - 1) / tmax;
    return (M + TM - 1) / TM * nch;
  };
  const int kd = kseg_for(c, tiles_for(tw), K);
  for (int k : kseg_candidates(kd, K)) cands.push_back({tw, k, 0});
  if (N > 32) {
    const int half = (int)std::min<int64_t>(tw, std::max<int64_t>(16, ((N + 1) / 2 + 15) / 16 * 16));
    if (half < tw) cands.push_back({half, kseg_for(c, tiles_for(half), K), 0});
  }
}

// Widest UMMA N whose s per-diagonal accumulators fit the 512 TMEM columns.
int tile_width(int s) {
  const int tn = (512 / s) / 16 * 16;
  return tn > TNMAX ? TNMAX : tn;
}

// C(i, j) = sum_r X(r, i) Y(r, j) (i < a, j < b) stored at C[i*scm + j*scn]; X, Y row-major m x a, m x b.
// The big operand X^T is read column-major; the row dimension m is split over CTAs in segments
// of 256 and partial results are added atomically.
int tc_gemm_tn(Ctx& c, int slices, const double* X, int64_t ldx, int64_t m, int64_t a_cols, const double* Y, int64_t ldy,
               int64_t b_cols, double* C, int64_t scm, int64_t scn) {
  if (slices < 3 || slices > MAXS || m <= 0 || a_cols <= 0 || b_cols <= 0) return TTR_ERR_UNSUPPORTED;
  if (scm != 1 && scn != 1) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  auto run = [&](const TuneVal& v) -> int {
    BPrep bp;
    TTR_CHECK(prep_b(c, Y, ldy, 1, m, b_cols, slices, bp, nullptr, v.tmax));
    Args a{};
    a.A = X; a.M = a_cols; a.K = m; a.sam = 1; a.sak = ldx;
    a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = b_cols; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
    a.C = C; a.scm = scm; a.scn = scn; a.err = c.d_flags;
    a.kseg = v.kseg;
    const unsigned ksplit = (unsigned)((m + a.kseg - 1) / a.kseg);
    dim3 grid((unsigned)((a_cols + TM - 1) / TM), (unsigned)bp.nchunks, ksplit);
    if (ksplit > 1) {
      TTR_CHECK(zero_region(c, C, a_cols, b_cols, scm, scn));
      return launch<ATOMIC, false>(c, a, grid, "tc_gemm_tn");
    }
    return launch<PLAIN, false>(c, a, grid, "tc_gemm_tn");
  };
  std::vector<TuneVal> cands;
  add_plain_candidates(c, cands, slices, a_cols, m, b_cols);
  TuneVal v;
  TTR_CHECK(tuned(c, TuneKey{TK_GEMM_TN, slices, a_cols, m, b_cols, 0}, cands, run, v));
  return run(v);
}

int tc_rl_step(Ctx& c, int slices, const double* Xk, int64_t r0, int64_t n, int64_t r1, const double* Wn, int64_t ldw,
               const int* Omi, int64_t ldoi, int64_t w, double* Wout, int64_t ldwo, BPlanes* keep) {
  if (n > TM || slices < 3 || slices > MAXS || !Omi) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  // timed: the library's kernel events around the contraction launch (not the B preparation)
  auto run_with = [&](const TuneVal& v, BPlanes* kp, bool timed) -> int {
    BPrep bp;
    TTR_CHECK(prep_b(c, Wn, ldw, 1, r1, w, slices, bp, kp, v.tmax));
    Args a{};
    a.A = Xk; a.M = r0 * n; a.K = r1; a.sam = r1; a.sak = 1;
    a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = w; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
    a.Omint = Omi; a.ldo = ldoi; a.nmode = n; a.g = v.g; a.slabs = r0; a.W = Wout; a.ldw = ldwo;
    a.err = c.d_flags;
    a.kseg = v.kseg;
    const unsigned ksplit = (unsigned)((r1 + a.kseg - 1) / a.kseg);
    if (ksplit > 1) {
      a.watomic = 1;
      TTR_CUDA(cudaMemset2DAsync(Wout, ldwo * sizeof(double), 0, w * sizeof(double), r0, c.stream));
    }
    dim3 grid((unsigned)((r0 + a.g - 1) / a.g), (unsigned)bp.nchunks, ksplit);
    if (timed) c.time_begin(Ctx::KT_RL);
    TTR_CHECK((launch<RLM, true>(c, a, grid, "tc_rl_step")));
    if (timed) c.time_end(8.0 * ((double)r0 * n * r1 + (double)r1 * w + (double)r0 * w));
    return TTR_OK;
  };
  // candidates: the default (all slabs of a 128-row tile, the split that fills one wave), the other
  // K splits, and tiles of half as many slabs
  const int tw = tile_width(slices);
  const int g0 = (int)(TM / n);
  const int64_t nch = (w + tw - 1) / tw;
  std::vector<TuneVal> cands;
  const int kd = kseg_for(c, (r0 + g0 - 1) / g0 * nch, r1);
  for (int k : kseg_candidates(kd, r1)) cands.push_back({tw, k, g0});
  if (g0 >= 2) {
    const int g1 = g0 / 2;
    cands.push_back({tw, kseg_for(c, (r0 + g1 - 1) / g1 * nch, r1), g1});
  }
  TuneVal v;
  TTR_CHECK(tuned(c, TuneKey{TK_RL, slices, r0, r1, w, n}, cands,
                  [&](const TuneVal& t) { return run_with(t, nullptr, false); }, v));
  return run_with(v, keep, true);
}

int tc_rl_step_grouped(Ctx& c, int slices, int ng, const double* const* Xk, const int64_t* r0, int64_t n,
                       const int64_t* r1, const double* Wn, int64_t ldw, int64_t Kall, const int64_t* off_n,
                       const int* Omi, int64_t ldoi, int64_t w, double* Wout, int64_t ldwo, const int64_t* off_out,
                       BPlanes* keep) {
  if (ng < 1 || ng > MAXG || n > TM || slices < 3 || slices > MAXS || !Omi) return TTR_ERR_UNSUPPORTED;
  for (int g = 0; g < ng; ++g)   // one K segment per group, inside the stacked rows
    if (r1[g] < 1 || r0[g] < 1 || off_n[g] % KC + r1[g] > KSEG || off_n[g] + r1[g] > Kall) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  BPrep bp;
  TTR_CHECK(prep_b(c, Wn, ldw, 1, Kall, w, slices, bp, keep));   // the whole stacked W_{k+1}
  Args a{};
  a.sak = 1;
  a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = w; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
  a.Omint = Omi; a.ldo = ldoi; a.nmode = n; a.g = (int)(TM / n); a.ldw = ldwo;
  a.err = c.d_flags;
  a.kseg = KSEG;
  Groups gr{};
  gr.n = ng;
  int tiles = 0;
  double bytes = 0.0;
  for (int g = 0; g < ng; ++g) {
    gr.tile0[g] = tiles;
    gr.A[g] = Xk[g]; gr.M[g] = r0[g] * n; gr.K[g] = r1[g]; gr.sam[g] = r1[g]; gr.sak[g] = 1;
    gr.slabs[g] = r0[g]; gr.koff[g] = off_n[g]; gr.W[g] = Wout + off_out[g] * ldwo;
    tiles += (int)((r0[g] + a.g - 1) / a.g);
    bytes += 8.0 * ((double)r0[g] * n * r1[g] + (double)r1[g] * w + (double)r0[g] * w);
  }
  gr.tile0[ng] = tiles;
  dim3 grid((unsigned)tiles, (unsigned)bp.nchunks, 1);
  c.time_begin(Ctx::KT_RL);
  TTR_CHECK((launch<RLM, true>(c, a, grid, "tc_rl_step", &gr)));
  c.time_end(bytes);
  return TTR_OK;
}

int tc_gemm_rowmajor(Ctx& c, int slices, const double* A, int64_t lda, int64_t M, int64_t K, const double* B,
                     int64_t ldb, int64_t N, double* C, int64_t ldc, const BPlanes* reuse) {
  if (slices < 3 || slices > MAXS || M <= 0 || N <= 0 || K <= 0) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  const bool reused = reuse && reuse->planes && reuse->src == B && reuse->ld == ldb && reuse->K == K &&
                      reuse->N == N && reuse->s == slices;
  auto run = [&](const TuneVal& v) -> int {
    BPrep bp;
    if (reused) {
      bp.planes = reuse->planes;                 // the digit planes of this operand are already made
      bp.Fmax = reuse->Fmax;
      bp.nchunks = reuse->nchunks;
      bp.kchunks = reuse->kchunks;
      bp.tn = reuse->tn;
    } else {
      TTR_CHECK(prep_b(c, B, ldb, 1, K, N, slices, bp, nullptr, v.tmax));
    }
    Args a{};
    a.A = A; a.M = M; a.K = K; a.sam = lda; a.sak = 1;
    a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = N; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
    a.C = C; a.scm = ldc; a.scn = 1; a.err = c.d_flags;
    a.kseg = v.kseg;
    const unsigned ksplit = (unsigned)((K + a.kseg - 1) / a.kseg);
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)bp.nchunks, ksplit);
    if (ksplit > 1) {
      TTR_CUDA(cudaMemset2DAsync(C, ldc * sizeof(double), 0, N * sizeof(double), M, c.stream));
      return launch<ATOMIC, true>(c, a, grid, "tc_sketch");
    }
    return launch<PLAIN, true>(c, a, grid, "tc_sketch");
  };
  std::vector<TuneVal> cands;
  if (reused) {
    // the planes fix the tile width: only the K split is free
    const int64_t tiles = (M + TM - 1) / TM * reuse->nchunks;
    for (int k : kseg_candidates(kseg_for(c, tiles, K), K)) cands.push_back({reuse->tn, k, 0});
  } else {
    add_plain_candidates(c, cands, slices, M, K, N);
  }
  TuneVal v;
  TTR_CHECK(tuned(c, TuneKey{TK_ROWMAJOR, slices, M, K, N, reused ? reuse->tn : 0}, cands, run, v));
  return run(v);
}

// Y = Mk (L x K, row-major ldm) @ H(X_{k+1}) (K x ncol, row-major), computed as
// Y^T = H(X_{k+1})^T Mk^T so that the big operand is the M side (column-major).
int tc_project(Ctx& c, int slices, const double* Mk, int64_t ldm, int64_t L, int64_t K, const double* Xn, int64_t ncol,
               double* Y) {
  if (slices < 3 || slices > MAXS || L <= 0 || ncol <= 0 || K <= 0) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  auto run = [&](const TuneVal& v) -> int {
    BPrep bp;
    TTR_CHECK(prep_b(c, Mk, 1, ldm, K, L, slices, bp, nullptr, v.tmax));
    Args a{};
    a.A = Xn; a.M = ncol; a.K = K; a.sam = 1; a.sak = ncol;
    a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = L; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
    a.C = Y; a.scm = 1; a.scn = ncol; a.err = c.d_flags;
    a.kseg = v.kseg;
    const unsigned ksplit = (unsigned)((K + a.kseg - 1) / a.kseg);
    dim3 grid((unsigned)((ncol + TM - 1) / TM), (unsigned)bp.nchunks, ksplit);
    if (ksplit > 1) {
      TTR_CUDA(cudaMemsetAsync(Y, 0, (size_t)L * ncol * sizeof(double), c.stream));
      return launch<ATOMIC, false>(c, a, grid, "tc_project");
    }
    return launch<PLAIN, false>(c, a, grid, "tc_project");
  };
  std::vector<TuneVal> cands;
  add_plain_candidates(c, cands, slices, ncol, K, L);
  TuneVal v;
  TTR_CHECK(tuned(c, TuneKey{TK_PROJECT, slices, ncol, K, L, 0}, cands, run, v));
  return run(v);
}

// C_g = A_g B for up to MAXG row-major A_g (M[g] x K, leading dimension lda[g]) sharing one row-major
// B (K x N, leading dimension ldb), in one launch: C_g row-major with leading dimension ldc.
int tc_gemm_shared_b(Ctx& c, int slices, int ng, const double* const* A, const int64_t* M, const int64_t* lda,
                     int64_t K, const double* B, int64_t ldb, int64_t N, double* const* C, int64_t ldc) {
  if (ng < 1 || ng > MAXG || slices < 3 || slices > MAXS || K < 1 || K > KSEG || N <= 0) return TTR_ERR_UNSUPPORTED;
  for (int g = 0; g < ng; ++g)
    if (M[g] < 1) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  BPrep bp;
  TTR_CHECK(prep_b(c, B, ldb, 1, K, N, slices, bp));
  Args a{};
  a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = N; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
  a.err = c.d_flags; a.kseg = KSEG;
  Groups gr{};
  gr.n = ng;
  int tiles = 0;
  for (int g = 0; g < ng; ++g) {
    gr.tile0[g] = tiles;
    gr.A[g] = A[g]; gr.M[g] = M[g]; gr.K[g] = K; gr.sam[g] = lda[g]; gr.sak[g] = 1;
    gr.koff[g] = 0; gr.C[g] = C[g]; gr.scm[g] = ldc; gr.scn[g] = 1;
    tiles += (int)((M[g] + TM - 1) / TM);
  }
  gr.tile0[ng] = tiles;
  dim3 grid((unsigned)tiles, (unsigned)bp.nchunks, 1);
  return launch<PLAIN, true>(c, a, grid, "tc_gemm_shared_b", &gr);
}

// Y^(g) = M(:, koff[g] : koff[g] + K[g]) H(X^(g)) for up to MAXG summands in one launch (the per-summand
// projection of a sum of TTs): summand g's result, L x (n_{k+1} rn[g]) with columns (i, c), is written
// to rows a, columns i * rstride + yoff[g] + c of Y (row length ldy).  M is L x Kall row-major
// (leading dimension ldm); H(X^(g)) is K[g] x ncol[g] row-major.
int tc_project_grouped(Ctx& c, int slices, int ng, const double* M, int64_t ldm, int64_t L, int64_t Kall,
                       const int64_t* koff, const int64_t* K, const double* const* Xn, const int64_t* ncol,
                       const int64_t* rn, double* Y, int64_t ldy, int64_t rstride, const int64_t* yoff) {
  if (ng < 1 || ng > MAXG || slices < 3 || slices > MAXS || L <= 0) return TTR_ERR_UNSUPPORTED;
  for (int g = 0; g < ng; ++g)
    if (K[g] < 1 || koff[g] % KC + K[g] > KSEG || koff[g] + K[g] > Kall || ncol[g] < 1 || rn[g] < 1 ||
        ncol[g] >= (int64_t)1 << 31)
      return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  BPrep bp;
  TTR_CHECK(prep_b(c, M, 1, ldm, Kall, L, slices, bp));   // B(k, j) = M(j, k), all Kall columns of M
  Args a{};
  a.Bp = bp.planes; a.Fmax = bp.Fmax; a.N = L; a.kchunks = bp.kchunks; a.s = slices; a.tn = bp.tn;
  a.err = c.d_flags; a.kseg = KSEG; a.rstride = rstride;
  Groups gr{};
  gr.n = ng;
  int tiles = 0;
  for (int g = 0; g < ng; ++g) {
    gr.tile0[g] = tiles;
    gr.A[g] = Xn[g]; gr.M[g] = ncol[g]; gr.K[g] = K[g]; gr.sam[g] = 1; gr.sak[g] = ncol[g];
    gr.koff[g] = koff[g]; gr.C[g] = Y + yoff[g]; gr.scm[g] = 1; gr.scn[g] = ldy; gr.rp[g] = rn[g];
    tiles += (int)((ncol[g] + TM - 1) / TM);
  }
  gr.tile0[ng] = tiles;
  dim3 grid((unsigned)tiles, (unsigned)bp.nchunks, 1);
  return launch<PLAIN, false>(c, a, grid, "tc_project", &gr);
}

// ---- reduced-precision sketch forms (TF32 / BF16 operands, FP32 accumulation): fs = 2 or 1 planes

int tc_rl_step_flt(Ctx& c, int fs, const double* Xk, int64_t r0, int64_t n, int64_t r1, const double* Wn, int64_t ldw,
                   const double* Om, int64_t ldo, int64_t w, double* Wout, int64_t ldwo) {
  if (n > TM || (fs != 1 && fs != 2) || !Om) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  BPrep bp;
  TTR_CHECK(prep_b_float(c, Wn, ldw, 1, r1, w, fs, bp));
  Args a{};
  a.A = Xk; a.M = r0 * n; a.K = r1; a.sam = r1; a.sak = 1;
  a.Bp = bp.planes; a.Fmax = nullptr; a.N = w; a.kchunks = bp.kchunks; a.s = fs; a.tn = bp.tn;
  a.Omd = Om; a.ldo = ldo; a.nmode = n; a.g = (int)(TM / n); a.slabs = r0; a.W = Wout; a.ldw = ldwo;
  a.err = c.d_flags; a.flt = 1;
  const int64_t tiles = (r0 + a.g - 1) / a.g * bp.nchunks;
  a.kseg = kseg_for(c, tiles, r1);
  const unsigned ksplit = (unsigned)((r1 + a.kseg - 1) / a.kseg);
  if (ksplit > 1) {
    a.watomic = 1;
    TTR_CUDA(cudaMemset2DAsync(Wout, ldwo * sizeof(double), 0, w * sizeof(double), r0, c.stream));
  }
  dim3 grid((unsigned)((r0 + a.g - 1) / a.g), (unsigned)bp.nchunks, ksplit);
  c.time_begin(Ctx::KT_RL);
  TTR_CHECK((launch<RLM, true>(c, a, grid, "tc_rl_step_flt")));
  c.time_end(8.0 * ((double)r0 * n * r1 + (double)r1 * w + (double)r0 * w));
  return TTR_OK;
}

int tc_gemm_rowmajor_flt(Ctx& c, int fs, const double* A, int64_t lda, int64_t M, int64_t K, const double* B,
                         int64_t ldb, int64_t N, double* C, int64_t ldc) {
  if ((fs != 1 && fs != 2) || M <= 0 || N <= 0 || K <= 0) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(ensure_err(c));
  BPrep bp;
  TTR_CHECK(prep_b_float(c, B, ldb, 1, K, N, fs, bp));
  Args a{};
  a.A = A; a.M = M; a.K = K; a.sam = lda; a.sak = 1;
  a.Bp = bp.planes; a.Fmax = nullptr; a.N = N; a.kchunks = bp.kchunks; a.s = fs; a.tn = bp.tn;
  a.C = C; a.scm = ldc; a.scn = 1; a.err = c.d_flags; a.flt = 1;
  const int64_t tiles = (M + TM - 1) / TM * bp.nchunks;
  a.kseg = kseg_for(c, tiles, K);
  const unsigned ksplit = (unsigned)((K + a.kseg - 1) / a.kseg);
  dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)bp.nchunks, ksplit);
  if (ksplit > 1) {
    TTR_CUDA(cudaMemset2DAsync(C, ldc * sizeof(double), 0, N * sizeof(double), M, c.stream));
    return launch<ATOMIC, true>(c, a, grid, "tc_sketch_flt");
  }
  return launch<PLAIN, true>(c, a, grid, "tc_sketch_flt");
}

}  // namespace ttr
