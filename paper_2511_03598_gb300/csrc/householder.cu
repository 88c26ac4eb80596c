// Householder QR of a tall m x b row-major matrix (m >= b) as two persistent cooperative kernels,
// for the deterministic TT-rounding (Algorithm 1), whose unfoldings of a formal sum are exactly
// rank-deficient: Householder reflections stay backward stable there (A = Q R + E with
// ||E|| = O(u ||A||)), which CholeskyQR does not.
//
//   factor:  for j = 0..b-1: a = A(j:, j); alpha = -sign(a_j) ||a||; v = a - alpha e_j;
//            A(j:, j+1:) -= beta v (v^T A(j:, j+1:)), beta = 2 / v^T v = 1 / (||a||^2 - alpha a_j)
//            R(j, j) = alpha; v is kept below the diagonal (v_j in vjj[j]).
//   apply:   Q E = H_0 H_1 ... H_{b-1} [E; 0] for a b x nq matrix E, accumulated backwards.
//
// Every CTA owns a contiguous block of rows.  Each step needs one cross-CTA reduction: for the
// factorization the dot products x_l = A(j:, j)^T A(j:, l) (l >= j, x_j = ||a||^2) together with
// row j itself, for the accumulation y = v^T Q(j:, :).  Partials go by FP64 atomics into one of
// three rotating buffers; after the barrier that completes step j every CTA reads buffer j % 3 and
// CTA 0 clears buffer (j + 2) % 3, which no CTA touches before the next barrier: one barrier per
// column.  The barrier is a counter/generation pair with a bounded spin (the error flag is set and
// the kernel returns when it runs out).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "engine.cuh"

namespace ttr {
namespace hh {

constexpr int NT = 256;
constexpr long long BAR_CYCLES = 4000000000LL;   // ~2 s
constexpr int BMAX = 4096;                       // widest matrix (columns staged in shared memory)

__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    ok_s = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
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
        __nanosleep(32);
      }
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

struct Args {
  double* A;        // m x b, row-major (overwritten: R above the diagonal, v below)
  int64_t lda;
  int64_t m;
  int b;
  double* vjj;      // b: v_j(j)
  double* beta;     // b: 2 / v_j^T v_j (0 for a zero column)
  // apply only
  const double* E;  // b x nq (ld lde)
  int64_t lde;
  int nq;
  double* Q;        // m x nq (ld ldq)
  int64_t ldq;
  // reductions
  double* buf;      // 3 x used doubles, zero on entry
  int used;
  unsigned* bar;
  int* err;
};

// Own rows live in dynamic shared memory when they fit (stage = 1), else they are used in place.
__global__ void __launch_bounds__(NT) factor_kernel(Args a, int stage) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double cs[BMAX];
  int64_t lo, hi;
  my_rows(a.m, lo, hi);
  const int b = a.b;
  double* Ar = stage ? sm : a.A + lo * a.lda;   // own rows: row i at Ar[(i - lo) * ldr]
  const int64_t ldr = stage ? b : a.lda;
  if (stage) {
    for (int64_t e = threadIdx.x; e < (hi - lo) * b; e += NT) sm[e] = a.A[(lo + e / b) * a.lda + e % b];
    __syncthreads();
  }
  int ri = 0;   // index of the next reduction
  auto bufp = [&](int i) { return a.buf + (int64_t)(i % 3) * a.used; };
  // partials of step j: x_t = sum_{i >= j, own rows} A(i, j) A(i, j + t), and row j (its owner)
  auto accumulate = [&](int j) {
    double* x = bufp(ri);
    double* row = x + b;
    const int nc = b - j;
    const int64_t r0 = max(lo, (int64_t)j) - lo, r1 = hi - lo;
    for (int t = threadIdx.x; t < nc; t += NT) {
      const int l = j + t;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int64_t i = r0;
      for (; i + 3 < r1; i += 4) {
        s0 = fma(Ar[i * ldr + j], Ar[i * ldr + l], s0);
        s1 = fma(Ar[(i + 1) * ldr + j], Ar[(i + 1) * ldr + l], s1);
        s2 = fma(Ar[(i + 2) * ldr + j], Ar[(i + 2) * ldr + l], s2);
        s3 = fma(Ar[(i + 3) * ldr + j], Ar[(i + 3) * ldr + l], s3);
      }
      for (; i < r1; ++i) s0 = fma(Ar[i * ldr + j], Ar[i * ldr + l], s0);
      const double s = (s0 + s1) + (s2 + s3);
      if (s != 0.0) atomicAdd(x + t, s);
      if (j >= lo && j < hi) row[t] = Ar[(j - lo) * ldr + l];
    }
  };
  accumulate(0);
  bool ok = true;
  for (int j = 0; j < b; ++j) {
    const double* x = bufp(ri);
    if (!grid_sync(a.bar, a.err)) {
      ok = false;
      break;
    }
    if (blockIdx.x == 0) {   // clear the buffer two reductions ahead
      double* z = bufp(ri + 2);
      for (int o = threadIdx.x; o < a.used; o += NT) z[o] = 0.0;
    }
    ++ri;
    const double* row = x + b;
    const int nc = b - j;
    const double nrm2 = __ldcg(x);
    const double ajj = __ldcg(row);
    double alpha = 0.0, vj = 0.0, beta = 0.0;
    if (nrm2 > 0.0) {
      const double nrm = sqrt(nrm2);
      alpha = ajj >= 0.0 ? -nrm : nrm;
      vj = ajj - alpha;
      beta = 1.0 / (nrm2 - alpha * ajj);   // 2 / v^T v, v^T v = 2 (||a||^2 + |a_j| ||a||)
    }
    for (int t = 1 + threadIdx.x; t < nc; t += NT) cs[t] = beta * (__ldcg(x + t) - alpha * __ldcg(row + t));
    __syncthreads();
    if (beta != 0.0) {
      for (int64_t i = max(lo, (int64_t)j) - lo; i < hi - lo; ++i) {
        const double vi = (i + lo == j) ? vj : Ar[i * ldr + j];
        for (int t = 1 + threadIdx.x; t < nc; t += NT) Ar[i * ldr + j + t] -= vi * cs[t];
      }
    }
    __syncthreads();
    if (j >= lo && j < hi && threadIdx.x == 0) Ar[(j - lo) * ldr + j] = alpha;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.vjj[j] = vj;
      a.beta[j] = beta;
    }
    __syncthreads();
    if (j + 1 < b) accumulate(j + 1);
  }
  if (stage) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (hi - lo) * b; e += NT) a.A[(lo + e / b) * a.lda + e % b] = sm[e];
  }
  (void)ok;
}

__global__ void __launch_bounds__(NT) apply_kernel(Args a, int stage) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double ys[BMAX];
  int64_t lo, hi;
  my_rows(a.m, lo, hi);
  const int b = a.b, nq = a.nq;
  const double* A = a.A;
  const int64_t lda = a.lda;
  double* Qr = stage ? sm : a.Q + lo * a.ldq;    // own rows of Q E
  const int64_t ldr = stage ? nq : a.ldq;
  // Q E = [E; 0] before the reflections
  for (int64_t i = 0; i < hi - lo; ++i)
    for (int t = threadIdx.x; t < nq; t += NT) Qr[i * ldr + t] = (lo + i < b) ? a.E[(lo + i) * a.lde + t] : 0.0;
  __syncthreads();
  int ri = 0;
  auto bufp = [&](int i) { return a.buf + (int64_t)(i % 3) * a.used; };
  // partials of y = v_j^T (Q E)(j:, :)
  auto accumulate = [&](int j) {
    double* y = bufp(ri);
    const double vj = __ldcg(a.vjj + j);
    const int64_t r0 = max(lo, (int64_t)j);
    for (int t = threadIdx.x; t < nq; t += NT) {
      double s0 = 0.0, s1 = 0.0;
      int64_t i = r0;
      for (; i + 1 < hi; i += 2) {
        s0 = fma((i == j) ? vj : __ldg(A + i * lda + j), Qr[(i - lo) * ldr + t], s0);
        s1 = fma(__ldg(A + (i + 1) * lda + j), Qr[(i + 1 - lo) * ldr + t], s1);
      }
      if (i < hi) s0 = fma((i == j) ? vj : __ldg(A + i * lda + j), Qr[(i - lo) * ldr + t], s0);
      const double s = s0 + s1;
      if (s != 0.0) atomicAdd(y + t, s);
    }
  };
  accumulate(b - 1);
  for (int j = b - 1; j >= 0; --j) {
    const double* y = bufp(ri);
    if (!grid_sync(a.bar, a.err)) break;
    if (blockIdx.x == 0) {
      double* z = bufp(ri + 2);
      for (int o = threadIdx.x; o < a.used; o += NT) z[o] = 0.0;
    }
    ++ri;
    const double beta = __ldcg(a.beta + j);
    const double vj = __ldcg(a.vjj + j);
    for (int t = threadIdx.x; t < nq; t += NT) ys[t] = beta * __ldcg(y + t);
    __syncthreads();
    if (beta != 0.0) {
      for (int64_t i = max(lo, (int64_t)j); i < hi; ++i) {
        const double vi = (i == j) ? vj : __ldg(A + i * lda + j);
        for (int t = threadIdx.x; t < nq; t += NT) Qr[(i - lo) * ldr + t] -= vi * ys[t];
      }
    }
    __syncthreads();
    if (j > 0) accumulate(j - 1);
  }
  if (stage) {
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (hi - lo) * nq; e += NT) a.Q[(lo + e / nq) * a.ldq + e % nq] = sm[e];
  }
}

// R (b x b, row-major, ld ldr) = the upper triangle of the factored A
__global__ void extract_r_kernel(const double* A, int64_t lda, int b, double* R, int64_t ldr) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)b * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b, l = e % b;
    R[i * ldr + l] = (l >= i) ? A[i * lda + l] : 0.0;
  }
}

struct DevInfo {
  int nsm = 0, coop = 0;
};

static int dev_info(DevInfo& out) {
  constexpr int MAXDEV = 64;
  static DevInfo info[MAXDEV];
  static std::mutex mu;
  int dev = 0;
  TTR_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  DevInfo local;
  DevInfo& di = (dev >= 0 && dev < MAXDEV) ? info[dev] : local;
  if (di.nsm == 0) {
    TTR_CUDA(cudaDeviceGetAttribute(&di.coop, cudaDevAttrCooperativeLaunch, dev));
    TTR_CUDA(cudaDeviceGetAttribute(&di.nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  out = di;
  return TTR_OK;
}

}  // namespace hh

static int hh_work(Ctx& c, HhWork& w, int b, int used) {
  if (!w.bar) {
    TTR_CHECK(c.alloc_t(&w.bar, 4));
    TTR_CUDA(cudaMemsetAsync(w.bar, 0, 4 * sizeof(unsigned), c.stream));
  }
  if (w.cap < used) {
    TTR_CHECK(c.alloc_t(&w.buf, (size_t)3 * used));
    w.cap = used;
  }
  if (w.bcap < b) {
    TTR_CHECK(c.alloc_t(&w.vjj, b));
    TTR_CHECK(c.alloc_t(&w.beta, b));
    w.bcap = b;
  }
  if (!c.d_flags) {
    TTR_CHECK(c.alloc_t(&c.d_flags, 4));
    TTR_CUDA(cudaMemsetAsync(c.d_flags, 0, 4 * sizeof(int), c.stream));
  }
  return TTR_OK;
}

static int hh_launch(Ctx& c, HhWork& w, bool factor, hh::Args& a, int used, const char* what) {
  hh::DevInfo di;
  TTR_CHECK(hh::dev_info(di));
  if (!di.coop) return set_error("householder: cooperative launch unsupported"), TTR_ERR_UNSUPPORTED;
  // one CTA per SM at most and none without rows: all resident at once
  const int nblocks = (int)std::min<int64_t>(di.nsm, a.m);
  const int64_t rpc = (a.m + nblocks - 1) / nblocks;
  const int64_t cols = factor ? a.b : a.nq;
  // own rows in shared memory when they fit next to the 32 KB of static arrays
  const size_t dyn = sizeof(double) * (size_t)rpc * (size_t)cols;
  const size_t limit = 160 * 1024;
  const int stage = dyn <= limit ? 1 : 0;
  const void* kern = factor ? (const void*)hh::factor_kernel : (const void*)hh::apply_kernel;
  if (stage) {
    static std::mutex mu;
    static size_t raised[2] = {0, 0};
    std::lock_guard<std::mutex> lock(mu);
    const int ki = factor ? 0 : 1;
    if (raised[ki] < limit) {   // the limit belongs to the kernel: raise it once to the most it takes
      TTR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
      raised[ki] = limit;
    }
  }
  a.buf = w.buf; a.used = used; a.bar = w.bar; a.err = c.d_flags;
  a.vjj = w.vjj; a.beta = w.beta;
  TTR_CUDA(cudaMemsetAsync(w.buf, 0, sizeof(double) * 3 * (size_t)used, c.stream));
  int st_arg = stage;
  void* params[] = {&a, &st_arg};
  TTR_CUDA(cudaLaunchCooperativeKernel(kern, dim3(nblocks), dim3(hh::NT), params, stage ? dyn : 0, c.stream));
  return c.check_launch(what);
}

int householder_qr(Ctx& c, HhWork& w, double* A, int64_t lda, int64_t m, int64_t b, double* R, int64_t ldr) {
  if (b <= 0) return TTR_OK;
  if (m < b) return set_error("householder_qr: more columns than rows"), TTR_ERR_ARG;
  if (b > hh::BMAX) return set_error("householder_qr: matrix too wide"), TTR_ERR_UNSUPPORTED;
  const int used = (int)((2 * b + 31) / 32 * 32);
  TTR_CHECK(hh_work(c, w, (int)b, used));
  hh::Args a{};
  a.A = A; a.lda = lda; a.m = m; a.b = (int)b;
  TTR_CHECK(hh_launch(c, w, true, a, used, "householder_factor"));
  if (R) {
    const unsigned blocks = (unsigned)std::min<int64_t>((b * b + 255) / 256, 1024);
    hh::extract_r_kernel<<<blocks, 256, 0, c.stream>>>(A, lda, (int)b, R, ldr);
    TTR_CHECK(c.check_launch("householder_r"));
  }
  return TTR_OK;
}

int householder_apply(Ctx& c, HhWork& w, const double* A, int64_t lda, int64_t m, int64_t b, const double* E,
                      int64_t lde, int64_t nq, double* Q, int64_t ldq) {
  if (b <= 0 || nq <= 0) return TTR_OK;
  if (m < b || b > hh::BMAX || nq > hh::BMAX || !E || !Q) return set_error("householder_apply: bad shape"), TTR_ERR_ARG;
  if (w.bcap < b || !w.bar) return set_error("householder_apply: no factorization in this workspace"), TTR_ERR_ARG;
  const int used = (int)((std::max<int64_t>(2 * b, nq) + 31) / 32 * 32);
  TTR_CHECK(hh_work(c, w, (int)b, used));
  hh::Args a{};
  a.A = const_cast<double*>(A); a.lda = lda; a.m = m; a.b = (int)b;
  a.E = E; a.lde = lde; a.nq = (int)nq; a.Q = Q; a.ldq = ldq;
  return hh_launch(c, w, false, a, used, "householder_apply");
}

}  // namespace ttr
