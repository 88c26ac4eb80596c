// One-sided (Hestenes) Jacobi SVD of a b x b matrix spread over many CTAs, for the deterministic
// TT-rounding (Algorithm 1) and the Remark 3.2 pass, whose factors R are 50..800 wide.
//
// On this part a single SM retires about two FP64 FMAs per clock, so the one-CTA Jacobi
// (kernels_fp64.cu) spends ~20 ms per sweep on a 210 x 210 factor.  Here a persistent cooperative
// kernel gives each CTA a share of the b/2 independent column pairs of a round-robin round and
// separates rounds by a grid barrier: b - 1 rounds per sweep, one barrier each.
//
// The columns of A are rotated as the rows of A^T (row j of At = column j of A) and V accumulates
// the same rotations on the rows of Vt, so every pair is two contiguous runs.  A pair is rotated when
// |a_p^T a_q| > 1e-15 ||a_p|| ||a_q||, unless both columns lie below the rounding level b u ||A||_F of
// the factor A came from.  The sweep loop ends after a sweep without rotations (at most 60).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "engine.cuh"
#include "rsqrt.cuh"

namespace ttr {
namespace jc {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr long long BAR_CYCLES = 4000000000LL;   // ~2 s
constexpr int MAX_SWEEPS = 60;

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

struct Args {
  const double* A;   // b x b row-major input (ld)
  int64_t ld;
  int b;
  double* At;        // b x b work (ld b): rows = columns of A; becomes U^T before sorting
  double* Vt;        // b x b work (ld b)
  double* sigma;     // b (unsorted column norms on return)
  unsigned* bar;
  int* err;
  int* flags;        // [0..MAX_SWEEPS): rotations seen in sweep s (zero on entry)
  double* nrm2;      // ||A||_F^2 (zero on entry)
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NW; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(NT) jacobi_kernel(Args a) {
  __shared__ double red[3 * NW];
  __shared__ double rot[2];
  const int b = a.b;
  const int64_t b2 = (b + 1) & ~1;
  const int npairs = (int)(b2 / 2);
  // At = A^T, Vt = I, ||A||_F^2; rows split over the CTAs
  double part = 0.0;
  for (int64_t j = blockIdx.x; j < b; j += gridDim.x)
    for (int i = threadIdx.x; i < b; i += NT) {
      const double v = a.A[(int64_t)i * a.ld + j];
      a.At[j * b + i] = v;
      part = fma(v, v, part);
      a.Vt[j * b + i] = (i == j) ? 1.0 : 0.0;
    }
  part = block_sum(part, red);
  if (threadIdx.x == 0 && part != 0.0) atomicAdd(a.nrm2, part);
  if (!grid_sync(a.bar, a.err)) return;
  const double floor_ = (double)b * 2.220446049250313e-16;
  const double tiny = floor_ * floor_ * __ldcg(a.nrm2);
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    int mine = 0;
    for (int64_t r = 0; r < b2 - 1; ++r) {
      for (int pi = blockIdx.x; pi < npairs; pi += gridDim.x) {
        const int64_t i1 = pi, i2 = b2 - 1 - pi;
        const int64_t p = (i1 == 0) ? 0 : 1 + ((i1 - 1 + r) % (b2 - 1));
        const int64_t q = (i2 == 0) ? 0 : 1 + ((i2 - 1 + r) % (b2 - 1));
        if (p >= b || q >= b) continue;
        double* xp = a.At + p * b;
        double* xq = a.At + q * b;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = threadIdx.x; i < b; i += NT) {
          const double x = __ldcg(xp + i), y = __ldcg(xq + i);
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
          const int w = threadIdx.x >> 5;
          red[w] = al;
          red[NW + w] = be;
          red[2 * NW + w] = ga;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          double A2 = 0.0, B2 = 0.0, G = 0.0;
          for (int w = 0; w < NW; ++w) {
            A2 += red[w];
            B2 += red[NW + w];
            G += red[2 * NW + w];
          }
          double cs, sn;
          jacobi_rotation(A2, B2, G, tiny, cs, sn);
          rot[0] = cs;
          rot[1] = sn;
        }
        __syncthreads();
        const double cs = rot[0], sn = rot[1];
        if (sn != 0.0) {
          mine = 1;
          double* vp = a.Vt + p * b;
          double* vq = a.Vt + q * b;
          for (int i = threadIdx.x; i < b; i += NT) {
            const double x = __ldcg(xp + i), y = __ldcg(xq + i);
            xp[i] = cs * x - sn * y;
            xq[i] = sn * x + cs * y;
            const double vx = __ldcg(vp + i), vy = __ldcg(vq + i);
            vp[i] = cs * vx - sn * vy;
            vq[i] = sn * vx + cs * vy;
          }
        }
      }
      if (!grid_sync(a.bar, a.err)) return;
    }
    if (threadIdx.x == 0 && mine) atomicOr(a.flags + sweep, 1);
    if (!grid_sync(a.bar, a.err)) return;
    if (__ldcg(a.flags + sweep) == 0) break;
  }
  // column norms
  for (int64_t j = blockIdx.x; j < b; j += gridDim.x) {
    double s = 0.0;
    for (int i = threadIdx.x; i < b; i += NT) {
      const double v = __ldcg(a.At + j * b + i);
      s = fma(v, v, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) a.sigma[j] = sqrt(s);
  }
}

// Sorting (descending) and the outputs: U (b x b, ld) with U(:, j) = a_{idx j} / sigma_{idx j},
// Vt (b x b, ld) with row j = row idx j of the accumulated Vt, sigma sorted.  One CTA.
__global__ void __launch_bounds__(1024) jacobi_finish_kernel(const double* At, const double* Vw, double* sig_work,
                                                             int b, double* sigma, double* U, double* Vt, int64_t ld,
                                                             int* bad) {
  extern __shared__ int idx[];
  // rank of column j among the norms (descending, ties by index): idx[rank] = j
  // (a non-finite norm sorts last, so the ranks always form a permutation)
  for (int j = threadIdx.x; j < b; j += blockDim.x) {
    const double sj = isfinite(sig_work[j]) ? sig_work[j] : -1.0;
    int rank = 0;
    for (int t = 0; t < b; ++t) {
      const double st = isfinite(sig_work[t]) ? sig_work[t] : -1.0;
      rank += (st > sj || (st == sj && t < j)) ? 1 : 0;
    }
    idx[rank] = j;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)b * b; e += blockDim.x) {
    const int64_t i = e / b, j = e % b;
    const int src = idx[j];
    const double s = sig_work[src];
    U[i * ld + j] = (s > 0.0) ? At[(int64_t)src * b + i] / s : ((i == j) ? 1.0 : 0.0);
    Vt[j * ld + i] = Vw[(int64_t)idx[j] * b + i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < b; ++j) {
      sigma[j] = sig_work[idx[j]];
      if (!isfinite(sigma[j])) *bad = 1;
    }
  }
}

}  // namespace jc

int jacobi_svd_multi(Ctx& c, const double* A, int64_t b, int64_t ld, double* sigma, double* U, double* Vt, int* bad) {
  if (b <= 0) return TTR_OK;
  if (b > 4096) return set_error("jacobi_svd_multi: matrix too large"), TTR_ERR_UNSUPPORTED;
  int dev = 0, nsm = 0, coop = 0;
  TTR_CUDA(cudaGetDevice(&dev));
  TTR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  TTR_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return set_error("jacobi_svd_multi: cooperative launch unsupported"), TTR_ERR_UNSUPPORTED;
  double *At = nullptr, *Vw = nullptr, *sw = nullptr, *nrm2 = nullptr;
  unsigned* bar = nullptr;
  int* flags = nullptr;
  TTR_CHECK(c.alloc_t(&At, b * b));
  TTR_CHECK(c.alloc_t(&Vw, b * b));
  TTR_CHECK(c.alloc_t(&sw, b));
  TTR_CHECK(c.alloc_t(&nrm2, 1));
  TTR_CHECK(c.alloc_t(&bar, 4));
  TTR_CHECK(c.alloc_t(&flags, jc::MAX_SWEEPS));
  TTR_CUDA(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), c.stream));
  TTR_CUDA(cudaMemsetAsync(flags, 0, jc::MAX_SWEEPS * sizeof(int), c.stream));
  TTR_CUDA(cudaMemsetAsync(nrm2, 0, sizeof(double), c.stream));
  if (!c.d_flags) {
    TTR_CHECK(c.alloc_t(&c.d_flags, 4));
    TTR_CUDA(cudaMemsetAsync(c.d_flags, 0, 4 * sizeof(int), c.stream));
  }
  jc::Args a{};
  a.A = A; a.ld = ld; a.b = (int)b; a.At = At; a.Vt = Vw; a.sigma = sw; a.bar = bar; a.err = c.d_flags;
  a.flags = flags; a.nrm2 = nrm2;
  // one CTA per SM, no more than there are pairs in a round
  const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(nsm, (b + 1) / 2));
  void* params[] = {&a};
  TTR_CUDA(cudaLaunchCooperativeKernel((const void*)jc::jacobi_kernel, dim3(nblocks), dim3(jc::NT), params, 0,
                                       c.stream));
  TTR_CHECK(c.check_launch("jacobi_svd_multi"));
  jc::jacobi_finish_kernel<<<1, 1024, sizeof(int) * b, c.stream>>>(At, Vw, sw, (int)b, sigma, U, Vt, ld, bad);
  return c.check_launch("jacobi_finish");
}

}  // namespace ttr
