// Per-core-parallel form of the right-to-left partial contractions (Algorithm 3), after the
// observation of the Conclusion (Sec. 5) that most of the sketching work is independent across
// the cores:
//   G_k(:, :, j) = sum_i X_k(:, i, :) Omega_k(i, j)          all cores k = t..d in one launch
//   W_d(:, j) = G_d(:, 0, j),  W_k(:, j) = G_k(:, :, j) W_{k+1}(:, j)
// The second line is the only right-to-left dependency left; it runs as one launch in which each
// CTA carries one sketch column (and one summand of a sum of TTs) through all cores.  The chain of
// d - t + 1 dependent contraction launches becomes two launches, at the price of the r_{k-1} r_k w
// values of every G_k (written once, read once): the form for latency-bound shapes, where the
// cores are small and the chain of launches dominates.  FP64 throughout.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "engine.cuh"

namespace ttr {
namespace pc {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

__global__ void __launch_bounds__(NT) g_kernel(const PcCore* tab, int64_t w) {
  const PcCore cr = tab[blockIdx.z];
  const int64_t R = cr.r0 * cr.r1;            // rows (a, c) of G_k, c fastest
  const int64_t row0 = (int64_t)blockIdx.x * TM, col0 = (int64_t)blockIdx.y * TN;
  if (row0 >= R || col0 >= w) return;
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  const int64_t nr1 = cr.n * cr.r1;
  for (int64_t k0 = 0; k0 < cr.n; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += NT) {
      const int kk = e / TM, rr = e % TM;
      const int64_t row = row0 + rr, i = k0 + kk;
      double v = 0.0;
      if (row < R && i < cr.n) {
        const int64_t a = row / cr.r1, c = row - a * cr.r1;
        v = cr.X[a * nr1 + i * cr.r1 + c];
      }
      As[kk][rr] = v;
    }
    for (int e = threadIdx.x; e < TK * TN; e += NT) {
      const int kk = e / TN, cc = e % TN;
      const int64_t i = k0 + kk, j = col0 + cc;
      Bs[kk][cc] = (i < cr.n && j < w) ? cr.Om[i * cr.ldom + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) av[m] = As[kk][tx + 16 * m];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][ty + 16 * q];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = fma(av[m], bv[q], acc[m][q]);
    }
    __syncthreads();
  }
  // G_k stored [j][a][c]: one contiguous r_{k-1} x r_k matrix per sketch column
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t row = row0 + tx + 16 * m, j = col0 + ty + 16 * q;
      if (row < R && j < w) cr.G[j * R + row] = acc[m][q];
    }
}

// One CTA per (sketch column j, summand s): the chain over the summand's cores, last to first.
__global__ void __launch_bounds__(NT) chain_kernel(const PcCore* tab, int ncores, int64_t w) {
  extern __shared__ double vs[];               // two vectors of rmax
  const int64_t j = blockIdx.x;
  const PcCore* cores = tab + (int64_t)blockIdx.y * ncores;   // cores t..d of this summand
  int64_t rmax = 1;
  for (int q = 0; q < ncores; ++q) rmax = max(rmax, cores[q].r0);
  double* v = vs;
  double* vn = vs + rmax;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  {
    const PcCore cr = cores[ncores - 1];       // k = d, r_d = 1: W_d(:, j) = G_d(:, 0, j)
    for (int64_t a = threadIdx.x; a < cr.r0; a += NT) {
      const double x = cr.G[j * cr.r0 + a];
      v[a] = x;
      cr.W[a * cr.ldw + j] = x;
    }
    __syncthreads();
  }
  for (int q = ncores - 2; q >= 0; --q) {
    const PcCore cr = cores[q];
    const double* g = cr.G + j * cr.r0 * cr.r1;
    for (int64_t a = warp; a < cr.r0; a += NT / 32) {
      double s = 0.0;
      for (int64_t c = lane; c < cr.r1; c += 32) s = fma(g[a * cr.r1 + c], v[c], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        vn[a] = s;
        cr.W[a * cr.ldw + j] = s;
      }
    }
    __syncthreads();
    double* t = v;
    v = vn;
    vn = t;
  }
}

}  // namespace pc

int rl_percore(Ctx& c, const std::vector<PcCore>& cores, int nsum, int64_t w) {
  if (cores.empty() || w <= 0) return TTR_OK;
  const int ncores = (int)(cores.size() / (size_t)nsum);
  if (ncores < 1 || (size_t)ncores * nsum != cores.size()) return set_error("rl_percore: bad core table"), TTR_ERR_ARG;
  if (w > 65535 * 64 || nsum > 65535) return set_error("rl_percore: too many columns"), TTR_ERR_UNSUPPORTED;
  PcCore* tab = nullptr;
  TTR_CHECK(c.alloc(reinterpret_cast<void**>(&tab), sizeof(PcCore) * cores.size()));
  TTR_CUDA(cudaMemcpyAsync(tab, cores.data(), sizeof(PcCore) * cores.size(), cudaMemcpyHostToDevice, c.stream));
  int64_t Rmax = 1, rmax = 1;
  for (const PcCore& p : cores) {
    Rmax = std::max(Rmax, p.r0 * p.r1);
    rmax = std::max(rmax, p.r0);
  }
  if (cores.size() > 65535) return set_error("rl_percore: too many cores"), TTR_ERR_UNSUPPORTED;
  const int64_t gx = (Rmax + pc::TM - 1) / pc::TM, gy = (w + pc::TN - 1) / pc::TN;
  if (gx > 0x7fffffff) return set_error("rl_percore: cores too large"), TTR_ERR_UNSUPPORTED;
  pc::g_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)cores.size()), pc::NT, 0, c.stream>>>(tab, w);
  TTR_CHECK(c.check_launch("percore_g"));
  const size_t smem = sizeof(double) * 2 * (size_t)rmax;
  if (smem > 200 * 1024) return set_error("rl_percore: ranks too large for the chain kernel"), TTR_ERR_UNSUPPORTED;
  if (smem > 48 * 1024)
    TTR_CUDA(cudaFuncSetAttribute((const void*)pc::chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  pc::chain_kernel<<<dim3((unsigned)w, (unsigned)nsum), pc::NT, smem, c.stream>>>(tab, ncores, w);
  return c.check_launch("percore_chain");
}

}  // namespace ttr
