// FP64 SIMT kernels of libttround: the native-FP64 contraction path and the small dense
// kernels (Gram matrices, Cholesky, norms, one-sided Jacobi SVD) that stay FP64 in every
// precision mode.
#include <math.h>

#include <algorithm>

#include "gaussian.cuh"
#include "ttr_internal.cuh"
#include "rsqrt.cuh"

namespace ttr {

// ----------------------------------------------------------------------------- GEMM
// 64 x 64 output tile, K chunks of 16 staged in shared memory, 256 threads x (4 x 4) outputs.
// The staging loop picks the thread-to-element mapping from the operand strides so that the
// global loads are coalesced along whichever index is contiguous.
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(Gemm g, int64_t kchunk) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * GT, n0 = (int64_t)blockIdx.x * GT;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(g.K, kb + kchunk);
  double acc[4][4] = {};
  const bool a_kfast = (g.sak == 1);
  const bool b_nfast = (g.sbn == 1) || (g.sbk != 1);
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int idx = tid + t * 256;
      int mm, kk;
      if (a_kfast) { kk = idx & 15; mm = idx >> 4; } else { mm = idx & 63; kk = idx >> 6; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < ke) ? g.A[gm * g.sam + gk * g.sak] : 0.0;
      int nn, kb2;
      if (b_nfast) { nn = idx & 63; kb2 = idx >> 6; } else { kb2 = idx & 15; nn = idx >> 4; }
      const int64_t gn = n0 + nn, gk2 = k0 + kb2;
      Bs[kb2][nn] = (gn < g.N && gk2 < ke) ? g.B[gk2 * g.sbk + gn * g.sbn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      double* cp = g.C + gm * g.scm + gn * g.scn;
      const double v = g.alpha * acc[i][j];
      if (gridDim.z > 1) atomicAdd(cp, v);
      else *cp = (g.beta == 0.0) ? v : fma(g.beta, *cp, v);
    }
  }
}

int gemm_f64(Ctx& c, const Gemm& g) {
  if (g.M <= 0 || g.N <= 0) return TTR_OK;
  int splits = g.split_k < 1 ? 1 : g.split_k;
  int64_t kchunk = (g.K + splits - 1) / splits;
  kchunk = ((kchunk + GK - 1) / GK) * GK;
  if (kchunk < GK) kchunk = GK;
  splits = (int)((g.K + kchunk - 1) / kchunk);
  if (splits < 1) splits = 1;
  dim3 grid((unsigned)((g.N + GT - 1) / GT), (unsigned)((g.M + GT - 1) / GT), (unsigned)splits);
  if (g.K <= 0) grid.z = 1;
  gemm_f64_kernel<<<grid, 256, 0, c.stream>>>(g, g.K <= 0 ? GK : kchunk);
  return c.check_launch("gemm_f64");
}

// ----------------------------------------------------------------------------- tall-skinny products
// C (a x b, row-major ldc) += X^T Y over rows [0, m): X(r, i) = X[r*ldx + i], Y(r, j) = Y[r*ldy + j].
// Each CTA takes a block of rows; every thread owns output elements (i, j) and accumulates
// over the block's rows, then adds its partial sum atomically (C is zeroed by the caller).
// FP64 work is exactly 2 m a b: no padding of the small dimensions.
__global__ void __launch_bounds__(256) gram_tn_kernel(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                                                       int64_t m, int64_t a, int64_t b, int64_t rows_per_block,
                                                       double* C, int64_t ldc) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(m, r0 + rows_per_block);
  for (int64_t o = threadIdx.x; o < a * b; o += blockDim.x) {
    const int64_t i = o / b, j = o % b;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t r = r0;
    for (; r + 3 < r1; r += 4) {
      s0 = fma(X[r * ldx + i], Y[r * ldy + j], s0);
      s1 = fma(X[(r + 1) * ldx + i], Y[(r + 1) * ldy + j], s1);
      s2 = fma(X[(r + 2) * ldx + i], Y[(r + 2) * ldy + j], s2);
      s3 = fma(X[(r + 3) * ldx + i], Y[(r + 3) * ldy + j], s3);
    }
    for (; r < r1; ++r) s0 = fma(X[r * ldx + i], Y[r * ldy + j], s0);
    atomicAdd(C + i * ldc + j, (s0 + s1) + (s2 + s3));
  }
}

int gram_tn(Ctx& c, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t a, int64_t b,
            double* C, int64_t ldc) {
  if (a <= 0 || b <= 0) return TTR_OK;
  TTR_CUDA(cudaMemset2DAsync(C, ldc * sizeof(double), 0, b * sizeof(double), a, c.stream));
  if (m <= 0) return TTR_OK;
  // enough row blocks to cover the GPU twice, at least 16 rows each
  int64_t blocks = std::min<int64_t>(304, std::max<int64_t>(1, m / 16));
  const int64_t rpb = (m + blocks - 1) / blocks;
  blocks = (m + rpb - 1) / rpb;
  gram_tn_kernel<<<(unsigned)blocks, 256, 0, c.stream>>>(X, ldx, Y, ldy, m, a, b, rpb, C, ldc);
  return c.check_launch("gram_tn");
}

// ---- Gram with in-kernel reduction: C (a x b) = X^T Y over m rows, a*b <= 1024.
// Each CTA writes its partial to ws[blockIdx][a*b]; the last CTA to finish (ticket counter,
// reset by that CTA) sums the partials.  Optionally that CTA then factors C + shift*I = R^T R
// (upper Cholesky, in shared memory) and writes R, 1/diag(R) and a breakdown flag, and/or
// zeroes *zero_out (an accumulator the next kernel adds into).
constexpr int GRAM_MAX = 1024;

// acc[q] += X(r, oi[q]) Y(r, oj[q]) over the nr staged rows, for the first NQ output slots
template <int NQ>
__device__ __forceinline__ void gram_rows(const double* Xs, const double* Ys, int nr, int a, int b, int ab,
                                          const int (&oi)[GRAM_MAX / 256], const int (&oj)[GRAM_MAX / 256],
                                          double (&acc)[GRAM_MAX / 256]) {
  for (int r = 0; r < nr; ++r) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (threadIdx.x + q * 256 < ab) acc[q] = fma(Xs[r * a + oi[q]], Ys[r * b + oj[q]], acc[q]);
  }
}

__global__ void __launch_bounds__(256) gram_reduce_kernel(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                                                           int64_t m, int a, int b, int64_t rpb, double* ws,
                                                           unsigned* ticket, double* C, int64_t ldc, int chol,
                                                           const double* shift, double* R, double* invd, int* bad,
                                                           double* zero_out, int sym) {
  __shared__ double G[GRAM_MAX];
  __shared__ int last;
  const int ab = a * b;
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int64_t r1 = min(m, r0 + rpb);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // Rows of this block in tiles staged in shared memory (coalesced row loads); every thread owns up
  // to GRAM_MAX / 256 outputs (i, j) and accumulates X(r, i) Y(r, j) over the tile's rows.
  __shared__ double tile[4096];
  const int tr = max(1, min(64, 4096 / (a + b)));
  double* Xs = tile;
  double* Ys = tile + tr * a;
  constexpr int OPT = GRAM_MAX / 256;
  int oi[OPT], oj[OPT];
  double acc[OPT];
  // sym (X == Y, a == b): only the upper triangle i <= j, b (b + 1) / 2 outputs, row by row
  const int nout = sym ? a * (a + 1) / 2 : ab;
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = threadIdx.x + q * 256;
    int i = 0, j = 0;
    if (o < nout) {
      if (sym) {
        int rem = o;
        while (rem >= b - i) {
          rem -= b - i;
          ++i;
        }
        j = i + rem;
      } else {
        i = o / b;
        j = o % b;
      }
    }
    oi[q] = i;
    oj[q] = j;
    acc[q] = 0.0;
  }
  for (int64_t t0 = r0; t0 < r1; t0 += tr) {
    const int nr = (int)min((int64_t)tr, r1 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * a; e += blockDim.x) Xs[e] = X[(t0 + e / a) * ldx + e % a];
    for (int e = threadIdx.x; e < nr * b; e += blockDim.x) Ys[e] = Y[(t0 + e / b) * ldy + e % b];
    __syncthreads();
    // only the slots that hold outputs in some thread are issued: FP64 instructions with every
    // lane masked off still take FP64 pipe time on this part
    switch ((nout + 255) >> 8) {
      case 1: gram_rows<1>(Xs, Ys, nr, a, b, nout, oi, oj, acc); break;
      case 2: gram_rows<2>(Xs, Ys, nr, a, b, nout, oi, oj, acc); break;
      case 3: gram_rows<3>(Xs, Ys, nr, a, b, nout, oi, oj, acc); break;
      default: gram_rows<4>(Xs, Ys, nr, a, b, nout, oi, oj, acc); break;
    }
  }
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = threadIdx.x + q * 256;
    if (o < nout) ws[(int64_t)blockIdx.x * ab + oi[q] * b + oj[q]] = acc[q];
  }
  (void)warp;
  (void)lane;
  (void)nw;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the partials of the other CTAs are read through L2 (__ldcg): L1 is not coherent across SMs
  // and the workspace is reused by every reduction of the call
  // eight independent partial sums keep eight L2 loads in flight per thread
  for (int o = threadIdx.x; o < ab; o += blockDim.x) {
    // the symmetric Gram keeps its partials in the upper triangle
    const int src = (sym && o / b > o % b) ? (o % b) * b + o / b : o;
    double t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = 0.0;
    unsigned blk = 0;
    for (; blk + 8 <= gridDim.x; blk += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] += __ldcg(ws + (int64_t)(blk + u) * ab + src);
    }
    for (; blk < gridDim.x; ++blk) t[0] += __ldcg(ws + (int64_t)blk * ab + src);
    const double v = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    G[o] = v;
    if (C) C[(o / b) * ldc + (o % b)] = v;
  }
  if (threadIdx.x == 0) {
    *ticket = 0u;
    if (zero_out) *zero_out = 0.0;
  }
  if (!chol) return;
  __syncthreads();
  // upper Cholesky in shared memory: G[j][c], c >= j, becomes R[j][c]
  __shared__ double piv;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  const double sh = shift ? *shift : 0.0;
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (threadIdx.x == 0) {
      double dsum = G[j * b + j] + sh;
      for (int p = 0; p < j; ++p) dsum -= G[p * b + j] * G[p * b + j];
      if (!(dsum > 0.0) || !isfinite(dsum)) {
        fail = 1;
        dsum = 1.0;
      }
      piv = sqrt(dsum);
      G[j * b + j] = piv;
    }
    __syncthreads();
    for (int col = j + 1 + threadIdx.x; col < b; col += blockDim.x) {
      double v = G[j * b + col];
      for (int p = 0; p < j; ++p) v -= G[p * b + j] * G[p * b + col];
      G[j * b + col] = v / piv;
    }
    __syncthreads();
  }
  for (int o = threadIdx.x; o < b * b; o += blockDim.x) {
    const int i = o / b, j = o % b;
    R[o] = (j >= i) ? G[o] : 0.0;
    if (i == j) invd[i] = 1.0 / G[o];
  }
  if (threadIdx.x == 0 && fail) *bad = 1;
}

int gram_reduce(Ctx& c, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t a, int64_t b,
                double* C, int64_t ldc, int chol, const double* shift, double* R, double* invd, int* bad,
                double* zero_out) {
  if (a * b > GRAM_MAX || a <= 0 || b <= 0) return TTR_ERR_UNSUPPORTED;
  if (chol && a != b) return TTR_ERR_UNSUPPORTED;
  TTR_CHECK(c.workspace());
  // blocks of at least 64 rows, at most 128 blocks (bounds the final reduction)
  int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(128, m / 64));
  const int64_t rpb = (std::max<int64_t>(m, 1) + blocks - 1) / blocks;
  blocks = std::max<int64_t>(1, (m + rpb - 1) / rpb);
  const int sym = (X == Y && ldx == ldy && a == b) ? 1 : 0;
  gram_reduce_kernel<<<(unsigned)blocks, 256, 0, c.stream>>>(X, ldx, Y, ldy, m, (int)a, (int)b, rpb, c.ws, c.ws_ticket,
                                                              C, ldc, chol, shift, R, invd, bad, zero_out, sym);
  return c.check_launch("gram_reduce");
}

// out (m x b) = X (m x b) R^{-1} for upper-triangular R (b x b, row-major) by forward
// substitution along each row: q_j = (x_j - sum_{i<j} q_i R_ij) / R_jj.  Row-parallel; BMAX is
// a compile-time bound so the row stays in registers.
template <int BMAX>
__global__ void __launch_bounds__(256) tri_solve_kernel(const double* X, int64_t ldx, int64_t m, int b, const double* R,
                                                         const double* invd, double* out, int64_t ldo) {
  __shared__ double Rs[BMAX * BMAX];
  __shared__ double id[BMAX];
  for (int o = threadIdx.x; o < BMAX * BMAX; o += blockDim.x) {
    const int i = o / BMAX, j = o % BMAX;
    Rs[o] = (i < b && j < b) ? R[i * b + j] : 0.0;
  }
  for (int o = threadIdx.x; o < BMAX; o += blockDim.x) id[o] = (o < b) ? invd[o] : 0.0;
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double q[BMAX];
    const double* xr = X + r * ldx;
#pragma unroll
    for (int j = 0; j < BMAX; ++j) q[j] = (j < b) ? xr[j] : 0.0;
#pragma unroll
    for (int j = 0; j < BMAX; ++j) {
      double v = q[j];
#pragma unroll
      for (int i = 0; i < j; ++i) v = fma(-q[i], Rs[i * BMAX + j], v);
      q[j] = v * id[j];
    }
    double* orow = out + r * ldo;
#pragma unroll
    for (int j = 0; j < BMAX; ++j)
      if (j < b) orow[j] = q[j];
  }
}

int tri_solve(Ctx& c, const double* X, int64_t ldx, int64_t m, int64_t b, const double* R, const double* invd,
              double* out, int64_t ldo) {
  if (b > 32) return TTR_ERR_UNSUPPORTED;
  if (m <= 0 || b <= 0) return TTR_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((m + 255) / 256, 1216);
  // the substitution is unrolled to BMAX columns, and FP64 instructions cost pipe time even with
  // their lanes masked off, so BMAX follows b in steps of 4
  switch ((b + 3) / 4) {
    case 1: tri_solve_kernel<4><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    case 2: tri_solve_kernel<8><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    case 3: tri_solve_kernel<12><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    case 4: tri_solve_kernel<16><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    case 5: tri_solve_kernel<20><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    case 6: tri_solve_kernel<24><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    case 7: tri_solve_kernel<28><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
    default: tri_solve_kernel<32><<<blocks, 256, 0, c.stream>>>(X, ldx, m, (int)b, R, invd, out, ldo); break;
  }
  return c.check_launch("tri_solve");
}

// C (m x n, ldc) = alpha * X (m x k, ldx) P (k x n, ldp) + beta * C, for small k and n: one
// thread per output element, P staged in shared memory (k*n <= 4096).
__global__ void __launch_bounds__(256) gemm_nn_small_kernel(const double* X, int64_t ldx, const double* P, int64_t ldp,
                                                             int64_t m, int64_t k, int64_t n, double* C, int64_t ldc,
                                                             double alpha, double beta, double* sumsq_out) {
  __shared__ double Ps[4096];
  __shared__ double red[8];
  for (int64_t e = threadIdx.x; e < k * n; e += blockDim.x) Ps[e] = P[(e / n) * ldp + (e % n)];
  __syncthreads();
  const int64_t tot = m * n;
  double ss = 0.0;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < tot; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = o / n, j = o % n;
    const double* xr = X + r * ldx;
    double s = 0.0;
    for (int64_t q = 0; q < k; ++q) s = fma(xr[q], Ps[q * n + j], s);
    double* cp = C + r * ldc + j;
    const double v = (beta == 0.0) ? alpha * s : fma(beta, *cp, alpha * s);
    *cp = v;
    ss = fma(v, v, ss);
  }
  if (sumsq_out) {
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(sumsq_out, t);
    }
  }
}

int gemm_nn_small(Ctx& c, const double* X, int64_t ldx, const double* P, int64_t ldp, int64_t m, int64_t k, int64_t n,
                  double* C, int64_t ldc, double alpha, double beta, double* sumsq_out) {
  if (m <= 0 || n <= 0) return TTR_OK;
  if (k * n > 4096) {
    if (sumsq_out) return TTR_ERR_UNSUPPORTED;
    Gemm g;
    g.M = m; g.N = n; g.K = k;
    g.A = X; g.sam = ldx; g.sak = 1;
    g.B = P; g.sbk = ldp; g.sbn = 1;
    g.C = C; g.scm = ldc; g.scn = 1;
    g.alpha = alpha; g.beta = beta;
    return gemm_f64(c, g);
  }
  const int64_t tot = m * n;
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 1216);
  gemm_nn_small_kernel<<<blocks, 256, 0, c.stream>>>(X, ldx, P, ldp, m, k, n, C, ldc, alpha, beta, sumsq_out);
  return c.check_launch("gemm_nn_small");
}

// ----------------------------------------------------------------------------- Omega
__global__ void omega_kernel(uint64_t seed, int32_t k_lo, const int64_t* nk, int64_t col0, int64_t w,
                             double* dst, int* dst_int, int64_t ostride, int64_t ld) {
  const int32_t kk = blockIdx.y;                       // core offset
  const int64_t n = nk[kk];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w, j = e % w;
    const int32_t q = omega_int(seed, (uint32_t)(k_lo + kk), (uint32_t)i, (uint32_t)(col0 + j));
    dst[kk * ostride + i * ld + j] = (double)q * (1.0 / kOmegaScale);
    if (dst_int) dst_int[kk * ostride + i * ld + j] = q;
  }
}

int omega_fill(Ctx& c, uint64_t seed, int32_t k_lo, int32_t k_hi, const int64_t* n_host, int64_t col0,
               int64_t col1, double* dst, int* dst_int, int64_t ostride, int64_t ld) {
  const int32_t nc = k_hi - k_lo + 1;
  const int64_t w = col1 - col0;
  if (nc <= 0 || w <= 0) return TTR_OK;
  int64_t* nk = nullptr;
  TTR_CHECK(c.alloc_t(&nk, nc));
  int64_t nmax = 0;
  for (int i = 0; i < nc; ++i) nmax = n_host[k_lo - 1 + i] > nmax ? n_host[k_lo - 1 + i] : nmax;
  TTR_CUDA(cudaMemcpyAsync(nk, n_host + (k_lo - 1), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, c.stream));
  const int64_t per = nmax * w;
  unsigned bx = (unsigned)((per + 255) / 256);
  if (bx > 1024) bx = 1024;
  omega_kernel<<<dim3(bx, nc), 256, 0, c.stream>>>(seed, k_lo, nk, col0, w, dst, dst_int, ostride, ld);
  return c.check_launch("omega_fill");
}

// Mode sizes of up to kOmegaByValue cores, passed to the kernel by value (kernel parameter space),
// so that filling Omega needs no device copy of them.
constexpr int kOmegaByValue = 256;
struct ModeSizes {
  int64_t n[kOmegaByValue];
};

__global__ void omega_kernel_byval(uint64_t seed, int32_t k_lo, ModeSizes nk, int64_t col0, int64_t w, double* dst,
                                   int64_t ostride, int64_t ld) {
  const int32_t kk = blockIdx.y;                       // core offset within this launch
  const int64_t n = nk.n[kk];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w, j = e % w;
    const int32_t q = omega_int(seed, (uint32_t)(k_lo + kk), (uint32_t)i, (uint32_t)(col0 + j));
    dst[kk * ostride + i * ld + j] = (double)q * (1.0 / kOmegaScale);
  }
}

// As omega_fill without dst_int, with the mode sizes n_host[0..nc-1] of cores k_lo..k_lo+nc-1 read
// on the host and handed to the kernels by value (kOmegaByValue cores per launch): allocates nothing
// and copies nothing.
int omega_fill_byval(Ctx& c, uint64_t seed, int32_t k_lo, int32_t nc, const int64_t* n_host, int64_t col0,
                     int64_t col1, double* dst, int64_t ostride, int64_t ld) {
  const int64_t w = col1 - col0;
  if (nc <= 0 || w <= 0) return TTR_OK;
  for (int32_t c0 = 0; c0 < nc; c0 += kOmegaByValue) {
    const int32_t cn = std::min<int32_t>(kOmegaByValue, nc - c0);
    ModeSizes ms;
    int64_t nmax = 0;
    for (int32_t i = 0; i < kOmegaByValue; ++i) ms.n[i] = i < cn ? n_host[c0 + i] : 0;
    for (int32_t i = 0; i < cn; ++i) nmax = std::max(nmax, ms.n[i]);
    const int64_t per = nmax * w;
    unsigned bx = (unsigned)((per + 255) / 256);
    if (bx > 1024) bx = 1024;
    if (bx == 0) bx = 1;
    omega_kernel_byval<<<dim3(bx, cn), 256, 0, c.stream>>>(seed, k_lo + c0, ms, col0, w, dst + (int64_t)c0 * ostride,
                                                          ostride, ld);
    TTR_CHECK(c.check_launch("omega_fill"));
  }
  return TTR_OK;
}

// ----------------------------------------------------------------------------- Omega reduction
__global__ void omega_reduce_kernel(const double* T, int64_t ldt, const double* Om, int64_t ldo, int64_t r0,
                                    int64_t n, int64_t w, double* W, int64_t ldw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r0 * w) return;
  const int64_t a = e / w, j = e % w;
  const double* t = T + a * n * ldt + j;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = fma(t[i * ldt], Om[i * ldo + j], s);
  W[a * ldw + j] = s;
}

int omega_reduce(Ctx& c, const double* T, int64_t ldt, const double* Om, int64_t ldo, int64_t r0, int64_t n,
                 int64_t w, double* W, int64_t ldw) {
  const int64_t tot = r0 * w;
  if (tot <= 0) return TTR_OK;
  omega_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(T, ldt, Om, ldo, r0, n, w, W, ldw);
  return c.check_launch("omega_reduce");
}

// ----------------------------------------------------------------------------- sum of squares
__global__ void sumsq_kernel(const double* S, int64_t m, int64_t b, int64_t sm, int64_t sb, double* out) {
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b, j = e % b;
    const double v = S[i * sm + j * sb];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

int sumsq(Ctx& c, const double* S, int64_t m, int64_t b, int64_t sm, int64_t sb, double* out) {
  const int64_t tot = m * b;
  if (tot <= 0) return TTR_OK;
  unsigned blocks = (unsigned)((tot + 255) / 256);
  if (blocks > 304) blocks = 304;
  sumsq_kernel<<<blocks, 256, 0, c.stream>>>(S, m, b, sm, sb, out);
  return c.check_launch("sumsq");
}

// S <- S - T (rows x cols, row-major), adding the sum of squares of the new S to *out if given.
__global__ void sub2d_kernel(double* S, int64_t lds, const double* T, int64_t ldt, int64_t m, int64_t b, double* out) {
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b, j = e % b;
    const double v = S[i * lds + j] - T[i * ldt + j];
    S[i * lds + j] = v;
    s = fma(v, v, s);
  }
  if (!out) return;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

int sub2d(Ctx& c, double* S, int64_t lds, const double* T, int64_t ldt, int64_t m, int64_t b, double* sumsq_out) {
  const int64_t tot = m * b;
  if (tot <= 0) return TTR_OK;
  unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 1216);
  sub2d_kernel<<<blocks, 256, 0, c.stream>>>(S, lds, T, ldt, m, b, sumsq_out);
  return c.check_launch("sub2d");
}

// ----------------------------------------------------------------------------- perturbation
// X(i, j) += scale * g(i, j), g standard Gaussian from the sketch generator with core index 0
// (a counter range the sketches never use).  Used to lift an exactly rank-deficient sketch.
__global__ void add_gaussian_kernel(double* X, int64_t m, int64_t b, int64_t ld, const double* scale, uint64_t seed) {
  const double sc = *scale;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / b, j = e % b;
    X[i * ld + j] += sc * gaussian_f64(seed, 0u, (uint32_t)i, (uint32_t)j);
  }
}

int add_gaussian(Ctx& c, double* X, int64_t m, int64_t b, int64_t ld, const double* scale_dev, uint64_t seed) {
  const int64_t tot = m * b;
  if (tot <= 0) return TTR_OK;
  add_gaussian_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 2048), 256, 0, c.stream>>>(X, m, b, ld, scale_dev, seed);
  return c.check_launch("add_gaussian");
}

// ----------------------------------------------------------------------------- Cholesky + inverse
// One CTA.  Upper factor R (G = R^T R) overwrites the upper triangle of G; Rinv = R^{-1}.
// Right-looking: step j takes the pivot, scales row j and updates the trailing upper triangle
// with one independent FMA per element, so the critical path is a few FP64 operations per column
// (not a dot product of length j); R^{-1} likewise, by rows from the last, each finished row of
// R^{-1} subtracted from the rows above it at once.  Pivots come from one reciprocal square root
// (r = 1/sqrt(d), R_jj = d r), with no FP64 square root or division.  inv (dynamic shared memory,
// b doubles) keeps the r_j for the inverse.
__global__ void __launch_bounds__(1024) chol_inv_kernel(double* G, int64_t b, int64_t ld, const double* shift,
                                                        double* Rinv, int* bad) {
  extern __shared__ double inv[];
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  if (tid == 0) fail = 0;
  const double sh = shift ? *shift : 0.0;
  for (int64_t j = tid; j < b; j += nt) G[j * ld + j] += sh;
  __syncthreads();
  __shared__ double rs;
  for (int64_t j = 0; j < b; ++j) {
    // thread 0 takes pivot j (R_jj = d r, r = 1/sqrt(d)); the others scale row j - 1 by r_{j-1},
    // which no later update reads unscaled
    if (tid == 0) {
      double d = G[j * ld + j];
      if (!(d > 0.0) || !isfinite(d)) {
        fail = 1;
        d = 1.0;
      }
      const double r = rsqrt_full(d);
      rs = r;
      inv[j] = r;
      G[j * ld + j] = d * r;
    }
    if (j > 0) {
      const double rp = inv[j - 1];
      for (int64_t col = j + tid; col < b; col += nt) G[(j - 1) * ld + col] *= rp;
    }
    __syncthreads();
    // G[p][q] -= R[j][p] R[j][q] = G[j][p] G[j][q] r^2 for j < p <= q: warps over rows p, lanes over q
    const double r2 = rs * rs;
    for (int64_t p = j + 1 + warp; p < b; p += nw) {
      const double t = G[j * ld + p] * r2;
      for (int64_t q = p + lane; q < b; q += 32) G[p * ld + q] = fma(-t, G[j * ld + q], G[p * ld + q]);
    }
    __syncthreads();
  }
  // Rinv starts as the identity (upper part); for p = b-1 .. 0: row p *= 1/R[p][p], then
  // Rinv[i][c] -= R[i][p] Rinv[p][c] for i < p, c >= p.
  for (int64_t e = tid; e < b * b; e += nt) {
    const int64_t i = e / b, col = e % b;
    Rinv[i * ld + col] = (i == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int64_t pr = b - 1; pr >= 0; --pr) {
    const double ip = inv[pr];
    for (int64_t col = pr + tid; col < b; col += nt) Rinv[pr * ld + col] *= ip;
    __syncthreads();
    for (int64_t i = warp; i < pr; i += nw) {
      const double rip = G[i * ld + pr];
      for (int64_t col = pr + lane; col < b; col += 32)
        Rinv[i * ld + col] = fma(-rip, Rinv[pr * ld + col], Rinv[i * ld + col]);
    }
    __syncthreads();
  }
  if (tid == 0 && fail) *bad = 1;
}

int chol_inv(Ctx& c, double* G, int64_t b, int64_t ld, const double* shift_dev, double* Rinv, int* bad) {
  if (b <= 0) return TTR_OK;
  if (b > 6144) return set_error("chol_inv: block wider than 6144 columns"), TTR_ERR_UNSUPPORTED;
  const int threads = b <= 64 ? 256 : 1024;
  const size_t smem = sizeof(double) * (size_t)b;
  if (smem > 48 * 1024)
    TTR_CUDA(cudaFuncSetAttribute((const void*)chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  chol_inv_kernel<<<1, threads, smem, c.stream>>>(G, b, ld, shift_dev, Rinv, bad);
  return c.check_launch("chol_inv");
}

// ----------------------------------------------------------------------------- host-driven block step
// From T = [Q, Q1]^T [Q1, S] ((cc + bb) x (bb + bn), leading dimension ldt) with C = T[:cc, :bb]:
//   G2 = T[cc:, :bb] - C^T C            (bb x bb, leading dimension bb)
//   Mn = T[cc:, bb:] - C^T T[:cc, bb:]  (bb x bn, leading dimension bn)
// One warp per output; the lanes split the sum over the cc rows of T.
__global__ void __launch_bounds__(256) block_step_gram_kernel(const double* T, int64_t ldt, int64_t cc, int64_t bb,
                                                              int64_t bn, double* G2, double* Mn) {
  const int lane = threadIdx.x & 31;
  const int64_t wcols = bb + bn;
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (o >= bb * wcols) return;
  const int64_t i = o / wcols, j = o % wcols;
  double s0 = 0.0, s1 = 0.0;
  int64_t p = lane;
  for (; p + 32 < cc; p += 64) {
    s0 = fma(T[p * ldt + i], T[p * ldt + j], s0);
    s1 = fma(T[(p + 32) * ldt + i], T[(p + 32) * ldt + j], s1);
  }
  if (p < cc) s0 = fma(T[p * ldt + i], T[p * ldt + j], s0);
  double s = s0 + s1;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    const double v = T[(cc + i) * ldt + j] - s;
    if (j < bb) G2[i * bb + j] = v;
    else Mn[i * bn + (j - bb)] = v;
  }
}

int block_step_gram(Ctx& c, const double* T, int64_t ldt, int64_t cc, int64_t bb, int64_t bn, double* G2,
                    double* Mn) {
  if (bb <= 0) return TTR_OK;
  const int64_t warps = bb * (bb + bn);
  block_step_gram_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, c.stream>>>(T, ldt, cc, bb, bn, G2, Mn);
  return c.check_launch("block_step_gram");
}

// out (b x n) = Rinv^T M for Rinv = R^{-1} upper triangular (b x b, leading dimension ldr)
__global__ void tri_t_mul_kernel(const double* Rinv, int64_t ldr, const double* M, int64_t b, int64_t n, double* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e % n;
    double v = 0.0;
    for (int64_t p = 0; p <= i; ++p) v = fma(Rinv[p * ldr + i], M[p * n + j], v);
    out[e] = v;
  }
}

int tri_t_mul(Ctx& c, const double* Rinv, int64_t ldr, const double* M, int64_t b, int64_t n, double* out) {
  if (b <= 0 || n <= 0) return TTR_OK;
  tri_t_mul_kernel<<<(unsigned)std::min<int64_t>((b * n + 255) / 256, 1024), 256, 0, c.stream>>>(Rinv, ldr, M, b, n,
                                                                                                  out);
  return c.check_launch("tri_t_mul");
}

// ----------------------------------------------------------------------------- copies
__global__ void copy2d_kernel(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    dst[i * ldd + j] = src[i * lds + j];
  }
}

int copy2d(Ctx& c, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int64_t cols) {
  if (rows <= 0 || cols <= 0) return TTR_OK;
  if (ldd == cols && lds == cols) {
    TTR_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)(rows * cols), cudaMemcpyDeviceToDevice, c.stream));
    return TTR_OK;
  }
  if (cols < 64) {
    // narrow strided rows (the block columns of the adaptive loop): one coalesced kernel pass
    const unsigned blocks = (unsigned)std::min<int64_t>((rows * cols + 255) / 256, 152 * 16);
    copy2d_kernel<<<blocks, 256, 0, c.stream>>>(dst, ldd, src, lds, rows, cols);
    return c.check_launch("copy2d");
  }
  TTR_CUDA(cudaMemcpy2DAsync(dst, ldd * sizeof(double), src, lds * sizeof(double), cols * sizeof(double), rows,
                             cudaMemcpyDeviceToDevice, c.stream));
  return TTR_OK;
}

int fill_zero(Ctx& c, double* p, int64_t count) {
  if (count <= 0) return TTR_OK;
  TTR_CUDA(cudaMemsetAsync(p, 0, count * sizeof(double), c.stream));
  return TTR_OK;
}

// ----------------------------------------------------------------------------- Jacobi SVD
// One-sided (Hestenes) Jacobi on the columns of a b x b matrix A, one CTA, b <= 1024.
// The columns are rotated as the rows of A^T, which lives in U's storage during the sweeps, so a
// warp reads and writes each column it rotates as one contiguous run; V accumulates the same
// rotations on the rows of Vt.  Round-robin pair ordering: in round r, position i pairs with
// position b2-1-i where positions hold players (0, 1+((i-1+r) mod (b2-1))).  One warp per pair.
// A pair is rotated when |a_p^T a_q| > 1e-15 ||a_p|| ||a_q||, unless both columns are below the
// rounding level b u ||A||_F of the factor A came from (their rotations change nothing above it).
// Singular values come out to about u ||A|| absolute (no Gram matrix is formed).
__global__ void __launch_bounds__(1024) jacobi_svd_kernel(double* A, int64_t b, int64_t ld, double* sigma,
                                                          double* U, double* Vt, int* bad) {
  extern __shared__ int sh_idx[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int64_t b2 = (b + 1) & ~1LL;
  double* At = U;                                    // row j of At = column j of A
  __shared__ double s_part[32];
  __shared__ int rotated;
  double nrm2 = 0.0;
  for (int64_t e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int64_t i = e / b, j = e % b;
    const double v = A[i * ld + j];
    At[j * ld + i] = v;
    nrm2 = fma(v, v, nrm2);
    Vt[i * ld + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
  if (lane == 0) s_part[warp] = nrm2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nwarps; ++w) t += s_part[w];
    s_part[0] = t;
  }
  __syncthreads();
  const double floor_ = (double)b * 2.220446049250313e-16;
  const double tiny = floor_ * floor_ * s_part[0];   // squared column norm of the rounding level
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int64_t r = 0; r < b2 - 1; ++r) {
      for (int64_t pi = warp; pi < b2 / 2; pi += nwarps) {
        const int64_t i1 = pi, i2 = b2 - 1 - pi;
        const int64_t p = (i1 == 0) ? 0 : 1 + ((i1 - 1 + r) % (b2 - 1));
        const int64_t q = (i2 == 0) ? 0 : 1 + ((i2 - 1 + r) % (b2 - 1));
        if (p >= b || q >= b) continue;
        double* xp = At + p * ld;
        double* xq = At + q * ld;
        double al = 0, be = 0, ga = 0;
        for (int64_t i = lane; i < b; i += 32) {
          const double x = xp[i], y = xq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        double cs, sn;
        jacobi_rotation(al, be, ga, tiny, cs, sn);
        if (sn != 0.0) {
          double* vp = Vt + p * ld;
          double* vq = Vt + q * ld;
          for (int64_t i = lane; i < b; i += 32) {
            const double x = xp[i], y = xq[i];
            xp[i] = cs * x - sn * y;
            xq[i] = sn * x + cs * y;
            const double vx = vp[i], vy = vq[i];
            vp[i] = cs * vx - sn * vy;
            vq[i] = sn * vx + cs * vy;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // sigma_j = ||a_j||; sort descending (selection sort by thread 0)
  for (int64_t j = warp; j < b; j += nwarps) {
    double s = 0;
    for (int64_t i = lane; i < b; i += 32) s = fma(At[j * ld + i], At[j * ld + i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sigma[j] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int64_t j = 0; j < b; ++j) sh_idx[j] = (int)j;
    for (int64_t j = 0; j < b; ++j) {
      int64_t best = j;
      for (int64_t t = j + 1; t < b; ++t)
        if (sigma[sh_idx[t]] > sigma[sh_idx[best]]) best = t;
      const int tmp = sh_idx[j];
      sh_idx[j] = sh_idx[best];
      sh_idx[best] = tmp;
    }
  }
  __syncthreads();
  // A (free now) <- the permuted rows of Vt
  for (int64_t e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int64_t j = e / b, i = e % b;
    A[j * ld + i] = Vt[(int64_t)sh_idx[j] * ld + i];
  }
  __syncthreads();
  // Vt's storage <- U(:, j) = a_{idx[j]} / sigma[idx[j]] (row-major U), read from At
  for (int64_t e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int64_t i = e / b, j = e % b;
    const int src = sh_idx[j];
    const double s = sigma[src];
    Vt[i * ld + j] = (s > 0.0) ? At[(int64_t)src * ld + i] / s : ((i == j) ? 1.0 : 0.0);
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int64_t i = e / b, j = e % b;
    U[i * ld + j] = Vt[i * ld + j];
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int64_t i = e / b, j = e % b;
    Vt[i * ld + j] = A[i * ld + j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int64_t j = 0; j < b; ++j) A[j] = sigma[sh_idx[j]];
    for (int64_t j = 0; j < b; ++j) sigma[j] = A[j];
    if (!isfinite(sigma[0])) *bad = 1;
  }
}

int jacobi_svd(Ctx& c, double* A, int64_t b, int64_t ld, double* sigma, double* U, double* Vt, int* bad) {
  if (b <= 0) return TTR_OK;
  if (b > 1024) return TTR_ERR_UNSUPPORTED;
  jacobi_svd_kernel<<<1, 1024, sizeof(int) * b, c.stream>>>(A, b, ld, sigma, U, Vt, bad);
  return c.check_launch("jacobi_svd");
}

}  // namespace ttr
