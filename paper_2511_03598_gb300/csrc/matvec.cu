// Rounding of an operator-applied TT vector y = A x (the operator application of TT-GMRES,
// Sec. 4.3; the MPO-MPS product structure the Introduction and Conclusion leave to future work)
// without forming the cores of y in the right-to-left pass.
//
// With operator cores A_k [a][i][j][g] (p_{k-1} x n_k x m_k x p_k; i output, j input index) and
// vector cores x_k [b][j][c] (r_{k-1} x m_k x r_k), the product has cores
//   y_k((a, b), i, (g, c)) = sum_j A_k(a, i, j, g) x_k(b, j, c)             (bond index a r + b)
// and Algorithm 3's step W_k((a,b), l) = sum_{i,(g,c)} y_k((a,b), i, (g,c)) W_{k+1}((g,c), l) Omega_k(i, l)
// is evaluated as
//   Ahat(a, j, g, l) = sum_i A_k(a, i, j, g) Omega_k(i, l)                  (Omega into the operator)
//   Z_g((b, j), l)   = sum_c x_k(b, j, c) W_{k+1}(g r_k + c, l)            (V(x_k) times a row block)
//   W_k((a,b), l)    = sum_{j, g} Ahat(a, j, g, l) Z_g((b, j), l)
// which costs 2 w (p n m p' + r m r' p' + p r m p') per core instead of 2 w (p r n p' r') for the
// formed core plus forming it (2 p r n m p' r'), and reads the small A_k and x_k instead of y_k.
// The left-to-right sweep forms one core of y at a time (mv_form) for the projection of the next
// core, never the whole product.
#include <stdint.h>

#include <algorithm>

#include "engine.cuh"

namespace ttr {

// y_k (p0 r0 x n x p1 r1, row-major [(a, b)][i][(g, c)]) from A_k and x_k
__global__ void mv_form_kernel(const double* A, int64_t p0, int64_t n, int64_t m, int64_t p1, const double* X,
                               int64_t r0, int64_t r1, double* Y) {
  const int64_t cols = p1 * r1, tot = p0 * r0 * n * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e % cols, rest = e / cols;
    const int64_t g = col / r1, c = col - g * r1;
    const int64_t i = rest % n, row = rest / n;
    const int64_t a = row / r0, b = row - a * r0;
    const double* ap = A + ((a * n + i) * m) * p1 + g;   // A(a, i, j, g) at ap[j p1]
    const double* xp = X + (b * m) * r1 + c;             // x(b, j, c) at xp[j r1]
    double s0 = 0.0, s1 = 0.0;
    int64_t j = 0;
    for (; j + 1 < m; j += 2) {
      s0 = fma(ap[j * p1], xp[j * r1], s0);
      s1 = fma(ap[(j + 1) * p1], xp[(j + 1) * r1], s1);
    }
    if (j < m) s0 = fma(ap[j * p1], xp[j * r1], s0);
    Y[e] = s0 + s1;
  }
}

// The same product with the operands staged: one CTA per (b, (a, g)) holds A_k(a, :, :, g) (n x m)
// and x_k(b, :, :) (m x r1) in shared memory and writes y_k((a, b), :, (g, :)).
__global__ void __launch_bounds__(256) mv_form_tiled_kernel(const double* A, int64_t p0, int64_t n, int64_t m,
                                                            int64_t p1, const double* X, int64_t r0, int64_t r1,
                                                            double* Y) {
  extern __shared__ double sm[];
  double* As = sm;               // [n][m]
  double* Xs = sm + n * m;       // [m][r1]
  const int64_t b = blockIdx.x, ag = blockIdx.y;
  const int64_t a = ag / p1, g = ag - a * p1;
  for (int64_t e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int64_t i = e / m, j = e - i * m;
    As[e] = A[((a * n + i) * m + j) * p1 + g];
  }
  for (int64_t e = threadIdx.x; e < m * r1; e += blockDim.x) Xs[e] = X[b * m * r1 + e];
  __syncthreads();
  const int64_t R1 = p1 * r1;
  for (int64_t e = threadIdx.x; e < n * r1; e += blockDim.x) {
    const int64_t i = e / r1, cc = e - i * r1;
    const double* ar = As + i * m;
    double s0 = 0.0, s1 = 0.0;
    int64_t j = 0;
    for (; j + 1 < m; j += 2) {
      s0 = fma(ar[j], Xs[j * r1 + cc], s0);
      s1 = fma(ar[j + 1], Xs[(j + 1) * r1 + cc], s1);
    }
    if (j < m) s0 = fma(ar[j], Xs[j * r1 + cc], s0);
    Y[((a * r0 + b) * n + i) * R1 + g * r1 + cc] = s0 + s1;
  }
}

int mv_form(Ctx& c, const double* A, int64_t p0, int64_t n, int64_t m, int64_t p1, const double* X, int64_t r0,
            int64_t r1, double* Y) {
  const int64_t tot = p0 * r0 * n * p1 * r1;
  if (tot <= 0) return TTR_OK;
  const size_t smem = sizeof(double) * (size_t)(n * m + m * r1);
  if (smem <= 48 * 1024 && r0 <= 0x7fffffff && p0 * p1 <= 65535) {
    mv_form_tiled_kernel<<<dim3((unsigned)r0, (unsigned)(p0 * p1)), 256, smem, c.stream>>>(A, p0, n, m, p1, X, r0, r1,
                                                                                        Y);
    return c.check_launch("mv_form");
  }
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16);
  mv_form_kernel<<<blocks, 256, 0, c.stream>>>(A, p0, n, m, p1, X, r0, r1, Y);
  return c.check_launch("mv_form");
}

// Ahat(a, (j, g), l) = sum_i A_k(a, i, (j, g)) Omega_k(i, l): the sketch block contracted into the
// operator core (p0 x (m p1) x w, l fastest)
__global__ void mv_ahat_kernel(const double* A, int64_t p0, int64_t n, int64_t mp1, const double* Om, int64_t ldom,
                               int64_t w, double* Ahat) {
  const int64_t tot = p0 * mp1 * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e % w, rest = e / w;
    const int64_t jg = rest % mp1, a = rest / mp1;
    const double* ap = A + a * n * mp1 + jg;      // A_k(a, i, (j, g)) at ap[i mp1]
    double s0 = 0.0, s1 = 0.0;
    int64_t i = 0;
    for (; i + 1 < n; i += 2) {
      s0 = fma(ap[i * mp1], Om[i * ldom + l], s0);
      s1 = fma(ap[(i + 1) * mp1], Om[(i + 1) * ldom + l], s1);
    }
    if (i < n) s0 = fma(ap[i * mp1], Om[i * ldom + l], s0);
    Ahat[e] = s0 + s1;
  }
}

int mv_ahat(Ctx& c, const double* A, int64_t p0, int64_t n, int64_t m, int64_t p1, const double* Om, int64_t ldom,
            int64_t w, double* Ahat) {
  const int64_t tot = p0 * m * p1 * w;
  if (tot <= 0) return TTR_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16);
  mv_ahat_kernel<<<blocks, 256, 0, c.stream>>>(A, p0, n, m * p1, Om, ldom, w, Ahat);
  return c.check_launch("mv_ahat");
}

// W_k((a, b), l) = sum_{j, g} Ahat(a, j, g, l) Z_g((b, j), l); with xb (the last core, p1 = r1 = 1)
// Z_0((b, j), l) = x_d(b, j) for every l.
__global__ void mv_reduce_kernel(const double* Ahat, const double* Z, const double* xb, int64_t p0, int64_t r0,
                                 int64_t m, int64_t p1, int64_t w, double* W, int64_t ldw) {
  const int64_t tot = p0 * r0 * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = e % w, row = e / w;
    const int64_t a = row / r0, b = row - a * r0;
    const double* ah = Ahat + (a * m * p1) * w + l;      // Ahat(a, j, g, l) at ah[(j p1 + g) w]
    double s = 0.0;
    if (xb) {
      const double* xr = xb + b * m;
      for (int64_t j = 0; j < m; ++j) s = fma(ah[j * w], xr[j], s);
    } else {
      for (int64_t g = 0; g < p1; ++g) {
        const double* zg = Z + (g * r0 * m + b * m) * w + l;   // Z_g((b, j), l) at zg[j w]
        for (int64_t j = 0; j < m; ++j) s = fma(ah[(j * p1 + g) * w], zg[j * w], s);
      }
    }
    W[row * ldw + l] = s;
  }
}

int mv_reduce(Ctx& c, const double* Ahat, const double* Z, const double* xb, int64_t p0, int64_t r0, int64_t m,
              int64_t p1, int64_t w, double* W, int64_t ldw) {
  const int64_t tot = p0 * r0 * w;
  if (tot <= 0) return TTR_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16);
  mv_reduce_kernel<<<blocks, 256, 0, c.stream>>>(Ahat, Z, xb, p0, r0, m, p1, w, W, ldw);
  return c.check_launch("mv_reduce");
}

}  // namespace ttr
