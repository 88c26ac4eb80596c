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

int mv_form(Ctx& c, const double* A, int64_t p0, int64_t n, int64_t m, int64_t p1, const double* X, int64_t r0,
            int64_t r1, double* Y) {
  const int64_t tot = p0 * r0 * n * p1 * r1;
  if (tot <= 0) return TTR_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 16);
  mv_form_kernel<<<blocks, 256, 0, c.stream>>>(A, p0, n, m, p1, X, r0, r1, Y);
  return c.check_launch("mv_form");
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
