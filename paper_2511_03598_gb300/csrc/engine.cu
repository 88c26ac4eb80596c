// Small FP64 helper kernels used by the driver (transposes and diagonal scalings).
#include <math.h>

#include "engine.cuh"

namespace ttr {

__global__ void transpose_kernel(const double* A, int64_t rows, int64_t cols, double* out) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, cc = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && cc < cols) ? A[r * cols + cc] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t cc = c0 + i, r = r0 + threadIdx.x;
    if (cc < cols && r < rows) out[cc * rows + r] = tile[threadIdx.x][i];
  }
}

int transpose_f64(Ctx& c, const double* A, int64_t rows, int64_t cols, double* out) {
  if (rows <= 0 || cols <= 0) return TTR_OK;
  dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_kernel<<<grid, dim3(32, 8), 0, c.stream>>>(A, rows, cols, out);
  return c.check_launch("transpose");
}

__global__ void scale_cols_kernel(double* U, int64_t ld, int64_t ncols, int64_t rows, const double* s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * ncols; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, j = e % ncols;
    U[i * ld + j] *= s[j];
  }
}

int scale_cols_f64(Ctx& c, double* U, int64_t ld, int64_t ncols, int64_t rows, const double* s) {
  const int64_t tot = rows * ncols;
  if (tot <= 0) return TTR_OK;
  scale_cols_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, c.stream>>>(U, ld, ncols, rows, s);
  return c.check_launch("scale_cols");
}

__global__ void scale_rows_kernel(double* A, int64_t ld, int64_t nrows, int64_t ncols, const double* s) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrows * ncols; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols, j = e % ncols;
    A[i * ld + j] *= s[i];
  }
}

int scale_rows_f64(Ctx& c, double* A, int64_t ld, int64_t nrows, int64_t ncols, const double* s) {
  const int64_t tot = nrows * ncols;
  if (tot <= 0) return TTR_OK;
  scale_rows_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, c.stream>>>(A, ld, nrows, ncols, s);
  return c.check_launch("scale_rows");
}

__global__ void identity_kernel(double* A, int64_t m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += (int64_t)gridDim.x * blockDim.x)
    A[e] = (e / m == e % m) ? 1.0 : 0.0;
}

int identity_f64(Ctx& c, double* A, int64_t m) {
  if (m <= 0) return TTR_OK;
  identity_kernel<<<(unsigned)std::min<int64_t>((m * m + 255) / 256, 4096), 256, 0, c.stream>>>(A, m);
  return c.check_launch("identity");
}

}  // namespace ttr
