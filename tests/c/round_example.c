/* Plain-C use of the libttround C ABI: build a small TT (the formal sum of two random TTs), round
 * it adaptively on the GPU, and check the result against the dense tensor.
 *
 *   cc -std=c11 -I include round_example.c -L paper_2511_03598_gb300 -lttround -lcudart -lm
 *
 * Checks: status OK, output cores 1..d-1 left-orthonormal to 1e-12, and
 * ||X - Y||_F <= tol ||X||_F with both tensors expanded densely (n^d = 4096 entries).
 * Prints "OK" on success; exits 1 otherwise. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "ttround.h"

#define D 4
#define N 8

static unsigned long long lcg_state = 12345u;
static double uniform(void) {
  lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
  return ((lcg_state >> 11) + 0.5) / 9007199254740992.0;
}
static double gauss(void) {
  const double u1 = uniform(), u2 = uniform();
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* dense tensor (N^D entries, index i_1 slowest) of a TT with ranks r and host cores c */
static void expand(const int64_t* r, double* const* c, double* out) {
  const int64_t total = (int64_t)pow(N, D);
  for (int64_t idx = 0; idx < total; ++idx) {
    int64_t rem = idx, ii[D];
    for (int k = D - 1; k >= 0; --k) {
      ii[k] = rem % N;
      rem /= N;
    }
    double vec[64] = {1.0};
    int64_t len = 1;
    for (int k = 0; k < D; ++k) {
      double nv[64] = {0.0};
      for (int64_t b = 0; b < r[k + 1]; ++b)
        for (int64_t a = 0; a < len; ++a) nv[b] += vec[a] * c[k][(a * N + ii[k]) * r[k + 1] + b];
      len = r[k + 1];
      memcpy(vec, nv, sizeof(double) * (size_t)len);
    }
    out[idx] = vec[0];
  }
}

int main(void) {
  /* two random TTs of ranks 3 and 2, summed formally: first core side by side, middle cores
   * block-diagonal, last core stacked (ranks 1, 5, 5, 5, 1) */
  const int64_t ra = 3, rb = 2, R = ra + rb;   /* the second summand has rank rb */
  int64_t n[D], r[D + 1];
  r[0] = 1;
  r[D] = 1;
  for (int k = 0; k < D; ++k) n[k] = N;
  for (int k = 1; k < D; ++k) r[k] = R;
  double* host[D];
  for (int k = 0; k < D; ++k) {
    const int64_t cnt = r[k] * N * r[k + 1];
    host[k] = (double*)calloc((size_t)cnt, sizeof(double));
    for (int64_t a = 0; a < r[k]; ++a)
      for (int64_t i = 0; i < N; ++i)
        for (int64_t c = 0; c < r[k + 1]; ++c) {
          /* first and last cores: both summands' entries; middle cores: the diagonal blocks */
          const int nonzero = (k == 0) || (k == D - 1) || ((a < ra) == (c < ra));
          if (nonzero) host[k][(a * N + i) * r[k + 1] + c] = gauss() / sqrt((double)(N * 3));
        }
  }
  double* dev[D];
  for (int k = 0; k < D; ++k) {
    const size_t bytes = sizeof(double) * (size_t)(r[k] * N * r[k + 1]);
    if (cudaMalloc((void**)&dev[k], bytes) != cudaSuccess) return 1;
    cudaMemcpy(dev[k], host[k], bytes, cudaMemcpyHostToDevice);
  }
  ttr_options opts;
  ttr_default_options(&opts);
  const double tol = 1e-10;
  ttr_result res;
  const int st = tt_round_adaptive(D, n, r, (const double* const*)dev, tol, 2, 7u, &opts, NULL, &res);
  if (st != TTR_OK) {
    fprintf(stderr, "tt_round_adaptive: %s (%s)\n", ttr_strerror(st), ttr_last_error());
    return 1;
  }
  double* out[D];
  for (int k = 0; k < D; ++k) {
    const int64_t cnt = res.ranks[k] * N * res.ranks[k + 1];
    out[k] = (double*)malloc(sizeof(double) * (size_t)cnt);
    cudaMemcpy(out[k], res.cores[k], sizeof(double) * (size_t)cnt, cudaMemcpyDeviceToHost);
  }
  int ok = 1;
  /* left-orthonormality of V(Y_k), k = 1..d-1 */
  for (int k = 0; k < D - 1; ++k) {
    const int64_t rows = res.ranks[k] * N, cols = res.ranks[k + 1];
    for (int64_t p = 0; p < cols; ++p)
      for (int64_t q = 0; q < cols; ++q) {
        double g = 0.0;
        for (int64_t row = 0; row < rows; ++row) g += out[k][row * cols + p] * out[k][row * cols + q];
        if (fabs(g - (p == q ? 1.0 : 0.0)) > 1e-12) ok = 0;
      }
  }
  const int64_t total = (int64_t)pow(N, D);
  double* X = (double*)malloc(sizeof(double) * (size_t)total);
  double* Y = (double*)malloc(sizeof(double) * (size_t)total);
  expand(r, host, X);
  expand(res.ranks, out, Y);
  double nx = 0.0, nd = 0.0;
  for (int64_t i = 0; i < total; ++i) {
    nx += X[i] * X[i];
    nd += (X[i] - Y[i]) * (X[i] - Y[i]);
  }
  if (!(sqrt(nd) <= tol * sqrt(nx))) ok = 0;
  printf("ranks");
  for (int k = 0; k <= D; ++k) printf(" %lld", (long long)res.ranks[k]);
  printf("  rel. error %.3e\n", sqrt(nd / nx));
  ttr_free(&res, NULL);
  for (int k = 0; k < D; ++k) {
    cudaFree(dev[k]);
    free(host[k]);
    free(out[k]);
  }
  free(X);
  free(Y);
  printf(ok ? "OK\n" : "FAILED\n");
  return ok ? 0 : 1;
}
