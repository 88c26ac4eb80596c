// Internal declarations shared by the libttround translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ttround.h"

namespace ttr {

// ----------------------------------------------------------------------------- errors
void set_error(const std::string& msg);
// The library's stream-ordered memory pool of the current device (keeps freed memory for reuse);
// nullptr if it cannot be made (callers then use the device's default pool).
cudaMemPool_t library_pool(cudaStream_t stream);

#define TTR_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::ttr::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return (e_ == cudaErrorMemoryAllocation) ? TTR_ERR_OOM : TTR_ERR_CUDA;        \
    }                                                                               \
  } while (0)

#define TTR_CHECK(expr)            \
  do {                             \
    int s_ = (expr);               \
    if (s_ != TTR_OK) return s_;   \
  } while (0)

// ----------------------------------------------------------------------------- context
// Per-call state: the stream, stream-ordered allocations made during the call (freed at the
// end unless handed to the caller) and a count of kernel launches.
struct Ctx {
  cudaStream_t stream = nullptr;
  int64_t launches = 0;
  std::vector<void*> owned;
  int* d_flags = nullptr;          // device status flags (0 = ok); bounded waits write here
  double* ws = nullptr;            // reduction workspace (128 x 1024 doubles) for gram_reduce
  unsigned* ws_ticket = nullptr;   // its completion counter (kept at zero between kernels)
  double* ac_part = nullptr;       // adaptive_core: rotating accumulation buffers (three)
  int ac_part_cap = 0;             // doubles per buffer
  double* ac_gwork = nullptr;      // adaptive_core: the CTAs' rows when they do not fit in shared memory
  size_t ac_gwork_bytes = 0;
  double* ac_red = nullptr;        // adaptive_core: reduced projection coefficients
  unsigned* ac_bar = nullptr;      // adaptive_core: grid barrier counter/generation
  int* ac_io = nullptr;            // adaptive_core: status, column count, estimate count, estimates
  int ac_io_cap = 0;               // estimates it can hold
  unsigned long long* ac_prof = nullptr;   // adaptive_core phase cycles (profiling only)
  unsigned long long* tc_prof = nullptr;   // tensor-core kernel phase cycles per mode (profiling only)
  void* bprep = nullptr;           // tensor-core B-operand workspace (digit planes, scales)
  double* ptmp = nullptr;          // sliced block projection: the product Q P before S -= Q P
  size_t ptmp_bytes = 0;
  unsigned* prep_bar = nullptr;    // grid barrier of the fused B preparation (counter, generation)
  size_t bprep_bytes = 0;
  int workspace();

  // optional launch timeline (environment TTR_PROFILE=1): an event after every launch; the time
  // between consecutive events is charged to the later launch (so it includes GPU idle time)
  std::vector<std::pair<const char*, cudaEvent_t>> prof;
  bool profiling = false;
  bool autotune = false;           // tensor-core launches: measure tile shapes on first use (ttr_options::autotune)
  int sm_share = 0;                // SMs this call's K-split launches are sized for (ttr_options::max_sms; 0: all)
  cudaEvent_t prof_start = nullptr;
  void prof_begin();
  void prof_report();

  // optional kernel timing (ttr_options::kernel_timing): event pairs around selected launches
  enum { KT_BLOCK_LOOP = 0, KT_RL = 1 };
  struct KernelTime {
    cudaEvent_t a, b;
    int kind;
    double work;
  };
  bool timing = false;
  std::vector<KernelTime> ktimes;
  void time_begin(int kind);
  void time_end(double work);
  void time_collect(ttr_result* out);   // after the stream has been synchronized

  int alloc(void** p, size_t bytes);
  template <typename T>
  int alloc_t(T** p, size_t count) {
    return alloc(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  int check_launch(const char* what);
  void release();
  ~Ctx() {
    prof_report();
    release();
  }
};

// ----------------------------------------------------------------------------- kernels (FP64 SIMT)
// General strided, batched FP64 GEMM: C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n),
// with X(i,j) = X[i*s_i + j*s_j].  split_k > 1 accumulates partial sums atomically into C
// (C must then be initialised by the caller and beta is ignored).
struct Gemm {
  int64_t M = 0, N = 0, K = 0;
  const double* A = nullptr;
  int64_t sam = 0, sak = 0;
  const double* B = nullptr;
  int64_t sbk = 0, sbn = 0;
  double* C = nullptr;
  int64_t scm = 0, scn = 0;
  double alpha = 1.0, beta = 0.0;
  int split_k = 1;
};
int gemm_f64(Ctx& c, const Gemm& g);

// C (a x b) = X^T Y over m rows (row-major operands; FP64; C zeroed here).
int gram_tn(Ctx& c, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t a, int64_t b,
            double* C, int64_t ldc);
// C = alpha X P + beta C with X m x k, P k x n (small k, n), row-major; if sumsq_out, the sum
// of squares of the new C is added to *sumsq_out.
int gemm_nn_small(Ctx& c, const double* X, int64_t ldx, const double* P, int64_t ldp, int64_t m, int64_t k, int64_t n,
                  double* C, int64_t ldc, double alpha, double beta, double* sumsq_out = nullptr);
// C (a x b, may be null) = X^T Y over m rows for a*b <= 1024, reduced inside the kernel; with
// chol, also R (b x b upper, C + shift I = R^T R), invd = 1/diag(R) and *bad on breakdown;
// zero_out (optional) is set to 0 once the reduction is complete.
int gram_reduce(Ctx& c, const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t a, int64_t b,
                double* C, int64_t ldc, int chol, const double* shift, double* R, double* invd, int* bad,
                double* zero_out);
// out = X R^{-1} (b <= 64) by row-parallel forward substitution.
int tri_solve(Ctx& c, const double* X, int64_t ldx, int64_t m, int64_t b, const double* R, const double* invd,
              double* out, int64_t ldo);

// Omega_k(:, col0:col1) for cores k = k_lo..k_hi (1-based); block k goes to
// dst + (k - k_lo) * ostride as row-major [i][j - col0] with leading dimension ld.
// dst_int (optional) receives 2^20 * Omega as integers in the same layout.
int omega_fill(Ctx& c, uint64_t seed, int32_t k_lo, int32_t k_hi, const int64_t* n_host,
               int64_t col0, int64_t col1, double* dst, int* dst_int, int64_t ostride, int64_t ld);

// omega_fill (no dst_int) for cores k_lo..k_lo+nc-1 with mode sizes n_host[0..nc-1] (host), which
// reach the kernels as kernel parameters: allocates nothing and copies nothing.
int omega_fill_byval(Ctx& c, uint64_t seed, int32_t k_lo, int32_t nc, const int64_t* n_host, int64_t col0,
                     int64_t col1, double* dst, int64_t ostride, int64_t ld);

// W_k(a, j) = sum_i T(a*n + i, j) * Omega(i, j) for a < r0, j < w  (Algorithm 3 epilogue)
int omega_reduce(Ctx& c, const double* T, int64_t ldt, const double* Om, int64_t ldo, int64_t r0,
                 int64_t n, int64_t w, double* W, int64_t ldw);

// Sum of squares of an m x b strided matrix, accumulated into *out (device, zeroed by caller).
int sumsq(Ctx& c, const double* S, int64_t m, int64_t b, int64_t sm, int64_t sb, double* out);
// S <- S - T (m x b, row-major); with sumsq_out, the sum of squares of the new S is added there.
int sub2d(Ctx& c, double* S, int64_t lds, const double* T, int64_t ldt, int64_t m, int64_t b, double* sumsq_out);

// Upper Cholesky of a b x b symmetric matrix (row-major, ld) in place, plus the inverse of
// the factor into Rinv (row-major, ld).  shift is added to the diagonal first.  *bad is set
// to 1 on a non-positive or non-finite pivot.
int chol_inv(Ctx& c, double* G, int64_t b, int64_t ld, const double* shift_dev, double* Rinv,
             int* bad);

// One block of the host-driven adaptive loop, from T = [Q, Q1]^T [Q1, S] ((cc + bb) x (bb + bn),
// leading dimension ldt), C = T[:cc, :bb]:  G2 = T[cc:, :bb] - C^T C (bb x bb) and
// Mn = T[cc:, bb:] - C^T T[:cc, bb:] (bb x bn).
int block_step_gram(Ctx& c, const double* T, int64_t ldt, int64_t cc, int64_t bb, int64_t bn, double* G2,
                    double* Mn);
// out (b x n) = Rinv^T M for upper-triangular Rinv (b x b, leading dimension ldr), M b x n.
int tri_t_mul(Ctx& c, const double* Rinv, int64_t ldr, const double* M, int64_t b, int64_t n, double* out);

// X += (*scale_dev) * G with G an m x b standard Gaussian matrix drawn from `seed`.
int add_gaussian(Ctx& c, double* X, int64_t m, int64_t b, int64_t ld, const double* scale_dev, uint64_t seed);

// Copies / fills
int copy2d(Ctx& c, double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows,
           int64_t cols);
int fill_zero(Ctx& c, double* p, int64_t count);

// Small-matrix SVD by one-sided Jacobi (Hestenes) on a b x b matrix in one CTA:
// A (row-major, ld) is overwritten; on return sigma (descending), U (b x b, ld) and
// Vt (b x b, ld) with A_in = U diag(sigma) Vt.
int jacobi_svd(Ctx& c, double* A, int64_t b, int64_t ld, double* sigma, double* U, double* Vt,
               int* bad);

}  // namespace ttr
