// Contraction engine: routes each contraction of the rounding algorithms to a kernel.
// FP64 mode uses the SIMT DFMA kernels; sliced mode sends the large contractions (partial
// contractions, sketches, next-core projections) to the tcgen05 tensor-core kernels and
// keeps the small dense work in FP64.
#pragma once

#include "ttr_internal.cuh"

namespace ttr {

// Digit planes and column scales of a B operand (K x N, row-major, leading dimension ld), kept
// by the call context so that a later contraction with the same operand need not slice it again.
struct BPlanes {
  uint4* planes = nullptr;
  int* Fmax = nullptr;
  int nchunks = 0, kchunks = 0, tn = 0, s = 0;
  const double* src = nullptr;
  int64_t ld = 0, K = 0, N = 0;
};

// Tensor-core path (ozaki_tc.cu).  Each returns TTR_ERR_UNSUPPORTED when a shape is outside
// what the kernel handles; the engine then uses the FP64 kernel for that call.
int tc_rl_step(Ctx& c, int slices, const double* Xk, int64_t r0, int64_t n, int64_t r1, const double* Wn,
               int64_t ldw, const int* Omi, int64_t ldoi, int64_t w, double* Wout, int64_t ldwo,
               BPlanes* keep = nullptr);
// The partial-contraction step of one core for up to kMaxGroup summands in one launch: summand g
// reads rows off_n[g].. of the stacked W_{k+1} (Kall rows) and writes rows off_out[g].. of the
// stacked W_k.  `keep`: the digit planes of the stacked W_{k+1}, for the sketch.
constexpr int kMaxGroup = 8;
int tc_rl_step_grouped(Ctx& c, int slices, int ng, const double* const* Xk, const int64_t* r0, int64_t n,
                       const int64_t* r1, const double* Wn, int64_t ldw, int64_t Kall, const int64_t* off_n,
                       const int* Omi, int64_t ldoi, int64_t w, double* Wout, int64_t ldwo, const int64_t* off_out,
                       BPlanes* keep);
// C_g = A_g B for up to kMaxGroup row-major A_g sharing one row-major B, in one launch.
int tc_gemm_shared_b(Ctx& c, int slices, int ng, const double* const* A, const int64_t* M, const int64_t* lda,
                     int64_t K, const double* B, int64_t ldb, int64_t N, double* const* C, int64_t ldc);
// The next-core projections of up to kMaxGroup summands in one launch (see Engine::project_group).
int tc_project_grouped(Ctx& c, int slices, int ng, const double* M, int64_t ldm, int64_t L, int64_t Kall,
                       const int64_t* koff, const int64_t* K, const double* const* Xn, const int64_t* ncol,
                       const int64_t* rn, double* Y, int64_t ldy, int64_t rstride, const int64_t* yoff);
int tc_gemm_tn(Ctx& c, int slices, const double* X, int64_t ldx, int64_t m, int64_t a_cols, const double* Y,
               int64_t ldy, int64_t b_cols, double* C, int64_t scm, int64_t scn);
int tc_gemm_rowmajor(Ctx& c, int slices, const double* A, int64_t lda, int64_t M, int64_t K, const double* B,
                     int64_t ldb, int64_t N, double* C, int64_t ldc, const BPlanes* reuse = nullptr);
int tc_project(Ctx& c, int slices, const double* Mk, int64_t ldm, int64_t L, int64_t K, const double* Xn,
               int64_t ncol, double* Y);
// Reduced-precision sketch forms (fs = 2: TF32 operands as BF16 head + tail; fs = 1: BF16 operands;
// FP32 accumulation): the partial-contraction step with FP64 Omega, and a row-major product.
int tc_rl_step_flt(Ctx& c, int fs, const double* Xk, int64_t r0, int64_t n, int64_t r1, const double* Wn, int64_t ldw,
                   const double* Om, int64_t ldo, int64_t w, double* Wout, int64_t ldwo);
int tc_gemm_rowmajor_flt(Ctx& c, int fs, const double* A, int64_t lda, int64_t M, int64_t K, const double* B,
                         int64_t ldb, int64_t N, double* C, int64_t ldc);

// Persistent cooperative kernel for the adaptive block loop of one core (adaptive_core.cu).
// *status: 0 done, 1 needs more sketch columns, 2 CholeskyQR breakdown at column *cc.
// double_float: block-loop arithmetic in double-float on the FP32 pipe (~2^-48 relative; used by
// the sliced form with at most 6 slices, whose contractions already err by ~3e-12, never where
// FP64 accuracy is promised); scale: a value of the order of the sketch entries (the input norm).
// The estimates (||S||_F^2 of each residual block, in order) come back in est_host (host, room for
// est_cap values; *nest of them are written).  bi: columns of each residual sketch (the estimate's
// width); ba <= bi: columns appended per block; tau: the stopping threshold.  Rows that do not fit in
// shared memory live in global memory; host_if_global returns TTR_ERR_UNSUPPORTED instead (the
// caller's host-driven loop, whose wide block projections run on the tensor cores, is faster there).
// tensor_products: the FP64 loop's per-row products as 8-slice tensor-core products where their
// shapes allow (at most 256 rows per CTA, rbar <= 512, ba + bi <= 64, room in shared memory).
bool adaptive_core_rows_fit(int64_t m, int b0, int bi, int rbar, int width, int max_sms);
// widest block (b_init or the residual sketch) the device block loop factors itself; a wider first
// block is factored on the host side before the loop starts at col(Q) = b_init
constexpr int kBlockLoopMaxBlock = 32;
int adaptive_core(Ctx& c, const double* Sall, int64_t lds, double* Q, int64_t ldq, double* S, int64_t m, int b0,
                  int bi, int ba, int rbar, int width, int cc0, double tau, double* est_host, int est_cap, int* status,
                  int* cc, int* nest, bool double_float, double scale, int max_sms, bool host_if_global,
                  bool tensor_products = false);

// Householder QR of a tall row-major m x b matrix (householder.cu), for the deterministic rounding.
// householder_qr overwrites A with the reflectors and R (R also copied to R, b x b, ld ldr, if
// given); householder_apply then writes Q E (m x nq, ld ldq) for a b x nq matrix E (E = I gives the
// thin Q).  The workspace keeps the reflector scalars of the last factorization.
struct HhWork {
  double* buf = nullptr;
  int cap = 0;
  unsigned* bar = nullptr;
  double* vjj = nullptr;
  double* beta = nullptr;
  int bcap = 0;
};
int householder_qr(Ctx& c, HhWork& w, double* A, int64_t lda, int64_t m, int64_t b, double* R, int64_t ldr);
int householder_apply(Ctx& c, HhWork& w, const double* A, int64_t lda, int64_t m, int64_t b, const double* E,
                      int64_t lde, int64_t nq, double* Q, int64_t ldq);

// Jacobi SVD of a b x b row-major A (ld) spread over the SMs (jacobi.cu), same outputs as
// jacobi_svd (sigma descending, U, Vt with ld); A is read only.
int jacobi_svd_multi(Ctx& c, const double* A, int64_t b, int64_t ld, double* sigma, double* U, double* Vt, int* bad);
// b from which the multi-CTA Jacobi is used
constexpr int64_t kJacobiMultiFrom = 48;

// Per-core-parallel partial contractions (percore.cu): one entry per core k = t..d of each summand
// (summand-major, cores in increasing k); G is that core's r0 x r1 x w scratch, W its rows of W_k
// (column 0 = the first sketch column of the call, leading dimension ldw), Om its Omega block.
struct PcCore {
  const double* X;
  int64_t r0, n, r1;
  const double* Om;
  int64_t ldom;
  double* G;
  double* W;
  int64_t ldw;
};
int rl_percore(Ctx& c, const std::vector<PcCore>& cores, int nsum, int64_t w);

// Operator-applied TT vectors (matvec.cu).  mv_form: the core y_k (p0 r0 x n x p1 r1) of y = A x from
// A_k (p0 x n x m x p1) and x_k (r0 x m x r1).  mv_reduce: W_k((a, b), l) = sum_{j,g} Ahat(a, j, g, l)
// Z_g((b, j), l) (Ahat p0 x m x p1 x w, Z p1 x (r0 m) x w); with xb, Z_0((b, j), l) = xb(b, j).
int mv_form(Ctx& c, const double* A, int64_t p0, int64_t n, int64_t m, int64_t p1, const double* X, int64_t r0,
            int64_t r1, double* Y);
int mv_reduce(Ctx& c, const double* Ahat, const double* Z, const double* xb, int64_t p0, int64_t r0, int64_t m,
              int64_t p1, int64_t w, double* W, int64_t ldw);
// Ahat(a, (j, g), l) = sum_i A_k(a, i, (j, g)) Omega_k(i, l), one launch (Omega n x w, leading dimension ldom)
int mv_ahat(Ctx& c, const double* A, int64_t p0, int64_t n, int64_t m, int64_t p1, const double* Om, int64_t ldom,
            int64_t w, double* Ahat);

// out[i] = the block loop's reciprocal square root of x[i] (positive, finite), for its self-test.
int rsqrt_selftest(Ctx& c, const double* x, double* out, int64_t n);
// the one-sided Jacobi rotation (cs, sn) for each triple (A2, B2, G) of abg, into cs_sn
int jacobi_rotation_selftest(Ctx& c, const double* abg, double tiny, double* cs_sn, int64_t n);

// Widest tensor-core tile (UMMA N) usable with s slices.
int tile_width(int s);

// Small helper kernels (engine.cu)
int transpose_f64(Ctx& c, const double* A, int64_t rows, int64_t cols, double* out);
int scale_cols_f64(Ctx& c, double* U, int64_t ld, int64_t ncols, int64_t rows, const double* s);
int scale_rows_f64(Ctx& c, double* A, int64_t ld, int64_t nrows, int64_t ncols, const double* s);   // row i *= s[i]
int identity_f64(Ctx& c, double* A, int64_t m);                                                      // A = I (m x m)

// rows x cc x bcols of a block projection from which the sliced form uses the tensor cores
constexpr double kSlicedProjectWork = 1 << 24;
// Most slices per operand of the tensor-core products: at 8, a product's error bound matches FP64's.
constexpr int kMaxSlices = 8;

struct Engine {
  int precision = TTR_PREC_FP64;
  int slices = 0;
  int fs = 0;      // reduced-precision sketch forms: planes per operand of the W chain and the sketch

  // the sliced tensor-core products run the contractions that are not sketches: every precision but
  // FP64 (the reduced-precision forms keep their projections FP64-accurate at 8 slices)
  bool sliced() const { return precision != TTR_PREC_FP64; }
  bool reduced() const { return fs > 0; }

  int init(Ctx& c, int prec, int sl, double tol) {
    (void)c;
    if (prec != TTR_PREC_FP64 && prec != TTR_PREC_SLICED && prec != TTR_PREC_TF32_SKETCH &&
        prec != TTR_PREC_BF16_SKETCH) {
      set_error("unknown precision");
      return TTR_ERR_ARG;
    }
    precision = prec;
    if (prec == TTR_PREC_TF32_SKETCH || prec == TTR_PREC_BF16_SKETCH) {
      fs = prec == TTR_PREC_TF32_SKETCH ? 2 : 1;
      slices = 8;
      return TTR_OK;
    }
    if (prec == TTR_PREC_SLICED) {
      if (sl == 0) {
        // enough 7-bit slices that the contraction error sits well below the tolerance:
        // about 7*slices - 4 bits survive; ask for 12 bits beyond -log2(tol), at least 4.
        double bits = (tol > 0.0) ? -log2(tol) + 12.0 : 53.0;
        sl = (int)ceil((bits + 4.0) / 7.0);
        if (sl < 4) sl = 4;
        if (sl > 8) sl = 8;
      }
      if (sl < 3 || sl > 8) {
        set_error("slices must be in [3, 8]");
        return TTR_ERR_ARG;
      }
    }
    slices = sl;
    return TTR_OK;
  }

  int small_gemm(Ctx& c, const Gemm& g) const { return gemm_f64(c, g); }

  // sketch columns worth drawing up front: one tensor-core tile in sliced mode
  int64_t natural_width() const { return sliced() ? tile_width(slices) : 64; }

  // S = Z W(:, cols): A row-major (sak == 1), B row-major (sbn == 1), C row-major (scn == 1);
  // `reuse`: planes of W kept by the right-to-left pass
  int sketch(Ctx& c, const Gemm& g, const BPlanes* reuse = nullptr) const {
    if (sliced() && g.sak == 1 && g.sbn == 1 && g.scn == 1 && g.split_k <= 1 && g.alpha == 1.0 && g.beta == 0.0) {
      int st = reduced() ? tc_gemm_rowmajor_flt(c, fs, g.A, g.sam, g.M, g.K, g.B, g.sbk, g.N, g.C, g.scm)
                         : tc_gemm_rowmajor(c, slices, g.A, g.sam, g.M, g.K, g.B, g.sbk, g.N, g.C, g.scm, reuse);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    return gemm_f64(c, g);
  }

  // W_k = sum_i [V(X_k) W_{k+1}](a, i, :) * Omega_k(i, :)   (Algorithm 3, one step)
  int rl_step(Ctx& c, const double* Xk, int64_t r0, int64_t n, int64_t r1, const double* Wn, int64_t ldw,
              const double* Om, const int* Omi, int64_t ldom, int64_t w, double* Wout, int64_t ldwo, double* T,
              BPlanes* keep = nullptr) const {
    if (reduced()) {
      int st = tc_rl_step_flt(c, fs, Xk, r0, n, r1, Wn, ldw, Om, ldom, w, Wout, ldwo);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    } else if (sliced()) {
      int st = tc_rl_step(c, slices, Xk, r0, n, r1, Wn, ldw, Omi, ldom, w, Wout, ldwo, keep);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    Gemm g;
    g.M = r0 * n; g.N = w; g.K = r1;
    g.A = Xk; g.sam = r1; g.sak = 1;
    g.B = Wn; g.sbk = ldw; g.sbn = 1;
    g.C = T; g.scm = w; g.scn = 1;
    TTR_CHECK(gemm_f64(c, g));
    return omega_reduce(c, T, w, Om, ldom, r0, n, w, Wout, ldwo);
  }

  // W_d = H(X_d) Omega_d for ng <= kMaxGroup summands (A[g]: r_{d-1} x n_d row-major, rows M[g]) sharing
  // Omega_d (n_d x w, leading dimension ldo), into C[g] (leading dimension ldc)
  int last_core_group(Ctx& c, int ng, const double* const* A, const int64_t* M, int64_t n, const double* Om,
                      int64_t ldo, int64_t w, double* const* C, int64_t ldc) const {
    if (reduced()) {
      for (int g = 0; g < ng; ++g) {
        int st = tc_gemm_rowmajor_flt(c, fs, A[g], n, M[g], n, Om, ldo, w, C[g], ldc);
        if (st == TTR_ERR_UNSUPPORTED) {
          Gemm q;
          q.M = M[g]; q.N = w; q.K = n;
          q.A = A[g]; q.sam = n; q.sak = 1;
          q.B = Om; q.sbk = ldo; q.sbn = 1;
          q.C = C[g]; q.scm = ldc; q.scn = 1;
          st = gemm_f64(c, q);
        }
        TTR_CHECK(st);
      }
      return TTR_OK;
    }
    if (sliced()) {
      int64_t lda[kMaxGroup];
      for (int g = 0; g < ng; ++g) lda[g] = n;
      int st = tc_gemm_shared_b(c, slices, ng, A, M, lda, n, Om, ldo, w, C, ldc);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    for (int g = 0; g < ng; ++g) {
      Gemm q;
      q.M = M[g]; q.N = w; q.K = n;
      q.A = A[g]; q.sam = n; q.sak = 1;
      q.B = Om; q.sbk = ldo; q.sbn = 1;
      q.C = C[g]; q.scm = ldc; q.scn = 1;
      TTR_CHECK(gemm_f64(c, q));
    }
    return TTR_OK;
  }

  // rl_step for ng <= kMaxGroup summands of a sum of TTs at once (rows off_n[g] of the stacked W_{k+1},
  // rows off_out[g] of the stacked W_k); one summand at a time where the grouped kernel does not apply
  int rl_step_group(Ctx& c, int ng, const double* const* Xk, const int64_t* r0, int64_t n, const int64_t* r1,
                    const double* Wn, int64_t ldw, int64_t Kall, const int64_t* off_n, const double* Om,
                    const int* Omi, int64_t ldom, int64_t w, double* Wout, int64_t ldwo, const int64_t* off_out,
                    double* T, BPlanes* keep = nullptr) const {
    if (sliced() && !reduced()) {
      int st = tc_rl_step_grouped(c, slices, ng, Xk, r0, n, r1, Wn, ldw, Kall, off_n, Omi, ldom, w, Wout, ldwo,
                                  off_out, keep);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    for (int g = 0; g < ng; ++g)
      TTR_CHECK(rl_step(c, Xk[g], r0[g], n, r1[g], Wn + off_n[g] * ldw, ldw, Om, Omi, ldom, w,
                        Wout + off_out[g] * ldwo, ldwo, T));
    return TTR_OK;
  }

  // Y = M H(X_{k+1}):  (L x K)(K x ncol), all row-major; M has leading dimension ldm >= K
  int project(Ctx& c, const double* Mk, int64_t ldm, int64_t L, int64_t K, const double* Xn, int64_t ncol,
              double* Y) const {
    if (sliced()) {
      int st = tc_project(c, slices, Mk, ldm, L, K, Xn, ncol, Y);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    Gemm g;
    g.M = L; g.N = ncol; g.K = K;
    g.A = Mk; g.sam = ldm; g.sak = 1;
    g.B = Xn; g.sbk = ncol; g.sbn = 1;
    g.C = Y; g.scm = ncol; g.scn = 1;
    return gemm_f64(c, g);
  }

  // T (a x b, leading dimension ldt) = Q(:, :a)^T B(:, :b) over `rows` rows.  Wide products (the
  // host-driven loop) go on the tensor cores in sliced form, each exact to the form's stated error,
  // instead of FP64 at 2 FMA per clock per SM.
  int tn_product(Ctx& c, const double* Q, int64_t ldq, int64_t rows, int64_t a, const double* Bm, int64_t ldb,
                 int64_t b, double* T, int64_t ldt) const {
    if (a <= 0 || b <= 0) return TTR_OK;
    if (sliced() && (double)rows * a * b >= kSlicedProjectWork) {
      int st = tc_gemm_tn(c, slices, Q, ldq, rows, a, Bm, ldb, b, T, ldt, 1);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    int st = gram_reduce(c, Q, ldq, Bm, ldb, rows, a, b, T, ldt, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != TTR_ERR_UNSUPPORTED) return st;
    return gram_tn(c, Q, ldq, Bm, ldb, rows, a, b, T, ldt);
  }

  // S (rows x n, leading dimension lds) <- S - Q(:, :k) P with P k x n (leading dimension ldp); with
  // sumsq_out, ||S||_F^2 of the result is stored there.
  int sub_product(Ctx& c, const double* Q, int64_t ldq, int64_t rows, int64_t k, const double* P, int64_t ldp,
                  int64_t n, double* S, int64_t lds, double* sumsq_out = nullptr) const {
    if (n <= 0) return TTR_OK;
    if (sumsq_out) TTR_CUDA(cudaMemsetAsync(sumsq_out, 0, sizeof(double), c.stream));
    if (k <= 0) return sumsq_out ? sumsq(c, S, rows, n, lds, 1, sumsq_out) : TTR_OK;
    if (sliced() && (double)rows * k * n >= kSlicedProjectWork) {
      const size_t need = sizeof(double) * (size_t)rows * n;
      if (c.ptmp_bytes < need) {
        void* t = nullptr;
        TTR_CHECK(c.alloc(&t, std::max(need, 2 * c.ptmp_bytes)));
        c.ptmp = static_cast<double*>(t);
        c.ptmp_bytes = std::max(need, 2 * c.ptmp_bytes);
      }
      int st = tc_gemm_rowmajor(c, slices, Q, ldq, rows, k, P, ldp, n, c.ptmp, n);   // Q P
      if (st == TTR_OK) return sub2d(c, S, lds, c.ptmp, n, rows, n, sumsq_out);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    int st = gemm_nn_small(c, Q, ldq, P, ldp, rows, k, n, S, lds, -1.0, 1.0, sumsq_out);
    if (st == TTR_ERR_UNSUPPORTED && sumsq_out) {
      TTR_CHECK(gemm_nn_small(c, Q, ldq, P, ldp, rows, k, n, S, lds, -1.0, 1.0, nullptr));
      return sumsq(c, S, rows, n, lds, 1, sumsq_out);
    }
    return st;
  }

  // P = Q(:, :cc)^T S;  S <- S - Q(:, :cc) P     (Eq. (3.5) / block Gram-Schmidt)
  // With sumsq_out, ||S||_F^2 of the result is stored there.
  int project_out(Ctx& c, const double* Q, int64_t ldq, int64_t rows, int64_t cc, double* S, int64_t lds,
                  int64_t bcols, double* P, double* sumsq_out = nullptr) const {
    if (cc > 0) TTR_CHECK(tn_product(c, Q, ldq, rows, cc, S, lds, bcols, P, bcols));
    return sub_product(c, Q, ldq, rows, cc, P, bcols, bcols, S, lds, sumsq_out);
  }

  // M (ccols x cols, ld cols) = Q(:, :ccols)^T Z   (M_k = Q_k^T V(Y_k))
  int left_project(Ctx& c, const double* Q, int64_t ldq, const double* Z, int64_t rows, int64_t cols, int64_t ccols,
                   double* M) const {
    if (sliced()) {
      // M^T = Z^T Q: big operand Z^T (column-major view), rows split over CTAs
      int st = tc_gemm_tn(c, slices, Z, cols, rows, cols, Q, ldq, ccols, M, 1, cols);
      if (st != TTR_ERR_UNSUPPORTED) return st;
    }
    return gram_tn(c, Q, ldq, Z, cols, rows, ccols, cols, M, cols);
  }

  // Next core of a sum of TTs, ng <= kMaxGroup summands at once: for summand g, the L x (n r_g) product
  // M(:, koff[g]:koff[g]+K[g]) H(X^(g)) goes to Ynext(a, i, yoff[g] + c), Ynext being L x n x R row-major.
  // Returns TTR_ERR_UNSUPPORTED when the grouped kernel does not apply (the caller goes summand by summand).
  int project_group(Ctx& c, int ng, const double* M, int64_t ldm, int64_t L, int64_t Kall, const int64_t* koff,
                    const int64_t* K, const double* const* Xn, int64_t n, const int64_t* rn, double* Ynext, int64_t R,
                    const int64_t* yoff) const {
    if (!sliced()) return TTR_ERR_UNSUPPORTED;
    int64_t ncol[kMaxGroup];
    for (int g = 0; g < ng; ++g) ncol[g] = n * rn[g];
    return tc_project_grouped(c, slices, ng, M, ldm, L, Kall, koff, K, Xn, ncol, rn, Ynext, n * R, R, yoff);
  }

  int transpose(Ctx& c, const double* A, int64_t rows, int64_t cols, double* out) const {
    return transpose_f64(c, A, rows, cols, out);
  }
  int scale_cols(Ctx& c, double* U, int64_t ld, int64_t ncols, int64_t rows, const double* s) const {
    return scale_cols_f64(c, U, ld, ncols, rows, s);
  }
  int scale_rows(Ctx& c, double* A, int64_t ld, int64_t nrows, int64_t ncols, const double* s) const {
    return scale_rows_f64(c, A, ld, nrows, ncols, s);
  }
  int identity(Ctx& c, double* A, int64_t m) const { return identity_f64(c, A, m); }
};

}  // namespace ttr
