/*
 * ttround.h - C ABI of libttround: randomized TT-rounding with Khatri-Rao-product (KRP)
 * sketches on one NVIDIA GB300 (sm_103a).
 *
 * Method: Al Daas, Ballard, Grigori, Martinez Aguilar, Saibaba, Verma, "Adaptive Randomized
 * Tensor Train Rounding using Khatri-Rao Products" (arXiv 2511.03598).
 *
 * TT layout (Sec. 2.2, Eq. (2.1)): a d-way tensor X = [X_1, ..., X_d] with cores
 * X_k in R^{r_{k-1} x n_k x r_k}, r_0 = r_d = 1.  Every core is one contiguous row-major
 * FP64 array [a][i][c] (a < r_{k-1}, i < n_k, c < r_k) in DEVICE memory, so that the
 * vertical unfolding V(X_k) is the row-major (r_{k-1} n_k) x r_k matrix and the horizontal
 * unfolding H(X_k) the row-major r_{k-1} x (n_k r_k) matrix, with no copies.
 *
 * Arguments common to the rounding calls
 *   d        number of cores, 2 <= d <= TTR_MAX_D.
 *   n        HOST array of d mode sizes, n[k] >= 1.
 *   r        HOST array of d+1 ranks, r[0] = r[d] = 1, r[k] >= 1.
 *   cores    HOST array of d DEVICE pointers; core k holds r[k]*n[k]*r[k+1] doubles and must
 *            be 8-byte aligned.  Read only; not retained after the call returns.
 *   stream   a cudaStream_t (passed as void*; NULL = legacy default stream).  All device
 *            work is ordered on it.  The call returns after the result is complete on the
 *            device and its ranks are known on the host (it synchronizes the stream).
 *   opts     optional (NULL = defaults, see ttr_default_options).
 *   out      result; on success the library owns out->cores (one stream-ordered device
 *            allocation on `stream`) and out->ranks / out->estimates (host); the caller
 *            releases them with ttr_free.  On error nothing is allocated and *out is zeroed
 *            except out->status.
 *
 * Device memory: stream-ordered allocations come from a memory pool private to the library (one
 * per device) that keeps up to 8 GiB of freed memory for reuse by later calls; it is returned to
 * the driver when the process exits.
 *
 * Errors: every call returns a ttr_status; the library never aborts, traps or exits.  Device
 * waits inside kernels are bounded; a wait that runs out reports TTR_ERR_TIMEOUT.
 *
 * Threading: calls on different streams may run concurrently from different host threads; give
 * each a share of the SMs (ttr_options::max_sms) so that their block loops can be resident
 * together.
 */
#ifndef TTROUND_H
#define TTROUND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TTR_MAX_D 4096
#define TTR_MAX_SUMMANDS 4096

typedef enum {
  TTR_OK = 0,
  TTR_ERR_ARG = 1,           /* invalid argument (d, n, r, pointers, tol, ell, block, opts) */
  TTR_ERR_OOM = 2,           /* a device or host allocation failed */
  TTR_ERR_NONFINITE = 3,     /* NaN/Inf met in a sketch, a norm or an estimate */
  TTR_ERR_QR_BREAKDOWN = 4,  /* CholeskyQR failed even after the shifted fallback */
  TTR_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
  TTR_ERR_CUDA = 6,          /* a CUDA runtime call failed (message in ttr_last_error) */
  TTR_ERR_UNSUPPORTED = 7    /* the request is outside what this build supports */
} ttr_status;

/* Arithmetic used for the large contractions (partial contractions, sketches, projections).
 * TTR_PREC_FP64: native FP64 FMA (DFMA) everywhere.
 * TTR_PREC_SLICED: the large contractions run on the BF16 tensor cores (tcgen05) on
 *   fixed-point slices of the FP64 operands with exact FP32 accumulation, recombined in
 *   integer/FP64 arithmetic; `slices` sets the number of 7-bit slices per operand (3..8);
 *   8 slices reproduce FP64 results to about 1e-15 relative, s slices to about s 2^(1-7s) of
 *   sum |a||b| per product.  The host-driven block loop, the Remark 3.2 pass, the truncation SVDs
 *   and every cross-CTA sum are FP64.  The persistent device block loop of Algorithm 6 (its
 *   CholeskyQR2 Gram matrices, block Gram-Schmidt and residual norms) is FP64 as well, unless
 *   ttr_options::block_loop_df asks for double-float at 3..6 slices.
 * TTR_PREC_TF32_SKETCH, TTR_PREC_BF16_SKETCH: the reduced-precision sketch forms.  Only the
 *   right-to-left partial contractions (the W chain, Algorithm 3, with its extensions) and the sketch
 *   S_k = V(Y_k) W_{k+1} take reduced-precision operands: TF32 (each operand rounded to FP32, then to
 *   TF32's 11 significant bits, and multiplied as an exact BF16 head + tail, three BF16 products) or
 *   BF16 (8 significant bits), with FP32 accumulation on the tensor cores and the Omega weighting and
 *   slab sums in FP64.  The next-core projections, QR, Gram matrices, estimator, truncations and
 *   Remark 3.2 pass stay FP64-accurate (8 slices for the large products, FP64 elsewhere).  A
 *   reduced-precision sketch captures the range of X up to a perturbation of about u_low ||X||
 *   (u_low = 2^-11 TF32, 2^-8 BF16), so at tolerances below that the block loop grows the ranks
 *   toward rbar_k; opts->adap_r then truncates the FP64-accurate result. */
typedef enum {
  TTR_PREC_FP64 = 0,
  TTR_PREC_SLICED = 1,
  TTR_PREC_TF32_SKETCH = 2,
  TTR_PREC_BF16_SKETCH = 3
} ttr_precision;

typedef struct {
  int32_t precision;      /* ttr_precision */
  int32_t slices;         /* TTR_PREC_SLICED only; 0 = choose from the tolerance */
  int32_t adap_r;         /* 1: append the right-to-left compression pass (Remark 3.2) */
  double adap_r_tau_scale;/* threshold of that pass = scale * tau (paper: 1.0) */
  double nrmx;            /* adaptive only: ||X|| if known (> 0), else estimated by Eq. (3.6) */
  double f_init, f_inc;   /* adaptive block fractions of Sec. 3.3, used when block <= 0 */
  int64_t width_hint;     /* initial sketch width drawn on the device (0 = automatic); never
                             changes results, only how often the partial contractions are
                             extended (Algorithm 5) */
  int32_t kernel_timing;  /* 1: time the block-loop and partial-contraction kernels with CUDA
                             events on `stream` (fields ms_block_loop ... of ttr_result) */
  int32_t max_sms;        /* largest number of SMs the persistent block-loop kernel (one CTA per
                             SM, all resident at once) may take; 0 = all.  Lets calls on different
                             streams run side by side: e.g. two calls with half the SMs each.  The
                             tensor-core launches that split K over CTAs size the split for the
                             same number of SMs (their CTAs may still run on any SM) */
  int32_t est_min;        /* adaptive only: the residual estimate of each block uses
                             max(b_inc, est_min) sketch columns, while b_inc columns are appended
                             (0 = b_inc, Algorithm 6 as printed; 0..4096) */
  double est_safety;      /* adaptive only: the block loop stops when the estimate is <= tau /
                             est_safety (1 = Algorithm 6 as printed; >= 1).  Sec. 3.4: a KRP
                             estimate from few columns over many remaining modes can fall far below
                             the residual it estimates; est_min = 10 with est_safety = 10 keeps the
                             result within tol on the operator-applied vector (d = 16, tol 1e-8),
                             where the printed rule ends at ~7 tol */
  int32_t rl_percore;     /* right-to-left partial contractions (Algorithm 3): 0 = the chain of
                             per-core contractions (default); 1 = the per-core-parallel form of the
                             Conclusion (Sec. 5): every G_k(:, :, j) = sum_i X_k(:, i, :) Omega_k(i, j)
                             in one launch, then W_k(:, j) = G_k(:, :, j) W_{k+1}(:, j) column by
                             column in another (FP64; scratch 8 sum_k r_{k-1} r_k w bytes); 2 = the
                             per-core form when that scratch is at most 32 MiB in FP64 precision, 2 MiB
                             in sliced precision, else the chain */
  int32_t block_loop_df;  /* TTR_PREC_SLICED with 3..6 slices: 1 = the device block loop's per-CTA
                             arithmetic in double-float (pairs of binary32, about 2^-48 relative, on
                             the FP32 pipe; cross-CTA sums stay FP64); 0 = FP64 (default: CholeskyQR2,
                             the Gram matrices and the estimator FP64 at every slice count) */
  int32_t block_loop_tc;  /* TTR_PREC_SLICED, FP64 block loop: 1 = its per-row products (the block
                             Gram-Schmidt coefficients, the Gram matrices of the second CholeskyQR
                             pass and the updates X - Q P) on the tensor cores as 8-slice products,
                             whose error bound is that of an FP64 product; 0 = FP64 FMA (default:
                             with K <= 256 per CTA these products are short, and the FMA form is
                             the faster one on the measured workloads).  The small factorizations,
                             the residual norms and every decision stay FP64 either way. */
  int32_t autotune;       /* TTR_PREC_SLICED: 1 = the tensor-core launches (partial contractions,
                             sketches, projections, tall products) choose their tile width, K split
                             and slabs per tile from a table of measured shapes: the first call of a
                             shape in the process times the candidates (each twice, on the call's
                             stream) and keeps the fastest; the choices leave the stated error of
                             the sliced form unchanged.  0 = the fixed rule (default) or a shape
                             already measured. */
} ttr_options;

typedef struct {
  int32_t status;         /* ttr_status of the call */
  int32_t d;
  int64_t* ranks;         /* host, d+1 output ranks */
  double** cores;         /* host array of d device pointers (one arena) */
  void* arena;            /* the device allocation behind cores */
  double tau;             /* per-core threshold used (adaptive, deterministic) */
  double nrmx;            /* norm used for tau (given or estimated) */
  int64_t width;          /* final number of sketch columns of W_2..W_d */
  int32_t extensions;     /* times Algorithm 5 appended columns to the partial contractions */
  int32_t n_estimates;    /* number of entries in estimates */
  double* estimates;      /* host: residual estimates ||S_k||_F / sqrt(b_e) in sweep order */
  int32_t* est_core;      /* host: core index k (1-based) of each estimate */
  float ms_sketch_rl;     /* device time of the right-to-left partial contractions */
  float ms_sweep_lr;      /* device time of the left-to-right sweep */
  float ms_total;         /* device time of the whole call */
  int64_t kernel_launches;/* kernels this call launched */
  /* with opts->kernel_timing (else 0): device time, from CUDA events recorded around each launch
   * on `stream`, and algorithmic work of the two dominant kernels */
  double ms_block_loop;   /* persistent adaptive block-loop kernel (Algorithm 6), all launches */
  double flops_block_loop;/* its FP64 arithmetic (2 flops per multiply-add) for the blocks run */
  double ms_rl_kernel;    /* tensor-core partial-contraction kernel (Algorithm 3), all launches */
  double bytes_rl_kernel; /* its algorithmic bytes: each core read once, W_{k+1} read, W_k written */
  int32_t n_block_loop;   /* launches timed */
  int32_t n_rl_kernel;
} ttr_result;

/* Fill `opts` with defaults: FP64, adap_r off, scale 1, nrmx 0 (estimate), f_init 0.1,
 * f_inc 0.05 (the values of Sec. 4.2), width_hint 0, kernel_timing 0, max_sms 0, est_min 0,
 * est_safety 1, rl_percore 0, block_loop_df 0, block_loop_tc 0, autotune 0. */
void ttr_default_options(ttr_options* opts);

/* Algorithm 4 (Sec. 3.2): fixed-rank randomize-then-orthogonalize with a KRP sketch.
 *   ell    target rank l >= 1 for every bond; l_k is clamped to
 *          min(l, l_{k-1} n_k, r_k, prod_{j>k} n_j).
 *   target if 0 < target < l, the left-orthonormal result is truncated to rank `target` by a
 *          right-to-left SVD pass (Remark 3.2 with a rank bound); <= 0 keeps rank l.
 *   seed   64-bit key of the Gaussian stream: Omega_k(i, j) = rint(2^20 g) / 2^20 with g the
 *          Box-Muller Gaussian of Philox4x32-10(counter (j, i, k, 0), key seed), k 1-based.  The
 *          same seed gives the same Omega as the CPU oracle, bit for bit.
 * Output cores 1..d-1 are left-orthonormal (V(Y_k)^T V(Y_k) = I). */
int tt_round_fixed(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores,
                   int64_t ell, int64_t target, uint64_t seed, const ttr_options* opts,
                   void* stream, ttr_result* out);

/* Algorithm 6 (Sec. 3.3) with Algorithm 5: adaptive-rank rounding to relative tolerance tol.
 *   tol    relative Frobenius tolerance eps > 0; per-core threshold tau = eps*nrmx/sqrt(d-1).
 *   block  > 0: b_init = b_inc = block; <= 0: b = ceil(f * rbar_k) with opts->f_init/f_inc.
 *   seed   as in tt_round_fixed; the first columns of the sketch are those of the fixed call.
 * The loop at core k stops when ||S_k||_F / sqrt(b_e) <= tau / opts->est_safety (Eq. (3.5)
 * residual sketch S_k of b_e = max(b_inc, opts->est_min) columns) or when col(Q_k) reaches rbar_k = min(rows, cols of V(Y_k), prod_{j>k} n_j) (the last factor
 * bounds the rank of V(Y_k) H(X_{k+1:d})).  Output cores 1..d-1 are left-orthonormal unless
 * opts->adap_r is set (then cores 2..d are right-orthonormal).  A zero tensor (norm 0, given or
 * estimated) gives the zero TT of ranks 1. */
int tt_round_adaptive(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores,
                      double tol, int64_t block, uint64_t seed, const ttr_options* opts,
                      void* stream, ttr_result* out);

/* Adaptive-rank rounding of a sum X = X^(1) + ... + X^(s) of TT tensors without forming the
 * block-diagonal formal sum (Remark 3.3; the sum forms of Algorithms 5 and 6 in Appendix D).
 *   s      number of summands, 1 <= s <= TTR_MAX_SUMMANDS.
 *   d, n   shared by every summand (n: host array of d mode sizes).
 *   r      host array of s pointers; r[i] points to the d+1 ranks of summand i (r[i][0] =
 *          r[i][d] = 1).
 *   cores  host array of s pointers; cores[i] points to the d device pointers of summand i, each
 *          core row-major [a][i][c] as in tt_round_fixed.  Summands may share core buffers (scaled
 *          copies that differ only in one core), which are read, never written or retained.
 *   tol, seed, opts, stream, out   as in tt_round_adaptive.
 *   block  > 0: b_init = b_inc = block; <= 0: b_init = max_i r_k^(i) clamped to rbar_k (the
 *          appendix's rule) and b_inc = ceil(opts->f_inc * rbar_k); opts->f_init is unused.
 * Every summand is contracted right to left with the same Omega into its own rows of W_k, so the
 * stacked W_k are the partial contractions of the formal sum, and V(Y_1) holds the summands'
 * first cores side by side.  Each next core is projected summand by summand, M^(i) H(X_{k+1}^(i)),
 * which costs sum_i r^(i)^2 instead of (sum_i r^(i))^2 per core.  In block mode the result is that
 * of tt_round_adaptive on the formal sum with the same seed, up to rounding.  Device memory is
 * sized by the formal ranks R_k = sum_i r_k^(i).  Errors: TTR_ERR_ARG for a bad summand (same
 * checks as tt_round_adaptive) or s out of range; otherwise as tt_round_adaptive. */
int tt_round_adaptive_sum(int32_t s, int32_t d, const int64_t* n, const int64_t* const* r,
                          const double* const* const* cores, double tol, int64_t block,
                          uint64_t seed, const ttr_options* opts, void* stream, ttr_result* out);

/* Adaptive-rank rounding (Algorithm 6, as tt_round_adaptive) of an operator-applied TT vector
 * y = A x, the rounding after each operator application in TT-GMRES (Sec. 4.3), without forming the
 * cores of y in the right-to-left pass (the MPO-MPS product structure named in the Introduction and
 * the Conclusion).
 *   n      HOST array of d output mode sizes (the modes of y).
 *   m      HOST array of d input mode sizes (the modes of x).
 *   p      HOST array of d+1 operator ranks, p[0] = p[d] = 1.
 *   A      HOST array of d DEVICE pointers; operator core k is p[k] x n[k] x m[k] x p[k+1] doubles,
 *          row-major [a][i][j][g] with i the output and j the input index:
 *          A(i_1..i_d; j_1..j_d) = A_1(i_1, j_1) ... A_d(i_d, j_d).
 *   r, x   ranks (d+1, r[0] = r[d] = 1) and DEVICE cores (r[k] x m[k] x r[k+1], [b][j][c]) of x.
 *   tol, block, seed, opts, stream, out   as in tt_round_adaptive (opts->rl_percore must be 0).
 * y has ranks p[k] r[k] with cores y_k((a, b), i, (g, c)) = sum_j A_k(a, i, j, g) x_k(b, j, c); the
 * result is that of tt_round_adaptive on those cores with the same seed, up to rounding.  Per core,
 * the partial contraction contracts Omega_k into A_k first, then V(x_k) with each operator-rank block
 * of W_{k+1}, then the two over (j, g); the left-to-right sweep forms one core of y at a time for the
 * projection of the next core.  Errors as tt_round_adaptive. */
int tt_round_adaptive_matvec(int32_t d, const int64_t* n, const int64_t* m, const int64_t* p,
                             const double* const* A, const int64_t* r, const double* const* x, double tol,
                             int64_t block, uint64_t seed, const ttr_options* opts, void* stream,
                             ttr_result* out);

/* Algorithm 1 (Sec. 2.3, Oseledets' TT-Rounding), FP64: right-to-left orthogonalization,
 * tau = ||Y_1|| tol / sqrt(d-1), left-to-right tau-truncated SVDs (smallest rank whose
 * discarded Frobenius tail is <= tau).  The baseline the randomized calls are measured
 * against. */
int tt_round_deterministic(int32_t d, const int64_t* n, const int64_t* r,
                           const double* const* cores, double tol, void* stream,
                           ttr_result* out);

/* ---------------------------------------------------------------------------------------
 * Request server (serving loop; no counterpart in the paper).  Rounding requests of different
 * d, n, ranks, tolerances and precisions are admitted in arrival order while their estimated
 * device footprint fits a memory budget, and run by `workers` host threads, each with its own
 * CUDA stream and an SM share of the persistent block-loop kernel, so that several roundings are
 * in flight at once.  A request is a sum of TTs (one summand for a plain TT) given in HOST
 * memory: the worker copies its cores to the device, rounds it with tt_round_adaptive_sum, and
 * copies the result back to host memory.  Times are host-clock: queueing (submit to admission)
 * and running (admission to result in host memory).
 * -------------------------------------------------------------------------------------- */
typedef struct ttr_server ttr_server;

typedef struct {
  int32_t workers;          /* roundings in flight at once (host thread + stream each), >= 1 */
  int32_t max_sms;          /* SMs the block loop of one request may take; 0 = SMs / workers */
  uint64_t device_budget;   /* bytes of device memory all admitted requests may hold at once */
  int32_t device;           /* CUDA device ordinal */
} ttr_server_config;

typedef struct {
  int32_t status;           /* ttr_status of the rounding */
  int32_t d;
  int64_t* ranks;           /* host, d+1 output ranks */
  double* data;             /* host, the output cores back to back */
  double** cores;           /* d host pointers into data */
  double ms_queue;          /* submit -> admission */
  double ms_run;            /* admission -> result in host memory (H2D, rounding, D2H) */
  uint64_t footprint;       /* device bytes the request was admitted with (estimate) */
  uint64_t bytes_in;        /* bytes of input cores copied to the device */
  int64_t admit_order;      /* 0-based position of the request in the order of admission */
  char message[256];        /* error text of a failed request (the worker's ttr_last_error) */
} ttr_server_result;

typedef struct {
  int64_t submitted, completed, failed, waiting, running;
  uint64_t in_use, peak_in_use;   /* admitted footprint now and at most so far */
} ttr_server_stats;

/* Start the worker threads (they make no CUDA call until a request arrives).  TTR_ERR_ARG for
 * workers < 1, a zero budget or a negative device; TTR_ERR_OOM if the server cannot be made. */
int ttr_server_create(const ttr_server_config* cfg, ttr_server** out);

/* Queue one rounding of X^(1) + ... + X^(s) to relative tolerance tol (arguments as in
 * tt_round_adaptive_sum, but `host_cores` are HOST pointers; pinned memory copies fastest).  The
 * caller keeps the n, r and core arrays valid until ttr_server_wait for this id returns.  opts may
 * be NULL (defaults); its max_sms is replaced by the server's.  The request id goes to *id.
 * Errors: TTR_ERR_ARG for bad shapes (checked here, before queueing), TTR_ERR_UNSUPPORTED when
 * the request's estimated footprint exceeds the whole budget. */
int ttr_server_submit(ttr_server* srv, int32_t s, int32_t d, const int64_t* n, const int64_t* const* r,
                      const double* const* const* host_cores, double tol, int64_t block, uint64_t seed,
                      const ttr_options* opts, int64_t* id);

/* Block until request `id` is done and hand over its result (release with
 * ttr_server_result_free).  Each id can be collected once: TTR_ERR_ARG for an unknown or already
 * collected id, and for all but one of several threads waiting on the same id.  Returns the
 * request's own status (its error text is in out->message). */
int ttr_server_wait(ttr_server* srv, int64_t id, ttr_server_result* out);

void ttr_server_result_free(ttr_server_result* res);

/* Counters of the server (any thread). */
int ttr_server_get_stats(ttr_server* srv, ttr_server_stats* out);

/* Let the running and queued requests finish, join the workers and release the server.
 * Results not waited for are freed. */
void ttr_server_destroy(ttr_server* srv);

/* Release what a successful call allocated (device arena on `stream`, host arrays) and zero
 * *out.  Safe on a zeroed or already freed result. */
void ttr_free(ttr_result* out, void* stream);

/* Static description of a status code. */
const char* ttr_strerror(int status);

/* Last error message of the calling host thread (CUDA error text, argument problem). */
const char* ttr_last_error(void);

/* Gaussian sketch block Omega_k(:, col0:col1) as produced on the device (Sec. 3.1), written
 * row-major [i][j - col0] to the DEVICE buffer `dst` (n_k * (col1 - col0) doubles, values on
 * the grid 2^-20).  For parity tests of the sketch stream. */
int ttr_sketch_omega(uint64_t seed, int32_t k, int64_t n_k, int64_t col0, int64_t col1,
                     double* dst, void* stream);

/* Right-to-left KRP partial contractions (Algorithm 3, Eqs. (3.1)-(3.3)) on sketch columns
 * [col0, col1), for k = d..t (1-based, 2 <= t <= d).  W[k-1] (k = t..d) are DEVICE buffers of
 * r[k-1] * (col1 - col0) doubles, row-major [a][j - col0]; W[k-1] for k < t are ignored.
 * precision/slices as in ttr_options.  For parity tests of the hot kernel and for callers
 * that want the sketches alone. */
int ttr_partial_contractions(int32_t d, const int64_t* n, const int64_t* r,
                             const double* const* cores, uint64_t seed, int64_t col0,
                             int64_t col1, int32_t t, int32_t precision, int32_t slices,
                             double* const* W, void* stream);

/* Self-test of the reciprocal square root the block loop's Cholesky factors use (a binary32 seed
 * refined by one third-order Newton-Householder step, in place of an FP64 division and square
 * root): out[i] = 1/sqrt(x[i]) for `count` positive finite doubles, both DEVICE buffers.  No
 * counterpart in the paper; for tests of that arithmetic against a correctly rounded reference. */
int ttr_selftest_rsqrt(const double* x, double* out, int64_t count, void* stream);

/* Self-test of the plane rotation of the one-sided Jacobi SVD (Sec. 2.3: the SVD of the small
 * triangular factor in the deterministic rounding and in the Remark 3.2 pass).  For each i < count,
 * abg[3i..3i+2] = (A2, B2, G): the squared norms of a column pair and their inner product; the
 * result cs_sn[2i..2i+1] = (cs, sn) with zeta = (B2 - A2) / (2 G), t = sign(zeta) / (|zeta| +
 * sqrt(1 + zeta^2)), cs = 1 / sqrt(1 + t^2), sn = cs t, or (1, 0) when G = 0, when
 * |G| <= 1e-15 sqrt(A2 B2) or when A2 and B2 both lie at or below `tiny` (>= 0).  Both arrays are
 * DEVICE buffers (3 count and 2 count doubles); the call returns once the results are written.
 * Returns TTR_ERR_ARG for null pointers, a negative count or tiny. */
int ttr_selftest_jacobi_rotation(const double* abg, double tiny, double* cs_sn, int64_t count, void* stream);

/* The partial contractions of ttr_partial_contractions (arguments, layout of W and results alike,
 * FP64) in the per-core-parallel form of the Conclusion (Sec. 5; ttr_options::rl_percore = 1):
 * all G_k(:, :, j) = sum_i X_k(:, i, :) Omega_k(i, j) for k = t..d in one launch, then
 * W_d(:, j) = G_d(:, 0, j) and W_k(:, j) = G_k(:, :, j) W_{k+1}(:, j) in a second launch with one
 * CTA per sketch column.  Scratch: 8 sum_{k=t..d} r_{k-1} r_k (col1 - col0) bytes (stream-ordered);
 * TTR_ERR_UNSUPPORTED when a rank exceeds 12800 (the chain keeps two vectors per CTA in shared
 * memory).  Synchronizes `stream` before returning. */
int ttr_partial_contractions_percore(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores,
                                     uint64_t seed, int64_t col0, int64_t col1, int32_t t, double* const* W,
                                     void* stream);

/* The partial contractions of Algorithm 3 on the product y = A x (arguments of the operator and the
 * vector as in tt_round_adaptive_matvec; seed, col0, col1, t, precision, slices, stream as in
 * ttr_partial_contractions), computed without forming y's cores: W[k-1] (k = t..d) are DEVICE buffers
 * of p[k-1] r[k-1] x (col1 - col0) doubles, rows (a, b) = a r[k-1] + b.  Synchronizes `stream`. */
int ttr_partial_contractions_matvec(int32_t d, const int64_t* n, const int64_t* m, const int64_t* p,
                                    const double* const* A, const int64_t* r, const double* const* x,
                                    uint64_t seed, int64_t col0, int64_t col1, int32_t t, int32_t precision,
                                    int32_t slices, double* const* W, void* stream);

/* Size of the device array that ttr_partial_contractions_noalloc uses as its scratch. */
#define TTR_STATIC_SCRATCH_BYTES (32u << 20)

/* The FP64 form of ttr_partial_contractions with its scratch in a static device array, for callers
 * that cannot allocate device memory: a host runtime that owns the whole device through its own
 * pool allocator and forbids side allocations, or a code path where an allocation could fail or
 * block.  The paper has no counterpart.
 *   Arguments, layout of W and results are those of ttr_partial_contractions with
 *   precision = TTR_PREC_FP64; the caller passes the inputs and the outputs W.
 *   Scratch: a file-scope device array of TTR_STATIC_SCRATCH_BYTES (32 MiB) that every GPU which
 *   loads the library's device code holds until the process exits.  The call needs
 *   8 * ((d-t+1) * max_{k>=t} n_k + max_{t<=k<d} r_{k-1} n_k) * (col1-col0)
 *   bytes of it and returns TTR_ERR_UNSUPPORTED (message in ttr_last_error) beyond the limit,
 *   before any device work.
 *   Allocates nothing: no cudaMalloc / cudaMallocAsync / cudaFree and no allocating library
 *   routine.  The first call on a device looks up the array's device address there
 *   (cudaGetSymbolAddress, with that device current); make that first call before any stream
 *   capture.
 *   All calls share the array and a call leaves its contents behind: calls whose work overlaps
 *   on the GPU (different streams, different host threads) race on it.  Calls ordered on one
 *   stream are safe.
 *   Unlike the other calls it does not synchronize and copies nothing between host and device:
 *   the mode sizes reach the kernels as kernel parameters.  It returns once its kernels are
 *   enqueued on `stream`, and W is ready when the stream reaches that point. */
int ttr_partial_contractions_noalloc(int32_t d, const int64_t* n, const int64_t* r,
                                     const double* const* cores, uint64_t seed, int64_t col0,
                                     int64_t col1, int32_t t, double* const* W, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TTROUND_H */
