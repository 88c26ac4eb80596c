// Host driver of libttround: argument checking, device buffers, the right-to-left sketch pass,
// the left-to-right sweeps of the fixed-rank and adaptive algorithms, the deterministic
// baseline and the C-ABI entry points.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "engine.cuh"
#include "ttr_internal.cuh"

namespace ttr {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// Stream-ordered allocations come from a memory pool of the library's own, one per device, which
// keeps up to kPoolKeepBytes of freed memory for the next call instead of handing it back to the
// driver at every synchronization (the default pool's release threshold is 0).  The pool is
// private to this process and this library; it changes no device setting.
static constexpr uint64_t kPoolKeepBytes = 8ull << 30;

cudaMemPool_t library_pool(cudaStream_t stream) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  (void)stream;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = kPoolKeepBytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

int Ctx::alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = library_pool(stream);
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, stream) : cudaMallocAsync(p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    *p = nullptr;
    return TTR_ERR_OOM;
  }
  owned.push_back(*p);
  return TTR_OK;
}

void Ctx::prof_begin() {
  const char* env = getenv("TTR_PROFILE");
  profiling = env && env[0] == '1';
  if (profiling) {
    cudaEventCreate(&prof_start);
    cudaEventRecord(prof_start, stream);
  }
}

void Ctx::prof_report() {
  if (!profiling || prof.empty()) return;
  cudaStreamSynchronize(stream);
  struct Acc {
    int n = 0;
    double ms = 0.0;
  };
  std::vector<std::pair<std::string, Acc>> acc;
  cudaEvent_t prev = prof_start;
  double total = 0.0;
  for (auto& pe : prof) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, prev, pe.second);
    total += ms;
    auto it = std::find_if(acc.begin(), acc.end(), [&](const std::pair<std::string, Acc>& a) { return a.first == pe.first; });
    if (it == acc.end()) {
      acc.push_back({pe.first, Acc{}});
      it = acc.end() - 1;
    }
    it->second.n++;
    it->second.ms += ms;
    prev = pe.second;
  }
  std::sort(acc.begin(), acc.end(), [](const std::pair<std::string, Acc>& a, const std::pair<std::string, Acc>& b) {
    return a.second.ms > b.second.ms;
  });
  fprintf(stderr, "[ttr profile] %zu launches, %.3f ms between first and last launch\n", prof.size(), total);
  for (auto& a : acc)
    fprintf(stderr, "[ttr profile] %-22s n=%5d  %9.3f ms  %5.1f%%  %8.2f us/launch\n", a.first.c_str(), a.second.n,
            a.second.ms, 100.0 * a.second.ms / std::max(total, 1e-9), 1e3 * a.second.ms / a.second.n);
  if (ac_prof) {
    static const char* names[] = {"stage rows", "first block QR", "fresh Q^T S", "residual (local)",
                                  "reduce B + estimate", "QR 1 (copy, apply)", "reorth (local sub)",
                                  "QR 2 (apply)", "write back", "(barrier waits)", "reduce B (local sums)",
                                  "QR 1 (factor)", "reorth (local Gram)", "reorth (reduction)",
                                  "reorth (G - C^T C)", "QR 2 (factor)", "QR 2 (next P)"};
    constexpr int NPH = (int)(sizeof(names) / sizeof(names[0]));
    unsigned long long cyc[NPH] = {};
    cudaMemcpy(cyc, ac_prof, sizeof(cyc), cudaMemcpyDeviceToHost);
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const double mhz = khz > 0 ? khz / 1e3 : 2070.0;
    for (int i = 0; i < NPH; ++i)
      fprintf(stderr, "[ttr profile]   adaptive_core %-22s %9.3f ms (CTA 0, %.0f MHz)\n", names[i], cyc[i] / mhz / 1e3,
              mhz);
  }
  if (tc_prof) {
    static const char* modes[] = {"plain", "atomic", "partial contraction"};
    static const char* names[] = {"setup", "row scan", "producer chunks", "MMA drain", "epilogue", "(MMA issue loop)"};
    unsigned long long cyc[18] = {};
    cudaMemcpy(cyc, tc_prof, sizeof(cyc), cudaMemcpyDeviceToHost);
    for (int m = 0; m < 3; ++m)
      for (int i = 0; i < 6; ++i)
        if (cyc[m * 6 + i])
          fprintf(stderr, "[ttr profile]   sliced %-20s %-18s %9.3f ms (CTA 0, cycles / 2070 MHz)\n", modes[m], names[i],
                  cyc[m * 6 + i] / 2070.0 / 1e3);
  }
  for (auto& pe : prof) cudaEventDestroy(pe.second);
  cudaEventDestroy(prof_start);
  prof.clear();
  profiling = false;
}

int Ctx::check_launch(const char* what) {
  ++launches;
  if (profiling) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, stream);
    prof.push_back({what, e});
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return TTR_ERR_CUDA;
  }
  return TTR_OK;
}

void Ctx::time_begin(int kind) {
  if (!timing) return;
  KernelTime t{nullptr, nullptr, kind, 0.0};
  cudaEventCreate(&t.a);
  cudaEventCreate(&t.b);
  cudaEventRecord(t.a, stream);
  ktimes.push_back(t);
}

void Ctx::time_end(double work) {
  if (!timing || ktimes.empty()) return;
  cudaEventRecord(ktimes.back().b, stream);
  ktimes.back().work = work;
}

void Ctx::time_collect(ttr_result* out) {
  for (auto& t : ktimes) {
    float ms = 0.f;
    if (out && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      if (t.kind == KT_BLOCK_LOOP) {
        out->ms_block_loop += ms;
        out->flops_block_loop += t.work;
        out->n_block_loop++;
      } else {
        out->ms_rl_kernel += ms;
        out->bytes_rl_kernel += t.work;
        out->n_rl_kernel++;
      }
    }
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  ktimes.clear();
}

int Ctx::workspace() {
  if (ws) return TTR_OK;
  TTR_CHECK(alloc_t(&ws, 128 * 1024));
  TTR_CHECK(alloc_t(&ws_ticket, 4));
  TTR_CUDA(cudaMemsetAsync(ws_ticket, 0, 4 * sizeof(unsigned), stream));
  return TTR_OK;
}

void Ctx::release() {
  time_collect(nullptr);
  for (void* p : owned) cudaFreeAsync(p, stream);
  owned.clear();
}

// Hand an allocation to the caller: it is no longer freed with the context.
static void disown(Ctx& c, void* p) {
  auto it = std::find(c.owned.begin(), c.owned.end(), p);
  if (it != c.owned.end()) c.owned.erase(it);
}

// ----------------------------------------------------------------------------- validation
struct TT {
  int d;
  const int64_t* n;
  const int64_t* r;
  const double* const* cores;
};

static int validate(const TT& X) {
  if (X.d < 2 || X.d > TTR_MAX_D) return set_error("d must be in [2, TTR_MAX_D]"), TTR_ERR_ARG;
  if (!X.n || !X.r || !X.cores) return set_error("n, r and cores must be non-null"), TTR_ERR_ARG;
  if (X.r[0] != 1 || X.r[X.d] != 1) return set_error("r[0] and r[d] must be 1"), TTR_ERR_ARG;
  for (int k = 0; k < X.d; ++k) {
    if (X.n[k] < 1) return set_error("mode sizes must be >= 1"), TTR_ERR_ARG;
    if (X.r[k + 1] < 1) return set_error("ranks must be >= 1"), TTR_ERR_ARG;
    if (!X.cores[k]) return set_error("null core pointer"), TTR_ERR_ARG;
    if (((uintptr_t)X.cores[k]) & 7) return set_error("core pointers must be 8-byte aligned"), TTR_ERR_ARG;
    const double big = (double)X.r[k] * (double)X.n[k] * (double)X.r[k + 1];
    if (big > 9.0e15) return set_error("core too large"), TTR_ERR_ARG;
  }
  return TTR_OK;
}

// Input of the right-to-left pass and of the adaptive rounding: one TT, or the sum of TTs that
// share d and the mode sizes, never formed (Remark 3.3).  R are the ranks of the formal sum, and
// off[i][k] is the first index of summand i in bond k of the formal sum (its rows of W_{k+1}, its
// columns of V(Y_k)); the outer bonds (k = 0, d) are shared.
// An operator-applied TT vector y = A x never formed (matvec.cu): operator cores A_k
// (p_{k-1} x n_k x m_k x p_k, [a][i][j][g]) and vector cores x_k (r_{k-1} x m_k x r_k).
struct Matvec {
  const int64_t* m = nullptr;        // input mode sizes (d)
  const int64_t* p = nullptr;        // operator ranks (d+1)
  const double* const* A = nullptr;  // operator cores (device)
  const int64_t* r = nullptr;        // vector ranks (d+1)
  const double* const* x = nullptr;  // vector cores (device)
};

struct SumTT {
  int d = 0;
  const int64_t* n = nullptr;
  const Matvec* mv = nullptr;        // set: the input is y = A x (parts empty, R = p r)
  std::vector<TT> parts;
  std::vector<int64_t> R;
  std::vector<std::vector<int64_t>> off;
  bool single() const { return parts.size() == 1; }
  TT shape() const { return TT{d, n, R.data(), nullptr}; }   // sizes of the formal sum only
  int64_t part_rank_max(int k) const {
    int64_t m = 1;
    for (const TT& P : parts) m = std::max(m, P.r[k]);
    return m;
  }
};

static SumTT single_sum(const TT& X) {
  SumTT S;
  S.d = X.d;
  S.n = X.n;
  S.parts.assign(1, X);
  S.R.assign(X.r, X.r + X.d + 1);
  S.off.assign(1, std::vector<int64_t>(X.d + 1, 0));
  return S;
}

static int make_sum(int32_t s, int32_t d, const int64_t* n, const int64_t* const* r, const double* const* const* cores,
                    SumTT& S) {
  if (s < 1 || s > TTR_MAX_SUMMANDS) return set_error("number of summands must be in [1, TTR_MAX_SUMMANDS]"), TTR_ERR_ARG;
  if (!r || !cores) return set_error("r and cores must be non-null"), TTR_ERR_ARG;
  S = SumTT{};
  S.d = d;
  S.n = n;
  for (int i = 0; i < s; ++i) {
    if (!r[i] || !cores[i]) return set_error("null rank or core array of a summand"), TTR_ERR_ARG;
    TT P{d, n, r[i], cores[i]};
    TTR_CHECK(validate(P));
    S.parts.push_back(P);
  }
  S.R.assign(d + 1, 1);
  S.off.assign(s, std::vector<int64_t>(d + 1, 0));
  for (int k = 1; k < d; ++k) {
    int64_t acc = 0;
    for (int i = 0; i < s; ++i) {
      S.off[i][k] = acc;
      acc += r[i][k];
    }
    S.R[k] = acc;
  }
  for (int k = 0; k < d; ++k)
    if ((double)S.R[k] * (double)n[k] * (double)S.R[k + 1] > 9.0e15) return set_error("formal sum too large"), TTR_ERR_ARG;
  return TTR_OK;
}

// The operator-applied input y = A x: checks the operator and vector cores and sets the ranks of y.
static int make_matvec(int32_t d, const int64_t* n, const int64_t* m, const int64_t* p, const double* const* A,
                       const int64_t* r, const double* const* x, Matvec& mv, SumTT& S) {
  if (d < 2 || d > TTR_MAX_D) return set_error("d must be in [2, TTR_MAX_D]"), TTR_ERR_ARG;
  if (!n || !m || !p || !A || !r || !x) return set_error("null operator or vector argument"), TTR_ERR_ARG;
  if (p[0] != 1 || p[d] != 1 || r[0] != 1 || r[d] != 1)
    return set_error("outer operator and vector ranks must be 1"), TTR_ERR_ARG;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || m[k] < 1 || p[k + 1] < 1 || r[k + 1] < 1) return set_error("sizes and ranks must be >= 1"), TTR_ERR_ARG;
    if (!A[k] || !x[k] || (((uintptr_t)A[k]) & 7) || (((uintptr_t)x[k]) & 7))
      return set_error("core pointers must be non-null and 8-byte aligned"), TTR_ERR_ARG;
    const double big = (double)p[k] * r[k] * (double)n[k] * (double)p[k + 1] * r[k + 1];
    if (big > 9.0e15 || (double)p[k] * n[k] * (double)m[k] * p[k + 1] > 9.0e15) return set_error("core too large"), TTR_ERR_ARG;
  }
  mv = Matvec{m, p, A, r, x};
  S = SumTT{};
  S.d = d;
  S.n = n;
  S.mv = &mv;
  S.R.assign(d + 1, 1);
  for (int k = 1; k < d; ++k) S.R[k] = p[k] * r[k];
  return TTR_OK;
}

static int64_t block_size(int64_t rbar, int64_t block, double frac) {
  int64_t b = block > 0 ? block : (int64_t)ceil((double)rbar * frac - 1e-9);
  return std::max<int64_t>(1, std::min<int64_t>(rbar, b));
}

static double dsync_read(Ctx& c, const double* dptr, int* status) {
  double v = 0.0;
  cudaError_t e = cudaMemcpyAsync(&v, dptr, sizeof(double), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    set_error(std::string("device read: ") + cudaGetErrorString(e));
    *status = TTR_ERR_CUDA;
  }
  return v;
}

static int isync_read(Ctx& c, const int* dptr, int* status) {
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, dptr, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) {
    set_error(std::string("device read: ") + cudaGetErrorString(e));
    *status = TTR_ERR_CUDA;
  }
  return v;
}

// Device-side bounded waits record failures in c.d_flags; report them once per call.
static int check_device_flags(Ctx& c) {
  if (!c.d_flags) return TTR_OK;
  int st = TTR_OK;
  const int v = isync_read(c, c.d_flags, &st);
  if (st != TTR_OK) return st;
  if (v) return set_error("a bounded device wait ran out"), TTR_ERR_TIMEOUT;
  return TTR_OK;
}

// ----------------------------------------------------------------------------- QR
// Thin QR of the m x b row-major matrix X (leading dimension ldx), in place: X <- Q.
// CholeskyQR3: three CholeskyQR passes.  Two passes orthonormalise a block of condition up to
// ~1e8; a numerically rank-deficient block (a sketch wider than the rank it has, as in a fixed
// rank above the true rank) leaves the completing directions of the second pass orthonormal only
// to O(1), and the third pass, on a block that is now near-orthonormal, restores them.  If a
// Cholesky pivot breaks down, shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto,
// Yanagisawa 2020) from the saved input.  Scratch: tmp and save (m x b, ld b), G and Rinv
// (b x b, ld b), dscal (>= 2 doubles), dflag (1 int).
struct QrWork {
  double* tmp = nullptr;
  double* save = nullptr;
  double* G = nullptr;
  double* Rinv = nullptr;
  double* dscal = nullptr;
  int* dflag = nullptr;
};

// out (m x b) = X R^{-1} for R^{-1} upper triangular (b x b, leading dimension b).  Wide, tall
// products in sliced form run on the tensor cores at 8 slices, whose error bound is that of an FP64
// product (below 64 columns the FP64 kernel is the faster one).
static int apply_rinv(Ctx& c, const Engine& E, const double* X, int64_t ldx, int64_t m, int64_t b, const double* Rinv,
                      double* out, int64_t ldo) {
  if (E.sliced() && b > 64 && (double)m * b * b >= kSlicedProjectWork) {
    const int st = tc_gemm_rowmajor(c, kMaxSlices, X, ldx, m, b, Rinv, b, b, out, ldo);
    if (st != TTR_ERR_UNSUPPORTED) return st;
  }
  return gemm_nn_small(c, X, ldx, Rinv, b, m, b, b, out, ldo, 1.0, 0.0);
}

static int chol_pass(Ctx& c, const Engine& E, double* X, int64_t ldx, int64_t m, int64_t b, double* out,
                     int64_t ldo, const QrWork& w, const double* shift) {
  if (E.sliced() && b > 32 && (double)m * b * b >= kSlicedProjectWork) {
    // wide, tall blocks in sliced form: the Gram matrix (and X R^{-1}, see apply_rinv) on the tensor
    // cores at 8 slices (FP64-accurate products); the Cholesky factorization itself stays FP64
    const int st = tc_gemm_tn(c, kMaxSlices, X, ldx, m, b, X, ldx, b, w.G, b, 1);
    if (st == TTR_OK) {
      TTR_CHECK(chol_inv(c, w.G, b, b, shift, w.Rinv, w.dflag));
      return apply_rinv(c, E, X, ldx, m, b, w.Rinv, out, ldo);
    }
    if (st != TTR_ERR_UNSUPPORTED) return st;
  }
  if (b <= 32) {
    // Gram, Cholesky and 1/diag in one kernel (w.G holds R, w.Rinv the inverse diagonal), then
    // a row-parallel triangular solve
    TTR_CHECK(gram_reduce(c, X, ldx, X, ldx, m, b, b, nullptr, 0, 1, shift, w.G, w.Rinv, w.dflag, nullptr));
    return tri_solve(c, X, ldx, m, b, w.G, w.Rinv, out, ldo);
  }
  TTR_CHECK(gram_tn(c, X, ldx, X, ldx, m, b, b, w.G, b));                 // G = X^T X
  TTR_CHECK(chol_inv(c, w.G, b, b, shift, w.Rinv, w.dflag));
  return apply_rinv(c, E, X, ldx, m, b, w.Rinv, out, ldo);                 // out = X R^{-1}
}

static int qr_inplace(Ctx& c, const Engine& E, double* X, int64_t ldx, int64_t m, int64_t b, const QrWork& w) {
  if (b <= 0) return TTR_OK;
  if (b > m) return set_error("qr: more columns than rows"), TTR_ERR_ARG;
  TTR_CUDA(cudaMemsetAsync(w.dflag, 0, sizeof(int), c.stream));
  TTR_CHECK(copy2d(c, w.save, b, X, ldx, m, b));
  TTR_CHECK(chol_pass(c, E, w.save, b, m, b, w.tmp, b, w, nullptr));
  TTR_CHECK(chol_pass(c, E, w.tmp, b, m, b, X, ldx, w, nullptr));
  TTR_CHECK(chol_pass(c, E, X, ldx, m, b, w.tmp, b, w, nullptr));
  TTR_CHECK(copy2d(c, X, ldx, w.tmp, b, m, b));
  int st = TTR_OK;
  const int bad = isync_read(c, w.dflag, &st);
  if (st != TTR_OK) return st;
  if (!bad) return TTR_OK;
  // shifted CholeskyQR3: shift = 11 (m b + b (b + 1)) u ||X||_F^2  (||X||_2 <= ||X||_F)
  TTR_CUDA(cudaMemsetAsync(w.dflag, 0, sizeof(int), c.stream));
  TTR_CUDA(cudaMemsetAsync(w.dscal, 0, 2 * sizeof(double), c.stream));
  TTR_CHECK(sumsq(c, w.save, m, b, b, 1, w.dscal));
  const double fro2 = dsync_read(c, w.dscal, &st);
  if (st != TTR_OK) return st;
  if (!(fro2 > 0.0) || !isfinite(fro2)) return set_error("qr: zero or non-finite input"), TTR_ERR_QR_BREAKDOWN;
  const double sh = 11.0 * ((double)m * b + (double)b * (b + 1)) * 1.1102230246251565e-16 * fro2;
  TTR_CUDA(cudaMemcpyAsync(w.dscal + 1, &sh, sizeof(double), cudaMemcpyHostToDevice, c.stream));
  // three passes that keep the saved input intact: save -> tmp (shifted) -> X -> tmp -> X
  TTR_CHECK(chol_pass(c, E, w.save, b, m, b, w.tmp, b, w, w.dscal + 1));
  TTR_CHECK(chol_pass(c, E, w.tmp, b, m, b, X, ldx, w, nullptr));
  TTR_CHECK(chol_pass(c, E, X, ldx, m, b, w.tmp, b, w, nullptr));
  TTR_CHECK(copy2d(c, X, ldx, w.tmp, b, m, b));
  const int bad2 = isync_read(c, w.dflag, &st);
  if (st != TTR_OK) return st;
  if (!bad2) return TTR_OK;
  // Exactly rank-deficient input (more sketch columns than the rank of the sketched matrix):
  // any orthonormal completion of its range is a valid thin-QR factor, and the completion
  // directions are orthogonal to the range, so they do not change the projected tensor.
  // Lift the deficiency with a seeded Gaussian perturbation of relative size 1e-13 and
  // repeat shifted CholeskyQR3 (the perturbed matrix has condition number ~1e13).
  TTR_CUDA(cudaMemsetAsync(w.dflag, 0, sizeof(int), c.stream));
  const double eps = 1e-13 * sqrt(fro2 / ((double)m * b));
  const double sh2 = sh * (1.0 + 1e-26 * (double)m * b);
  double hv[2] = {eps, sh2};
  TTR_CUDA(cudaMemcpyAsync(w.dscal + 2, hv, 2 * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  TTR_CHECK(add_gaussian(c, w.save, m, b, b, w.dscal + 2, 0x5eed5eed5eed5eedULL));
  TTR_CHECK(chol_pass(c, E, w.save, b, m, b, w.tmp, b, w, w.dscal + 3));
  TTR_CHECK(chol_pass(c, E, w.tmp, b, m, b, X, ldx, w, nullptr));
  TTR_CHECK(chol_pass(c, E, X, ldx, m, b, w.tmp, b, w, nullptr));
  TTR_CHECK(copy2d(c, X, ldx, w.tmp, b, m, b));
  const int bad3 = isync_read(c, w.dflag, &st);
  if (st != TTR_OK) return st;
  if (bad3) return set_error("qr: CholeskyQR breakdown after shift and perturbation"), TTR_ERR_QR_BREAKDOWN;
  return TTR_OK;
}

// ----------------------------------------------------------------------------- RL sketch pass
// Algorithm 3 on columns [col0, col1) for k = d..t: W_k(:, col0:col1) with W_k row-major,
// leading dimension ldw.  Omega blocks go to Om (core k at (k-1)*om_stride, ld ldom).
struct Sketch {
  std::vector<double*> W;   // W[k-1] for k = 2..d (index 0 unused)
  int64_t ldw = 0;
  int64_t width = 0;        // columns computed so far
  double* Om = nullptr;
  int* Omi = nullptr;        // 2^20 * Omega as integers, same layout as Om
  int64_t om_stride = 0, ldom = 0;
  double* T = nullptr;      // (max r_{k-1} n_k) x ldw scratch
  int extensions = 0;
  std::vector<BPlanes> wplanes;   // digit planes of W_{k+1}(:, 0:width) made by the first pass (index k)
  bool percore = false;           // per-core-parallel form of the pass (rl_percore)
};

// rl_percore = 2 takes the per-core form up to this much scratch: in FP64 form, where it replaces a
// chain of FP64 GEMM launches; in sliced form only for small shapes, where launch latency dominates
// the chain of tensor-core launches (measured: 2x faster on the 6-core workload, slower from the
// operator-applied vector up)
static constexpr double kPercoreAutoBytesFp64 = 32.0 * 1024 * 1024;
static constexpr double kPercoreAutoBytesSliced = 2.0 * 1024 * 1024;
static bool percore_auto(const Engine& E, double bytes) {
  return bytes <= (E.precision == TTR_PREC_FP64 ? kPercoreAutoBytesFp64 : kPercoreAutoBytesSliced);
}

// Scratch bytes of the per-core-parallel pass on w columns for cores t..d of every summand.
static double percore_bytes(const SumTT& X, int t, int64_t w) {
  double tot = 0.0;
  for (const TT& P : X.parts)
    for (int k = t; k <= X.d; ++k) tot += 8.0 * (double)P.r[k - 1] * (double)P.r[k] * (double)w;
  return tot;
}

// Algorithm 3 on y = A x without forming y's cores (matvec.cu), columns [col0, col1), Omega already
// in s.Om: per core, Ahat = Omega contracted into A_k, Z_g = V(x_k) W_{k+1}(g-th row block), and
// W_k = the (j, g) contraction of the two.
static int rl_pass_matvec(Ctx& c, const Engine& E, const SumTT& X, int64_t col0, int64_t col1, int t, Sketch& s) {
  const Matvec& v = *X.mv;
  const int d = X.d;
  const int64_t w = col1 - col0;
  int64_t amax = 1, zmax = 1;
  for (int k = t; k <= d; ++k) {
    amax = std::max(amax, v.p[k - 1] * v.m[k - 1] * v.p[k] * w);
    zmax = std::max(zmax, v.p[k] * v.r[k - 1] * v.m[k - 1] * w);
  }
  double *Ahat = nullptr, *Z = nullptr;
  TTR_CHECK(c.alloc_t(&Ahat, amax));
  TTR_CHECK(c.alloc_t(&Z, zmax));
  for (int k = d; k >= t; --k) {
    const int64_t p0 = v.p[k - 1], p1 = v.p[k], r0 = v.r[k - 1], r1 = v.r[k], n = X.n[k - 1], m = v.m[k - 1];
    const double* Om = s.Om + (int64_t)(k - 1) * s.om_stride;
    // Ahat(a, (j, g), l) = sum_i A_k(a, i, (j, g)) Omega_k(i, l)
    TTR_CHECK(mv_ahat(c, v.A[k - 1], p0, n, m, p1, Om, s.ldom, w, Ahat));
    if (k == d) {
      TTR_CHECK(mv_reduce(c, Ahat, nullptr, v.x[d - 1], p0, r0, m, 1, w, s.W[d - 1] + col0, s.ldw));
      continue;
    }
    for (int64_t gi = 0; gi < p1; ++gi) {   // Z_g = V(x_k) W_{k+1}(g r_k : (g+1) r_k, :)
      Gemm z;
      z.M = r0 * m; z.N = w; z.K = r1;
      z.A = v.x[k - 1]; z.sam = r1; z.sak = 1;
      z.B = s.W[k] + col0 + gi * r1 * s.ldw; z.sbk = s.ldw; z.sbn = 1;
      z.C = Z + gi * r0 * m * w; z.scm = w; z.scn = 1;
      TTR_CHECK(E.sketch(c, z));
    }
    TTR_CHECK(mv_reduce(c, Ahat, Z, nullptr, p0, r0, m, p1, w, s.W[k - 1] + col0, s.ldw));
  }
  return TTR_OK;
}

// The per-core-parallel form (Conclusion, Sec. 5) of Algorithm 3 on columns [col0, col1), FP64:
// all G_k in one launch, then the column-wise chain in another.
static int rl_pass_percore(Ctx& c, const SumTT& X, int64_t col0, int64_t col1, int t, Sketch& s) {
  const int d = X.d;
  const int64_t w = col1 - col0;
  const int ns = (int)X.parts.size();
  double* G = nullptr;
  TTR_CHECK(c.alloc_t(&G, (int64_t)ceil(percore_bytes(X, t, w) / 8.0)));
  std::vector<PcCore> tab;
  tab.reserve((size_t)ns * (d - t + 1));
  int64_t goff = 0;
  for (int p = 0; p < ns; ++p) {
    const TT& P = X.parts[p];
    for (int k = t; k <= d; ++k) {
      PcCore e;
      e.X = P.cores[k - 1];
      e.r0 = P.r[k - 1]; e.n = X.n[k - 1]; e.r1 = P.r[k];
      e.Om = s.Om + (int64_t)(k - 1) * s.om_stride; e.ldom = s.ldom;
      e.G = G + goff;
      e.W = s.W[k - 1] + X.off[p][k - 1] * s.ldw + col0; e.ldw = s.ldw;
      goff += e.r0 * e.r1 * w;
      tab.push_back(e);
    }
  }
  return rl_percore(c, tab, ns, w);
}

static int rl_pass(Ctx& c, const Engine& E, const SumTT& X, uint64_t seed, int64_t col0, int64_t col1, int t,
                   Sketch& s) {
  const int d = X.d;
  const int64_t w = col1 - col0;
  if (w <= 0) return TTR_OK;
  TTR_CHECK(omega_fill(c, seed, t, d, X.n, col0, col1, s.Om + (int64_t)(t - 1) * s.om_stride,
                       s.Omi + (int64_t)(t - 1) * s.om_stride, s.om_stride, s.ldom));
  if (X.mv) return rl_pass_matvec(c, E, X, col0, col1, t, s);
  if (s.percore) return rl_pass_percore(c, X, col0, col1, t, s);
  // digit planes of W_{k+1} (all summands' rows) are kept for the sketch
  const bool keep = col0 == 0;
  if (keep) s.wplanes.assign(d + 1, BPlanes{});
  // each summand with the same Omega, into its own rows of the stacked W_k (Remark 3.3)
  const int ns = (int)X.parts.size();
  for (int p0 = 0; p0 < ns; p0 += kMaxGroup) {   // W_d = H(X_d) Omega_d  (r_{d-1} x n_d) (n_d x w)
    const int ng = std::min(kMaxGroup, ns - p0);
    const double* A[kMaxGroup];
    int64_t M[kMaxGroup];
    double* C[kMaxGroup];
    for (int g = 0; g < ng; ++g) {
      A[g] = X.parts[p0 + g].cores[d - 1];
      M[g] = X.parts[p0 + g].r[d - 1];
      C[g] = s.W[d - 1] + X.off[p0 + g][d - 1] * s.ldw + col0;
    }
    TTR_CHECK(E.last_core_group(c, ng, A, M, X.n[d - 1], s.Om + (int64_t)(d - 1) * s.om_stride, s.ldom, w, C, s.ldw));
  }
  for (int k = d - 1; k >= t; --k) {
    const double* Om = s.Om + (int64_t)(k - 1) * s.om_stride;
    const int* Omi = s.Omi + (int64_t)(k - 1) * s.om_stride;
    if (X.single()) {
      const TT& P = X.parts[0];
      TTR_CHECK(E.rl_step(c, P.cores[k - 1], P.r[k - 1], X.n[k - 1], P.r[k], s.W[k] + col0, s.ldw, Om, Omi, s.ldom, w,
                          s.W[k - 1] + col0, s.ldw, s.T, keep ? &s.wplanes[k] : nullptr));
      continue;
    }
    // the summands of one core, kMaxGroup per launch
    for (int p0 = 0; p0 < ns; p0 += kMaxGroup) {
      const int ng = std::min(kMaxGroup, ns - p0);
      const double* Xk[kMaxGroup];
      int64_t r0[kMaxGroup], r1[kMaxGroup], offn[kMaxGroup], offo[kMaxGroup];
      for (int g = 0; g < ng; ++g) {
        const TT& P = X.parts[p0 + g];
        Xk[g] = P.cores[k - 1];
        r0[g] = P.r[k - 1];
        r1[g] = P.r[k];
        offn[g] = X.off[p0 + g][k];
        offo[g] = X.off[p0 + g][k - 1];
      }
      // planes are kept when one launch takes every summand (they then cover all rows of W_{k+1})
      TTR_CHECK(E.rl_step_group(c, ng, Xk, r0, X.n[k - 1], r1, s.W[k] + col0, s.ldw, X.R[k], offn, Om, Omi, s.ldom,
                                w, s.W[k - 1] + col0, s.ldw, offo, s.T, keep && ns <= kMaxGroup ? &s.wplanes[k] : nullptr));
    }
  }
  return TTR_OK;
}

static int sketch_alloc(Ctx& c, const TT& X, int64_t wcap, Sketch& s) {
  const int d = X.d;
  int64_t nmax = 1, rowsmax = 1, tot = 0;
  for (int k = 0; k < d; ++k) {
    nmax = std::max(nmax, X.n[k]);
    rowsmax = std::max(rowsmax, X.r[k] * X.n[k]);
    if (k >= 1) tot += X.r[k] * wcap;
  }
  s.ldw = wcap;
  s.W.assign(d, nullptr);
  double* base = nullptr;
  TTR_CHECK(c.alloc_t(&base, std::max<int64_t>(tot, 1)));
  int64_t off = 0;
  for (int k = 2; k <= d; ++k) {
    s.W[k - 1] = base + off;
    off += X.r[k - 1] * wcap;
  }
  s.ldom = wcap;
  s.om_stride = nmax * wcap;
  TTR_CHECK(c.alloc_t(&s.Om, (int64_t)d * s.om_stride));
  TTR_CHECK(c.alloc_t(&s.Omi, (int64_t)d * s.om_stride));
  TTR_CHECK(c.alloc_t(&s.T, rowsmax * wcap));
  return TTR_OK;
}

// ----------------------------------------------------------------------------- result helpers
static void result_zero(ttr_result* out) {
  if (out) memset(out, 0, sizeof(*out));
}

struct Timer {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  Timer() {
    for (auto& x : e) cudaEventCreate(&x);
  }
  ~Timer() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  void rec(int i, cudaStream_t s) { cudaEventRecord(e[i], s); }
  float ms(int a, int b) {
    float v = 0.f;
    cudaEventElapsedTime(&v, e[a], e[b]);
    return v;
  }
};

// Allocates the output arena (worst case: the input size) and host arrays.
static int result_alloc(Ctx& c, const TT& X, ttr_result* out) {
  int64_t tot = 0;
  for (int k = 0; k < X.d; ++k) tot += X.r[k] * X.n[k] * X.r[k + 1];
  double* arena = nullptr;
  TTR_CHECK(c.alloc_t(&arena, tot));
  out->arena = arena;
  out->d = X.d;
  out->ranks = (int64_t*)calloc(X.d + 1, sizeof(int64_t));
  out->cores = (double**)calloc(X.d, sizeof(double*));
  if (!out->ranks || !out->cores) return set_error("host allocation"), TTR_ERR_OOM;
  return TTR_OK;
}

static void result_host_free(ttr_result* out) {
  free(out->ranks);
  free(out->cores);
  free(out->estimates);
  free(out->est_core);
  out->ranks = nullptr;
  out->cores = nullptr;
  out->estimates = nullptr;
  out->est_core = nullptr;
}

// ----------------------------------------------------------------------------- LR sweep buffers
struct Sweep {
  double* Y[2] = {nullptr, nullptr};  // current unprojected core H(Y_k) and the next one
  double* Q = nullptr;                 // rows x qcap
  int64_t qcap = 0;
  double* S = nullptr;                 // rows x bcap
  double* P = nullptr;                 // rmax x bcap
  double* M = nullptr;                 // rmax x rmax
  double* ytmp = nullptr;              // one summand's block of the next core (sums only)
  double* ycore = nullptr;             // one formed core of y = A x (operator-applied input only)
  int64_t bcap = 0;
  QrWork qr;
};

static int sweep_alloc(Ctx& c, const TT& X, int64_t bcap, Sweep& s) {
  int64_t cmax = 1, rowsmax = 1, rmax = 1;
  for (int k = 0; k < X.d; ++k) {
    cmax = std::max(cmax, X.r[k] * X.n[k] * X.r[k + 1]);
    rowsmax = std::max(rowsmax, X.r[k] * X.n[k]);
    rmax = std::max(rmax, X.r[k + 1]);
  }
  s.qcap = rmax;
  s.bcap = std::max<int64_t>(1, bcap);
  TTR_CHECK(c.alloc_t(&s.Y[0], cmax));
  TTR_CHECK(c.alloc_t(&s.Y[1], cmax));
  TTR_CHECK(c.alloc_t(&s.Q, rowsmax * s.qcap));
  TTR_CHECK(c.alloc_t(&s.S, rowsmax * s.bcap));
  TTR_CHECK(c.alloc_t(&s.P, rmax * s.bcap));
  TTR_CHECK(c.alloc_t(&s.M, rmax * rmax));
  const int64_t qb = std::max(s.bcap, rmax);
  TTR_CHECK(c.alloc_t(&s.qr.tmp, rowsmax * qb));
  TTR_CHECK(c.alloc_t(&s.qr.save, rowsmax * qb));
  TTR_CHECK(c.alloc_t(&s.qr.G, qb * qb));
  TTR_CHECK(c.alloc_t(&s.qr.Rinv, qb * qb));
  TTR_CHECK(c.alloc_t(&s.qr.dscal, 8));
  TTR_CHECK(c.alloc_t(&s.qr.dflag, 4));
  return TTR_OK;
}

// M = Q^T Z  (c x cols), then Ynext = M H(X_{k+1})  (c x n r).  For a sum of TTs, M splits into
// the column blocks M^(i) of the summands and the next core is projected summand by summand:
// M^(i) H(X_{k+1}^(i)) fills the columns of summand i in the right bond of Ynext, and at the last
// core (shared right bond 1) the summands' products add up (Appendix D).
// Zd: for a sum, the summands' last cores stacked (R_{d-1} x n_d, the formal sum's last core)
static int project_next(Ctx& c, const Engine& E, const Sweep& s, const double* Z, int64_t rows, int64_t cols,
                        int64_t ccols, const SumTT& X, int k, double* Ynext, const double* Zd = nullptr) {
  TTR_CHECK(E.left_project(c, s.Q, s.qcap, Z, rows, cols, ccols, s.M));
  const int64_t nk = X.n[k];
  if (X.mv) {
    // one core of y = A x at a time: y_{k+1} into scratch, then M y_{k+1}
    const Matvec& v = *X.mv;
    TTR_CHECK(mv_form(c, v.A[k], v.p[k], nk, v.m[k], v.p[k + 1], v.x[k], v.r[k], v.r[k + 1], s.ycore));
    return E.project(c, s.M, cols, ccols, cols, s.ycore, nk * X.R[k + 1], Ynext);
  }
  if (X.single()) {
    // H(X_{k+1}) is cols x (n_{k+1} r_{k+2}), row-major
    return E.project(c, s.M, cols, ccols, cols, X.parts[0].cores[k], nk * X.parts[0].r[k + 1], Ynext);
  }
  if (k == X.d - 1 && Zd) return E.project(c, s.M, cols, ccols, cols, Zd, nk, Ynext);   // H(Y_d) = M H(X_d)
  const int ns = (int)X.parts.size();
  // one summand: M^(p) H(X_{k+1}^(p)) through a scratch block into its columns of Ynext, or at the
  // last core added into Ynext
  auto one = [&](int p) -> int {
    const TT& P = X.parts[p];
    const double* Mp = s.M + X.off[p][k];
    if (k == X.d - 1) {
      Gemm g;
      g.M = ccols; g.N = nk; g.K = P.r[k];
      g.A = Mp; g.sam = cols; g.sak = 1;
      g.B = P.cores[k]; g.sbk = nk; g.sbn = 1;
      g.C = Ynext; g.scm = nk; g.scn = 1;
      g.beta = p == 0 ? 0.0 : 1.0;
      return E.small_gemm(c, g);
    }
    const int64_t rn = P.r[k + 1];
    TTR_CHECK(E.project(c, Mp, cols, ccols, P.r[k], P.cores[k], nk * rn, s.ytmp));
    return copy2d(c, Ynext + X.off[p][k + 1], X.R[k + 1], s.ytmp, rn, ccols * nk, rn);
  };
  for (int p0 = 0; p0 < ns; p0 += kMaxGroup) {
    const int ng = std::min(kMaxGroup, ns - p0);
    if (k < X.d - 1) {
      // the chunk's blocks of the next core in one launch, straight into Ynext
      const double* Xn[kMaxGroup];
      int64_t koff[kMaxGroup], K[kMaxGroup], rn[kMaxGroup], yoff[kMaxGroup];
      for (int g = 0; g < ng; ++g) {
        const TT& P = X.parts[p0 + g];
        Xn[g] = P.cores[k];
        koff[g] = X.off[p0 + g][k];
        K[g] = P.r[k];
        rn[g] = P.r[k + 1];
        yoff[g] = X.off[p0 + g][k + 1];
      }
      const int st = E.project_group(c, ng, s.M, cols, ccols, cols, koff, K, Xn, nk, rn, Ynext, X.R[k + 1], yoff);
      if (st != TTR_ERR_UNSUPPORTED) {
        TTR_CHECK(st);
        continue;
      }
    }
    for (int g = 0; g < ng; ++g) TTR_CHECK(one(p0 + g));
  }
  return TTR_OK;
}

// ----------------------------------------------------------------------------- SVD pass (Remark 3.2)
// Right-to-left truncation of the left-orthonormal TT held as out->cores / out->ranks, in place
// in a fresh arena.  Threshold tau (<= 0: none) and optional rank cap.
static int svd_pass_rl(Ctx& c, const Engine& E, ttr_result* out, const int64_t* n, double tau, int64_t max_rank) {
  const int d = out->d;
  int64_t* r = out->ranks;
  int64_t rmax = 1, cmax = 1;
  for (int k = 0; k < d; ++k) {
    rmax = std::max(rmax, r[k + 1]);
    cmax = std::max(cmax, r[k] * n[k] * r[k + 1]);
  }
  // work copies of every core (they shrink), then pack into a new arena
  std::vector<double*> Yc(d);
  for (int k = 0; k < d; ++k) {
    TTR_CHECK(c.alloc_t(&Yc[k], std::max<int64_t>(r[k] * n[k] * r[k + 1], 1)));
    TTR_CUDA(cudaMemcpyAsync(Yc[k], out->cores[k], sizeof(double) * r[k] * n[k] * r[k + 1], cudaMemcpyDeviceToDevice,
                             c.stream));
  }
  double *Ht, *R, *U, *Vt, *sig, *tmp;
  QrWork w;
  TTR_CHECK(c.alloc_t(&Ht, cmax));
  TTR_CHECK(c.alloc_t(&R, rmax * rmax));
  TTR_CHECK(c.alloc_t(&U, rmax * rmax));
  TTR_CHECK(c.alloc_t(&Vt, rmax * rmax));
  TTR_CHECK(c.alloc_t(&sig, rmax));
  TTR_CHECK(c.alloc_t(&tmp, cmax));
  TTR_CHECK(c.alloc_t(&w.tmp, cmax));
  TTR_CHECK(c.alloc_t(&w.save, cmax));
  TTR_CHECK(c.alloc_t(&w.G, rmax * rmax));
  TTR_CHECK(c.alloc_t(&w.Rinv, rmax * rmax));
  TTR_CHECK(c.alloc_t(&w.dscal, 8));
  TTR_CHECK(c.alloc_t(&w.dflag, 4));
  std::vector<double> hs(rmax);
  for (int k = d - 1; k >= 1; --k) {
    const int64_t r0 = r[k], nk = n[k], r1 = r[k + 1];
    const int64_t m = nk * r1;  // rows of H(Y_k)^T
    if (r0 > m) continue;       // cannot be reduced by a thin QR of H^T; keep rank
    // Ht = H(Y_k)^T  (m x r0, row-major ld r0): Ht[(i,c), a] = Y[a][i][c]
    TTR_CHECK(E.transpose(c, Yc[k], r0, m, Ht));
    TTR_CHECK(qr_inplace(c, E, Ht, r0, m, r0, w));             // Ht <- Q  (m x r0)
    // R = Q^T H(Y_k)^T  (r0 x r0)
    Gemm g;
    g.M = r0; g.N = r0; g.K = m;
    g.A = Ht; g.sam = 1; g.sak = r0;
    g.B = Yc[k]; g.sbk = 1; g.sbn = m;                       // H(Y_k)^T(row, a) = Y[a*m + row]
    g.C = R; g.scm = r0; g.scn = 1;
    g.split_k = (int)std::min<int64_t>(std::max<int64_t>(1, m / 256), 64);
    TTR_CHECK(fill_zero(c, R, r0 * r0));
    TTR_CHECK(E.small_gemm(c, g));
    // SVD of R^T = U S Vt: Jacobi on R^T (transpose R into U's storage first)
    TTR_CHECK(E.transpose(c, R, r0, r0, tmp));                // tmp = R^T (r0 x r0)
    TTR_CUDA(cudaMemsetAsync(w.dflag, 0, sizeof(int), c.stream));
    if (r0 >= kJacobiMultiFrom)
      TTR_CHECK(jacobi_svd_multi(c, tmp, r0, r0, sig, U, Vt, w.dflag));
    else
      TTR_CHECK(jacobi_svd(c, tmp, r0, r0, sig, U, Vt, w.dflag));
    TTR_CUDA(cudaMemcpyAsync(hs.data(), sig, sizeof(double) * r0, cudaMemcpyDeviceToHost, c.stream));
    TTR_CUDA(cudaStreamSynchronize(c.stream));
    int64_t rp = r0;
    if (tau > 0.0) {
      // smallest rp >= 1 with sqrt(sum_{i >= rp} s_i^2) <= tau
      std::vector<double> tail(r0 + 1, 0.0);
      for (int64_t i = r0 - 1; i >= 0; --i) tail[i] = tail[i + 1] + hs[i] * hs[i];
      rp = r0;
      for (int64_t q = 1; q <= r0; ++q)
        if (sqrt(tail[q]) <= tau) {
          rp = q;
          break;
        }
    }
    if (max_rank > 0) rp = std::min(rp, max_rank);
    // H(Y_k) <- Vt[:rp] Q^T   (rp x m):  new[p][row] = sum_j Vt[p][j] Q[row][j]
    Gemm h;
    h.M = rp; h.N = m; h.K = r0;
    h.A = Vt; h.sam = r0; h.sak = 1;
    h.B = Ht; h.sbk = 1; h.sbn = r0;
    h.C = tmp; h.scm = m; h.scn = 1;
    TTR_CHECK(E.small_gemm(c, h));
    TTR_CUDA(cudaMemcpyAsync(Yc[k], tmp, sizeof(double) * rp * m, cudaMemcpyDeviceToDevice, c.stream));
    // V(Y_{k-1}) <- V(Y_{k-1}) U[:, :rp] diag(s)  ((r_{k-1} n_{k-1}) x r0) (r0 x rp)
    TTR_CHECK(E.scale_cols(c, U, r0, rp, r0, sig));
    const int64_t rows = r[k - 1] * n[k - 1];
    Gemm v;
    v.M = rows; v.N = rp; v.K = r0;
    v.A = Yc[k - 1]; v.sam = r0; v.sak = 1;
    v.B = U; v.sbk = r0; v.sbn = 1;
    v.C = tmp; v.scm = rp; v.scn = 1;
    TTR_CHECK(E.small_gemm(c, v));
    TTR_CUDA(cudaMemcpyAsync(Yc[k - 1], tmp, sizeof(double) * rows * rp, cudaMemcpyDeviceToDevice, c.stream));
    r[k] = rp;
  }
  // pack into the existing arena (it is at least as large)
  int64_t off = 0;
  double* arena = (double*)out->arena;
  for (int k = 0; k < d; ++k) {
    const int64_t sz = r[k] * n[k] * r[k + 1];
    TTR_CUDA(cudaMemcpyAsync(arena + off, Yc[k], sizeof(double) * sz, cudaMemcpyDeviceToDevice, c.stream));
    out->cores[k] = arena + off;
    off += sz;
  }
  return TTR_OK;
}

// ----------------------------------------------------------------------------- fixed rank
static int round_fixed(const TT& X, int64_t ell, int64_t target, uint64_t seed, const ttr_options& o,
                       cudaStream_t stream, ttr_result* out) {
  if (ell < 1) return set_error("ell must be >= 1"), TTR_ERR_ARG;
  Ctx c;
  c.stream = stream;
  c.prof_begin();
  c.timing = o.kernel_timing != 0;
  c.autotune = o.autotune != 0;
  c.sm_share = o.max_sms;
  Timer tm;
  tm.rec(0, stream);
  Engine E;
  TTR_CHECK(E.init(c, o.precision, o.slices, 0.0));
  const int d = X.d;
  const SumTT XS = single_sum(X);
  if (o.rl_percore < 0 || o.rl_percore > 2) return set_error("rl_percore must be 0, 1 or 2"), TTR_ERR_ARG;
  Sketch s;
  TTR_CHECK(sketch_alloc(c, X, ell, s));
  s.percore = o.rl_percore == 1 || (o.rl_percore == 2 && percore_auto(E, percore_bytes(XS, 2, ell)));
  TTR_CHECK(rl_pass(c, E, XS, seed, 0, ell, 2, s));
  s.width = ell;
  tm.rec(1, stream);
  Sweep w;
  int64_t rmax = 1;
  for (int k = 1; k < d; ++k) rmax = std::max(rmax, X.r[k]);
  TTR_CHECK(sweep_alloc(c, X, std::min(ell, rmax), w));
  TTR_CHECK(result_alloc(c, X, out));
  double* arena = (double*)out->arena;
  int64_t off = 0, lprev = 1;
  const double* Z = X.cores[0];
  int cur = 0;
  out->ranks[0] = 1;
  for (int k = 1; k < d; ++k) {
    const int64_t rows = lprev * X.n[k - 1], cols = X.r[k];
    double right = 1.0;
    for (int j = k; j < d; ++j) right = std::min(right * (double)X.n[j], 1e18);
    int64_t lk = std::min<int64_t>(std::min<int64_t>(ell, rows), cols);
    if ((double)lk > right) lk = (int64_t)right;
    // S = Z W_{k+1}(:, 0:lk) -> Q (ld qcap)
    Gemm g;
    g.M = rows; g.N = lk; g.K = cols;
    g.A = Z; g.sam = cols; g.sak = 1;
    g.B = s.W[k]; g.sbk = s.ldw; g.sbn = 1;
    g.C = w.Q; g.scm = w.qcap; g.scn = 1;
    TTR_CHECK(E.sketch(c, g));
    TTR_CHECK(qr_inplace(c, E, w.Q, w.qcap, rows, lk, w.qr));
    double* Ynext = w.Y[cur];
    TTR_CHECK(project_next(c, E, w, Z, rows, cols, lk, XS, k, Ynext));
    TTR_CHECK(copy2d(c, arena + off, lk, w.Q, w.qcap, rows, lk));
    out->cores[k - 1] = arena + off;
    out->ranks[k] = lk;
    off += rows * lk;
    Z = Ynext;
    cur ^= 1;
    lprev = lk;
  }
  const int64_t last = lprev * X.n[d - 1];
  TTR_CUDA(cudaMemcpyAsync(arena + off, Z, sizeof(double) * last, cudaMemcpyDeviceToDevice, stream));
  out->cores[d - 1] = arena + off;
  out->ranks[d] = 1;
  if (target > 0 && target < ell) TTR_CHECK(svd_pass_rl(c, E, out, X.n, 0.0, target));
  tm.rec(2, stream);
  TTR_CUDA(cudaStreamSynchronize(stream));
  TTR_CHECK(check_device_flags(c));
  out->width = ell;
  out->ms_sketch_rl = tm.ms(0, 1);
  out->ms_sweep_lr = tm.ms(1, 2);
  out->ms_total = tm.ms(0, 2);
  out->kernel_launches = c.launches;
  c.time_collect(out);
  disown(c, out->arena);
  return TTR_OK;
}

// ----------------------------------------------------------------------------- adaptive
// appendix_blocks: the block rule of the sum algorithm in Appendix D when block <= 0 (b_init =
// max_i r_k^(i), initial sketch width max_{i,k} r_k^(i)) instead of the fractions f_init of Sec. 3.3.
static int round_adaptive(const SumTT& X, double tol, int64_t block, uint64_t seed, const ttr_options& o,
                          cudaStream_t stream, ttr_result* out, bool appendix_blocks = false) {
  if (!(tol > 0.0) || !isfinite(tol)) return set_error("tol must be positive and finite"), TTR_ERR_ARG;
  if (block <= 0 && !((appendix_blocks || (o.f_init > 0.0 && o.f_init < 1.0)) && o.f_inc > 0.0 && o.f_inc < 1.0))
    return set_error("f_init and f_inc must lie in (0, 1)"), TTR_ERR_ARG;
  if (o.est_min < 0 || o.est_min > 4096) return set_error("est_min must lie in [0, 4096]"), TTR_ERR_ARG;
  if (!(o.est_safety >= 1.0) || !isfinite(o.est_safety)) return set_error("est_safety must be finite and >= 1"), TTR_ERR_ARG;
  Ctx c;
  c.stream = stream;
  c.prof_begin();
  c.timing = o.kernel_timing != 0;
  c.autotune = o.autotune != 0;
  c.sm_share = o.max_sms;
  Timer tm;
  tm.rec(0, stream);
  const int d = X.d;
  int64_t rmax = 1, rpart = 1;
  for (int k = 1; k < d; ++k) {
    rmax = std::max(rmax, X.R[k]);
    rpart = std::max(rpart, X.part_rank_max(k));
  }
  const bool appendix = appendix_blocks && block <= 0;
  const int64_t w0 = std::max<int64_t>(1, block > 0 ? block
                                                    : appendix ? rpart : (int64_t)ceil((double)rmax * o.f_init - 1e-9));
  const int64_t binc_max = block > 0 ? std::min(block, rmax) : block_size(rmax, 0, o.f_inc);
  const int64_t binit_max = block > 0 ? std::min(block, rmax) : appendix ? rpart : block_size(rmax, 0, o.f_init);
  // residual sketches hold max(b_inc, est_min) columns (reading R16), past col(Q) <= rmax
  const int64_t best_max = std::max<int64_t>(binc_max, o.est_min);
  const int64_t wcap = std::max(w0, rmax + best_max);
  Engine E;
  TTR_CHECK(E.init(c, o.precision, o.slices, tol));
  if (o.rl_percore < 0 || o.rl_percore > 2) return set_error("rl_percore must be 0, 1 or 2"), TTR_ERR_ARG;
  Sketch s;
  TTR_CHECK(sketch_alloc(c, X.shape(), wcap, s));
  s.percore = o.rl_percore == 1 || (o.rl_percore == 2 && percore_auto(E, percore_bytes(X, 2, wcap)));
  // Columns of W are a prefix of one counter-based stream, so how many are drawn up front (and how
  // the rest are appended) never changes a result; draw one tensor-core tile width up front and
  // grow geometrically, which keeps the number of right-to-left passes small.
  int64_t wdev = std::min(wcap, std::max<int64_t>(w0, E.natural_width()));
  if (o.width_hint > 0) wdev = std::min(wcap, std::max(w0, o.width_hint));
  TTR_CHECK(rl_pass(c, E, X, seed, 0, wdev, 2, s));
  s.width = wdev;
  // V(Y_1): the first core, or for a sum the summands' first cores side by side (Appendix D)
  const double* Z1 = X.mv ? nullptr : X.parts[0].cores[0];
  if (X.mv) {
    // V(Y_1) = the first core of y = A x (1 x n_1 x p_1 r_1), formed
    double* z = nullptr;
    TTR_CHECK(c.alloc_t(&z, X.n[0] * X.R[1]));
    const Matvec& v = *X.mv;
    TTR_CHECK(mv_form(c, v.A[0], 1, X.n[0], v.m[0], v.p[1], v.x[0], 1, v.r[1], z));
    Z1 = z;
  } else if (!X.single()) {
    double* z = nullptr;
    TTR_CHECK(c.alloc_t(&z, X.n[0] * X.R[1]));
    for (size_t p = 0; p < X.parts.size(); ++p)
      TTR_CHECK(copy2d(c, z + X.off[p][1], X.R[1], X.parts[p].cores[0], X.parts[p].r[1], X.n[0], X.parts[p].r[1]));
    Z1 = z;
  }
  // for a sum, the last cores stacked: the formal sum's last core, projected in one product
  double* Zd = nullptr;
  if (!X.single() && !X.mv) {
    TTR_CHECK(c.alloc_t(&Zd, X.R[d - 1] * X.n[d - 1]));
    for (size_t p = 0; p < X.parts.size(); ++p)
      TTR_CUDA(cudaMemcpyAsync(Zd + X.off[p][d - 1] * X.n[d - 1], X.parts[p].cores[d - 1],
                               sizeof(double) * X.parts[p].r[d - 1] * X.n[d - 1], cudaMemcpyDeviceToDevice, stream));
  }
  // norm: given, or Eq. (3.6) with the first w0 columns of W_2
  double* dscal = nullptr;
  TTR_CHECK(c.alloc_t(&dscal, 8));
  double nrmx = o.nrmx;
  int st = TTR_OK;
  if (!(nrmx > 0.0)) {
    double* E1 = nullptr;
    TTR_CHECK(c.alloc_t(&E1, X.n[0] * w0));
    Gemm g;
    g.M = X.n[0]; g.N = w0; g.K = X.R[1];
    g.A = Z1; g.sam = X.R[1]; g.sak = 1;
    g.B = s.W[1]; g.sbk = s.ldw; g.sbn = 1;
    g.C = E1; g.scm = w0; g.scn = 1;
    TTR_CHECK(E.small_gemm(c, g));
    TTR_CUDA(cudaMemsetAsync(dscal, 0, sizeof(double), stream));
    TTR_CHECK(sumsq(c, E1, X.n[0], w0, w0, 1, dscal));
    const double ss = dsync_read(c, dscal, &st);
    if (st != TTR_OK) return st;
    nrmx = sqrt(ss) / sqrt((double)w0);
    if (!isfinite(nrmx)) return set_error("non-finite norm estimate"), TTR_ERR_NONFINITE;
  }
  if (nrmx == 0.0) {
    // X = 0 (the estimate vanishes only then, with probability one): the zero TT of ranks 1
    // (reading R15)
    TTR_CHECK(result_alloc(c, X.shape(), out));
    double* arena = (double*)out->arena;
    int64_t off = 0;
    for (int k = 0; k < d; ++k) {
      out->cores[k] = arena + off;
      out->ranks[k] = 1;
      off += X.n[k];
    }
    out->ranks[d] = 1;
    TTR_CUDA(cudaMemsetAsync(arena, 0, sizeof(double) * off, stream));
    tm.rec(1, stream);
    tm.rec(2, stream);
    TTR_CUDA(cudaStreamSynchronize(stream));
    TTR_CHECK(check_device_flags(c));
    out->tau = 0.0;
    out->nrmx = 0.0;
    out->width = s.width;
    out->extensions = s.extensions;
    out->n_estimates = 0;
    out->estimates = (double*)calloc(1, sizeof(double));
    out->est_core = (int32_t*)calloc(1, sizeof(int32_t));
    if (!out->estimates || !out->est_core) return set_error("host allocation"), TTR_ERR_OOM;
    out->ms_sketch_rl = tm.ms(0, 1);
    out->ms_total = tm.ms(0, 2);
    out->kernel_launches = c.launches;
    c.time_collect(out);
    disown(c, out->arena);
    return TTR_OK;
  }
  const double tau = tol * nrmx / sqrt((double)(d - 1));
  const double tau_stop = tau / o.est_safety;   // reading R16: the loop stops at est <= tau / beta
  tm.rec(1, stream);
  Sweep w;
  TTR_CHECK(sweep_alloc(c, X.shape(), std::max(best_max, binit_max), w));
  if (X.mv) {
    int64_t ymax = 1;
    for (int k = 1; k < d; ++k) ymax = std::max(ymax, X.R[k] * X.n[k] * X.R[k + 1]);
    TTR_CHECK(c.alloc_t(&w.ycore, ymax));
  } else if (!X.single()) {
    int64_t ymax = 1;
    for (int k = 1; k < d; ++k) ymax = std::max(ymax, X.n[k] * X.part_rank_max(k + 1));
    TTR_CHECK(c.alloc_t(&w.ytmp, w.qcap * ymax));
  }
  TTR_CHECK(result_alloc(c, X.shape(), out));
  int64_t rowsmax = 1;
  for (int k = 0; k < d; ++k) rowsmax = std::max(rowsmax, X.R[k] * X.n[k]);
  double* Sall = nullptr;                       // Z W_{k+1}(:, 0:width): every sketch column of core k
  TTR_CHECK(c.alloc_t(&Sall, rowsmax * wcap));
  struct Probe {
    double ss;
    int flag;
  };
  Probe* dprobe = nullptr;                      // residual sum of squares + QR breakdown flag
  TTR_CHECK(c.alloc(reinterpret_cast<void**>(&dprobe), sizeof(Probe)));
  struct HostLoop {                             // buffers of the host-driven loop (made on first use)
    double* T = nullptr;                        // [Q, Q1]^T [Q1, S_next]
    double* Mn = nullptr;                       // Q1^T S_next - C^T Q^T S_next
    double* Pn = nullptr;                       // the next block's coefficients on Q_new
    double* Bt[2] = {nullptr, nullptr};         // [Q1, S_next] of alternate blocks
  } hl;
  std::vector<double> ests;
  std::vector<int32_t> est_core;
  double* arena = (double*)out->arena;
  int64_t off = 0, lprev = 1;
  const double* Z = Z1;
  int cur = 0;
  out->ranks[0] = 1;
  int64_t sk_cols = 0;                          // columns of Sall computed for the current core
  auto sketch_cols = [&](int k, int64_t rows, int64_t cols, int64_t c0, int64_t c1) -> int {
    if (c1 <= c0) return TTR_OK;
    Gemm g;
    g.M = rows; g.N = c1 - c0; g.K = cols;
    g.A = Z; g.sam = cols; g.sak = 1;
    g.B = s.W[k] + c0; g.sbk = s.ldw; g.sbn = 1;
    g.C = Sall + c0; g.scm = wcap; g.scn = 1;
    return E.sketch(c, g, (size_t)k < s.wplanes.size() ? &s.wplanes[k] : nullptr);
  };
  auto ensure = [&](int k, int64_t need, int64_t rows, int64_t cols) -> int {
    if (s.width < need) {
      if (need > s.ldw) return set_error("sketch capacity exceeded"), TTR_ERR_ARG;
      const int64_t target = std::min(s.ldw, std::max(need, s.width + std::max(binc_max, s.width / 2)));
      TTR_CHECK(rl_pass(c, E, X, seed, s.width, target, k + 1, s));   // Algorithm 5: append columns
      s.width = target;
      s.extensions++;
    }
    if (sk_cols < s.width) {
      TTR_CHECK(sketch_cols(k, rows, cols, sk_cols, s.width));
      sk_cols = s.width;
    }
    return TTR_OK;
  };
  // CholeskyQR2 without a host round trip; a breakdown only raises dprobe->flag.
  auto qr_try = [&](double* Xq, int64_t ldx, int64_t m, int64_t b) -> int {
    QrWork q2 = w.qr;
    q2.dflag = &dprobe->flag;
    TTR_CHECK(chol_pass(c, E, Xq, ldx, m, b, w.qr.tmp, b, q2, nullptr));
    return chol_pass(c, E, w.qr.tmp, b, m, b, Xq, ldx, q2, nullptr);
  };
  // estimates of one core land here (the device loop writes them, the host copies them out)
  std::vector<double> hest((size_t)rmax + 8);
  const bool device_loop = getenv("TTR_HOST_LOOP") == nullptr;
  for (int k = 1; k < d; ++k) {
    const int64_t rows = lprev * X.n[k - 1], cols = X.R[k];
    // the rank of V(Y_k) H(X_{k+1:d}) is also at most prod_{j>k} n_j (reading R14)
    int64_t right = 1;
    for (int j = k; j < d && right < rows; ++j) right = std::min<int64_t>(right * X.n[j], (int64_t)1 << 62);
    const int64_t rbar = std::min(std::min(rows, cols), right);
    const int64_t b0 = appendix ? std::min(rbar, X.part_rank_max(k)) : block_size(rbar, block, o.f_init);
    const int64_t ba = block_size(rbar, block, o.f_inc);   // columns appended per block
    const int64_t bi = std::max<int64_t>(ba, o.est_min);   // columns of each residual sketch (R16)
    sk_cols = 0;
    TTR_CHECK(ensure(k, std::min(rbar, b0) + bi, rows, cols));
    int64_t cc = 0;
    bool done = false;
    if (device_loop) {
      // the whole block loop on the device; the host steps in only to append sketch columns, to
      // factor a first block wider than the device loop's factors, or to redo a block whose
      // CholeskyQR broke down
      // blocks whose projections the host-driven loop puts on the tensor cores (sliced form): there
      // a block loop with its rows in global memory (FP64 pipe) is slower than the host-driven one
      const bool wide_tc = E.sliced() && (double)rows * rbar * bi >= kSlicedProjectWork;
      const bool device_runs = !wide_tc || adaptive_core_rows_fit(rows, (int)std::min<int64_t>(b0, bi), (int)bi,
                                                                  (int)rbar, (int)wcap, o.max_sms);
      if (device_runs && b0 > kBlockLoopMaxBlock && bi <= kBlockLoopMaxBlock) {
        TTR_CHECK(copy2d(c, w.Q, w.qcap, Sall, wcap, rows, b0));
        TTR_CHECK(qr_inplace(c, E, w.Q, w.qcap, rows, b0, w.qr));
        cc = b0;
        if (cc >= rbar) done = true;
      }
      int guard = 0;
      while (!done) {
        if (++guard > 4 * (int)rbar + 16) return set_error("adaptive loop did not terminate"), TTR_ERR_TIMEOUT;
        int status = 0, ccn = 0, nest = 0;
        st = adaptive_core(c, Sall, wcap, w.Q, w.qcap, w.S, rows, (int)(cc > 0 ? std::min(b0, bi) : b0), (int)bi,
                           (int)ba, (int)rbar, (int)sk_cols, (int)cc, tau_stop, hest.data(), (int)hest.size(), &status,
                           &ccn, &nest,
                           E.precision == TTR_PREC_SLICED && E.slices <= 6 && o.block_loop_df, nrmx, o.max_sms,
                           wide_tc, E.sliced() && o.block_loop_tc != 0);
        if (st == TTR_ERR_UNSUPPORTED) break;
        if (st != TTR_OK) return st;
        for (int q = 0; q < nest; ++q) {
          const double e = sqrt(hest[q]) / sqrt((double)bi);      // the device returns ||S||_F^2
          if (!isfinite(e)) return set_error("non-finite residual estimate"), TTR_ERR_NONFINITE;
          ests.push_back(e);
          est_core.push_back(k);
        }
        cc = ccn;
        if (status == 0) {
          done = true;
        } else if (status == 1) {
          TTR_CHECK(ensure(k, cc + bi, rows, cols));
        } else {
          // CholeskyQR breakdown: redo that factorization with the shifted/perturbed fallbacks
          if (cc == 0) {
            TTR_CHECK(copy2d(c, w.Q, w.qcap, Sall, wcap, rows, b0));
            TTR_CHECK(qr_inplace(c, E, w.Q, w.qcap, rows, b0, w.qr));
            cc = b0;
          } else {
            const int64_t bb = std::min(ba, rbar - cc);
            TTR_CHECK(copy2d(c, w.Q + cc, w.qcap, w.S, bi, rows, bb));
            TTR_CHECK(qr_inplace(c, E, w.Q + cc, w.qcap, rows, bb, w.qr));
            TTR_CHECK(E.project_out(c, w.Q, w.qcap, rows, cc, w.Q + cc, w.qcap, bb, w.P));
            TTR_CHECK(qr_inplace(c, E, w.Q + cc, w.qcap, rows, bb, w.qr));
            cc += bb;
          }
          if (cc >= rbar) done = true;
        }
      }
    }
    if (!done) {
    // Host-driven loop (blocks wider than the device loop supports), with the device loop's algebra:
    // after the first CholeskyQR pass Q1 of a residual block, one product [Q, Q1]^T [Q1, S_next]
    // gives C = Q^T Q1, the Gram matrix Q1^T Q1 - C^T C of Q1 - Q C (the second pass) and the next
    // block's coefficients, and one product Q [C, Q^T S_next] applies both, so each block reads Q
    // twice.  The residual of the next block is S_next - Q (Q^T S_next) - Q_new P_new with
    // P_new = R2^{-T} (Q1^T S_next - C^T Q^T S_next).  A CholeskyQR breakdown (seen at the next host
    // read) redoes that block with the robust fallbacks.
    TTR_CUDA(cudaMemsetAsync(dprobe, 0, sizeof(Probe), stream));
    TTR_CHECK(copy2d(c, w.Q, w.qcap, Sall, wcap, rows, b0));
    TTR_CHECK(qr_try(w.Q, w.qcap, rows, b0));
    cc = b0;
    if (!hl.T) {
      const int64_t bmax = w.bcap;
      TTR_CHECK(c.alloc_t(&hl.T, (w.qcap + bmax) * 2 * bmax));
      TTR_CHECK(c.alloc_t(&hl.Mn, bmax * bmax));
      TTR_CHECK(c.alloc_t(&hl.Pn, bmax * bmax));
      TTR_CHECK(c.alloc_t(&hl.Bt[0], rowsmax * 2 * bmax));
      TTR_CHECK(c.alloc_t(&hl.Bt[1], rowsmax * 2 * bmax));
    }
    QrWork q1 = w.qr;
    q1.dflag = &dprobe->flag;
    double* Rcur = w.S;              // residual sketch of the block at cc (rows x bi)
    int64_t ldr = bi;
    const double* Rprev = nullptr;   // that of the block appended last (for a fallback)
    int64_t ldp = 0, prev_bb = 0;
    bool phase1_checked = false, pending = true;
    int buf = 0;
    auto residual = [&]() -> int {   // Rcur = S_all(:, cc:cc+bi) - Q Q^T S_all(:, cc:cc+bi)
      TTR_CHECK(ensure(k, cc + bi, rows, cols));
      TTR_CHECK(copy2d(c, Rcur, ldr, Sall + cc, wcap, rows, bi));
      return E.project_out(c, w.Q, w.qcap, rows, cc, Rcur, ldr, bi, w.P, &dprobe->ss);
    };
    if (cc < rbar) TTR_CHECK(residual());
    while (cc < rbar) {
      Probe hp;
      TTR_CUDA(cudaMemcpyAsync(&hp, dprobe, sizeof(Probe), cudaMemcpyDeviceToHost, stream));
      TTR_CUDA(cudaStreamSynchronize(stream));
      pending = false;
      if (hp.flag) {
        // a CholeskyQR pass of the last factorization broke down: redo it robustly, then the
        // residual of the current block
        TTR_CUDA(cudaMemsetAsync(dprobe, 0, sizeof(Probe), stream));
        if (!phase1_checked) {
          TTR_CHECK(copy2d(c, w.Q, w.qcap, Sall, wcap, rows, b0));
          TTR_CHECK(qr_inplace(c, E, w.Q, w.qcap, rows, b0, w.qr));
        } else {
          const int64_t c0 = cc - prev_bb;
          TTR_CHECK(copy2d(c, w.Q + c0, w.qcap, Rprev, ldp, rows, prev_bb));
          TTR_CHECK(qr_inplace(c, E, w.Q + c0, w.qcap, rows, prev_bb, w.qr));
          TTR_CHECK(E.project_out(c, w.Q, w.qcap, rows, c0, w.Q + c0, w.qcap, prev_bb, w.P));
          TTR_CHECK(qr_inplace(c, E, w.Q + c0, w.qcap, rows, prev_bb, w.qr));
        }
        phase1_checked = true;
        TTR_CHECK(residual());
        continue;
      }
      phase1_checked = true;
      const double est = sqrt(hp.ss) / sqrt((double)bi);
      if (!isfinite(est)) return set_error("non-finite residual estimate"), TTR_ERR_NONFINITE;
      ests.push_back(est);
      est_core.push_back(k);
      if (!(est > tau_stop)) break;
      const int64_t bb = std::min(ba, rbar - cc), nxt = cc + bb;
      const bool want = nxt < rbar;
      if (want) TTR_CHECK(ensure(k, nxt + bi, rows, cols));
      const int64_t bn = want ? bi : 0, tw = bb + bn;
      // first pass: Q1 = Rcur(:, :bb) R1^{-1} into Q(:, cc:cc+bb)
      TTR_CHECK(chol_pass(c, E, Rcur, ldr, rows, bb, w.Q + cc, w.qcap, q1, nullptr));
      // [Q1, S_next] side by side, then T = [Q, Q1]^T [Q1, S_next]
      double* Bt = hl.Bt[buf];
      TTR_CHECK(copy2d(c, Bt, tw, w.Q + cc, w.qcap, rows, bb));
      if (want) TTR_CHECK(copy2d(c, Bt + bb, tw, Sall + nxt, wcap, rows, bi));
      TTR_CHECK(E.tn_product(c, w.Q, w.qcap, rows, cc + bb, Bt, tw, tw, hl.T, tw));
      // G2 = Q1^T Q1 - C^T C (into the QR workspace), Mn = Q1^T S_next - C^T Q^T S_next
      TTR_CHECK(block_step_gram(c, hl.T, tw, cc, bb, bn, w.qr.G, hl.Mn));
      TTR_CHECK(chol_inv(c, w.qr.G, bb, bb, nullptr, w.qr.Rinv, &dprobe->flag));
      // [Q1 - Q C, S_next - Q Q^T S_next] in one pass over Q, then Q_new = (Q1 - Q C) R2^{-1}
      TTR_CHECK(E.sub_product(c, w.Q, w.qcap, rows, cc, hl.T, tw, tw, Bt, tw));
      TTR_CHECK(apply_rinv(c, E, Bt, tw, rows, bb, w.qr.Rinv, w.Q + cc, w.qcap));
      Rprev = Rcur;
      ldp = ldr;
      prev_bb = bb;
      cc = nxt;
      pending = true;
      if (want) {
        // residual of the next block: S_next - Q Q^T S_next - Q_new P_new, with its sum of squares
        TTR_CHECK(tri_t_mul(c, w.qr.Rinv, bb, hl.Mn, bb, bi, hl.Pn));
        TTR_CHECK(E.sub_product(c, w.Q + cc - bb, w.qcap, rows, bb, hl.Pn, bi, bi, Bt + bb, tw, &dprobe->ss));
        Rcur = Bt + bb;
        ldr = tw;
        buf ^= 1;
      }
    }
    if (pending) {
      // the last factorization was never checked: a breakdown there is redone robustly
      Probe hp;
      TTR_CUDA(cudaMemcpyAsync(&hp, dprobe, sizeof(Probe), cudaMemcpyDeviceToHost, stream));
      TTR_CUDA(cudaStreamSynchronize(stream));
      if (hp.flag) {
        if (!phase1_checked) {
          TTR_CHECK(copy2d(c, w.Q, w.qcap, Sall, wcap, rows, b0));
          TTR_CHECK(qr_inplace(c, E, w.Q, w.qcap, rows, b0, w.qr));
        } else {
          const int64_t c0 = cc - prev_bb;
          TTR_CHECK(copy2d(c, w.Q + c0, w.qcap, Rprev, ldp, rows, prev_bb));
          TTR_CHECK(qr_inplace(c, E, w.Q + c0, w.qcap, rows, prev_bb, w.qr));
          TTR_CHECK(E.project_out(c, w.Q, w.qcap, rows, c0, w.Q + c0, w.qcap, prev_bb, w.P));
          TTR_CHECK(qr_inplace(c, E, w.Q + c0, w.qcap, rows, prev_bb, w.qr));
        }
      }
    }
    }
    double* Ynext = w.Y[cur];
    TTR_CHECK(project_next(c, E, w, Z, rows, cols, cc, X, k, Ynext, Zd));
    TTR_CHECK(copy2d(c, arena + off, cc, w.Q, w.qcap, rows, cc));
    out->cores[k - 1] = arena + off;
    out->ranks[k] = cc;
    off += rows * cc;
    Z = Ynext;
    cur ^= 1;
    lprev = cc;
  }
  const int64_t last = lprev * X.n[d - 1];
  TTR_CUDA(cudaMemcpyAsync(arena + off, Z, sizeof(double) * last, cudaMemcpyDeviceToDevice, stream));
  out->cores[d - 1] = arena + off;
  out->ranks[d] = 1;
  if (o.adap_r) TTR_CHECK(svd_pass_rl(c, E, out, X.n, tau * o.adap_r_tau_scale, 0));
  tm.rec(2, stream);
  TTR_CUDA(cudaStreamSynchronize(stream));
  TTR_CHECK(check_device_flags(c));
  out->tau = tau;
  out->nrmx = nrmx;
  out->width = s.width;
  out->extensions = s.extensions;
  out->n_estimates = (int32_t)ests.size();
  out->estimates = (double*)calloc(std::max<size_t>(1, ests.size()), sizeof(double));
  out->est_core = (int32_t*)calloc(std::max<size_t>(1, ests.size()), sizeof(int32_t));
  if (!out->estimates || !out->est_core) return set_error("host allocation"), TTR_ERR_OOM;
  std::copy(ests.begin(), ests.end(), out->estimates);
  std::copy(est_core.begin(), est_core.end(), out->est_core);
  out->ms_sketch_rl = tm.ms(0, 1);
  out->ms_sweep_lr = tm.ms(1, 2);
  out->ms_total = tm.ms(0, 2);
  out->kernel_launches = c.launches;
  c.time_collect(out);
  disown(c, out->arena);
  return TTR_OK;
}

// ----------------------------------------------------------------------------- deterministic
// Algorithm 1 in FP64.  Every QR is a Householder QR (householder.cu), backward stable also on the
// exactly rank-deficient unfoldings of a formal sum, and every SVD is one-sided Jacobi on the small
// triangular factor R (no Gram matrix, so singular values down to about u ||A|| are resolved and no
// direction is dropped before the truncation).

// SVD of the rows x cols row-major A (rows >= cols) through its R factor: A is overwritten by the
// Householder reflectors, and on return R = U S V^T with sig (device, cols, descending) and its
// host copy hsig, U in sw.U and V^T in sw.Vt (cols x cols each).  The left factor Q U of A is then
// householder_apply(A, E = U(:, :rp)).
struct SvdWork {
  double* R = nullptr;
  double* U = nullptr;
  double* Vt = nullptr;
  double* sig = nullptr;
  int* flag = nullptr;
};

static int svd_tall(Ctx& c, HhWork& hw, double* A, int64_t rows, int64_t cols, const SvdWork& sw,
                    std::vector<double>& hsig) {
  TTR_CHECK(householder_qr(c, hw, A, cols, rows, cols, sw.R, cols));
  TTR_CUDA(cudaMemsetAsync(sw.flag, 0, sizeof(int), c.stream));
  if (cols >= kJacobiMultiFrom)
    TTR_CHECK(jacobi_svd_multi(c, sw.R, cols, cols, sw.sig, sw.U, sw.Vt, sw.flag));
  else
    TTR_CHECK(jacobi_svd(c, sw.R, cols, cols, sw.sig, sw.U, sw.Vt, sw.flag));
  hsig.resize(cols);
  int bad = 0;
  TTR_CUDA(cudaMemcpyAsync(hsig.data(), sw.sig, sizeof(double) * cols, cudaMemcpyDeviceToHost, c.stream));
  TTR_CUDA(cudaMemcpyAsync(&bad, sw.flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  TTR_CUDA(cudaStreamSynchronize(c.stream));
  if (bad) return set_error("deterministic rounding: non-finite singular values"), TTR_ERR_NONFINITE;
  return TTR_OK;
}

static int64_t tail_rank(const std::vector<double>& s, int64_t n, double tau) {
  // smallest rp >= 1 with sqrt(sum_{i >= rp} s_i^2) <= tau (the truncated SVD of Algorithm 1)
  std::vector<double> tail(n + 1, 0.0);
  for (int64_t i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + s[i] * s[i];
  for (int64_t q = 1; q <= n; ++q)
    if (sqrt(tail[q]) <= tau) return q;
  return n;
}

static int round_deterministic(const TT& X, double tol, cudaStream_t stream, ttr_result* out) {
  if (!(tol > 0.0) || !isfinite(tol)) return set_error("tol must be positive and finite"), TTR_ERR_ARG;
  Ctx c;
  c.stream = stream;
  c.prof_begin();
  Timer tm;
  tm.rec(0, stream);
  Engine E;
  TTR_CHECK(E.init(c, TTR_PREC_FP64, 0, tol));
  const int d = X.d;
  std::vector<int64_t> r(X.r, X.r + d + 1);
  int64_t cmax = 1, rmax = 1;
  for (int k = 0; k < d; ++k) {
    cmax = std::max(cmax, X.r[k] * X.n[k] * X.r[k + 1]);
    rmax = std::max(rmax, std::max(X.r[k + 1], X.r[k]));
  }
  std::vector<double*> Y(d);
  for (int k = 0; k < d; ++k) {
    const int64_t sz = X.r[k] * X.n[k] * X.r[k + 1];
    TTR_CHECK(c.alloc_t(&Y[k], sz));
    TTR_CUDA(cudaMemcpyAsync(Y[k], X.cores[k], sizeof(double) * sz, cudaMemcpyDeviceToDevice, stream));
  }
  double *tmp, *tmp2;
  TTR_CHECK(c.alloc_t(&tmp, cmax));
  TTR_CHECK(c.alloc_t(&tmp2, cmax));
  SvdWork sw;
  TTR_CHECK(c.alloc_t(&sw.R, rmax * rmax));
  TTR_CHECK(c.alloc_t(&sw.U, rmax * rmax));
  TTR_CHECK(c.alloc_t(&sw.Vt, rmax * rmax));
  TTR_CHECK(c.alloc_t(&sw.sig, rmax));
  TTR_CHECK(c.alloc_t(&sw.flag, 4));
  HhWork hw;
  // ---- OrthogonalizeRL: H(Y_k)^T = Q R, H(Y_k) <- Q^T, V(Y_{k-1}) <- V(Y_{k-1}) R^T
  for (int k = d - 1; k >= 1; --k) {
    const int64_t r0 = r[k], nk = X.n[k], r1 = r[k + 1], m = nk * r1;
    const int64_t rows = r[k - 1] * X.n[k - 1];
    if (r0 > m) {
      // the rows of H(Y_k) span at most R^m: H(Y_k) = H(Y_k) I_m, so H(Y_k) <- I_m (orthonormal
      // rows) and V(Y_{k-1}) <- V(Y_{k-1}) H(Y_k) (the rank drops to m, the tensor is unchanged)
      Gemm v;
      v.M = rows; v.N = m; v.K = r0;
      v.A = Y[k - 1]; v.sam = r0; v.sak = 1;
      v.B = Y[k]; v.sbk = m; v.sbn = 1;
      v.C = tmp; v.scm = m; v.scn = 1;
      TTR_CHECK(E.small_gemm(c, v));
      TTR_CUDA(cudaMemcpyAsync(Y[k - 1], tmp, sizeof(double) * rows * m, cudaMemcpyDeviceToDevice, stream));
      TTR_CHECK(E.identity(c, Y[k], m));
      r[k] = m;
      continue;
    }
    TTR_CHECK(E.transpose(c, Y[k], r0, m, tmp));            // tmp = H(Y_k)^T  (m x r0)
    TTR_CHECK(householder_qr(c, hw, tmp, r0, m, r0, sw.R, r0));   // reflectors in tmp, R (r0 x r0)
    TTR_CHECK(E.identity(c, sw.U, r0));
    TTR_CHECK(householder_apply(c, hw, tmp, r0, m, r0, sw.U, r0, r0, tmp2, r0));   // tmp2 = Q (m x r0)
    TTR_CHECK(E.transpose(c, tmp2, m, r0, Y[k]));           // H(Y_k) = Q^T  (r0 x m)
    // V(Y_{k-1}) <- V(Y_{k-1}) R^T  ((r_{k-1} n_{k-1}) x r0)(r0 x r0)
    Gemm v;
    v.M = rows; v.N = r0; v.K = r0;
    v.A = Y[k - 1]; v.sam = r0; v.sak = 1;
    v.B = sw.R; v.sbk = 1; v.sbn = r0;
    v.C = tmp; v.scm = r0; v.scn = 1;
    TTR_CHECK(E.small_gemm(c, v));
    TTR_CUDA(cudaMemcpyAsync(Y[k - 1], tmp, sizeof(double) * rows * r0, cudaMemcpyDeviceToDevice, stream));
  }
  // ---- tau = ||Y_1|| tol / sqrt(d-1)
  double* dsc;
  TTR_CHECK(c.alloc_t(&dsc, 2));
  TTR_CUDA(cudaMemsetAsync(dsc, 0, sizeof(double), stream));
  TTR_CHECK(sumsq(c, Y[0], X.n[0] * r[1], 1, 1, 1, dsc));
  int st = TTR_OK;
  const double nrm = sqrt(dsync_read(c, dsc, &st));
  if (st != TTR_OK) return st;
  const double tau = nrm * tol / sqrt((double)(d - 1));
  // ---- compression: [Q, R] = QR(V(Y_k)), [U, S, V] = SVD(R, tau), V(Y_k) <- Q U,
  //      H(Y_{k+1}) <- S V^T H(Y_{k+1})
  std::vector<double> hs;
  for (int k = 0; k < d - 1; ++k) {
    const int64_t rows = r[k] * X.n[k], cols = r[k + 1];
    const int64_t ncol = X.n[k + 1] * r[k + 2];
    int64_t rp = 0;
    if (rows >= cols) {
      TTR_CHECK(copy2d(c, tmp2, cols, Y[k], cols, rows, cols));
      TTR_CHECK(svd_tall(c, hw, tmp2, rows, cols, sw, hs));            // reflectors of V(Y_k) in tmp2
      rp = tail_rank(hs, cols, tau);
      // V(Y_k) <- Q U(:, :rp)
      TTR_CHECK(householder_apply(c, hw, tmp2, cols, rows, cols, sw.U, cols, rp, Y[k], rp));
      // H(Y_{k+1}) <- diag(s) V^T(:rp, :) H(Y_{k+1})
      TTR_CHECK(E.scale_rows(c, sw.Vt, cols, rp, cols, sw.sig));
      Gemm v;
      v.M = rp; v.N = ncol; v.K = cols;
      v.A = sw.Vt; v.sam = cols; v.sak = 1;
      v.B = Y[k + 1]; v.sbk = ncol; v.sbn = 1;
      v.C = tmp; v.scm = ncol; v.scn = 1;
      TTR_CHECK(E.small_gemm(c, v));
    } else {
      // wide: V(Y_k)^T (cols x rows, tall) = Q2 R2, R2 = U2 S V2^T, so V(Y_k) = V2 S (Q2 U2)^T
      TTR_CHECK(E.transpose(c, Y[k], rows, cols, tmp));                 // tmp = V(Y_k)^T  (cols x rows)
      TTR_CHECK(svd_tall(c, hw, tmp, cols, rows, sw, hs));              // reflectors in tmp
      rp = tail_rank(hs, rows, tau);
      // V(Y_k) <- V2(:, :rp)  (rows x rp): V2 = Vt^T
      TTR_CHECK(E.transpose(c, sw.Vt, rows, rows, sw.R));               // R = V2 (rows x rows)
      TTR_CHECK(copy2d(c, Y[k], rp, sw.R, rows, rows, rp));
      // H(Y_{k+1}) <- diag(s) (Q2 U2(:, :rp))^T H(Y_{k+1})
      TTR_CHECK(householder_apply(c, hw, tmp, rows, cols, rows, sw.U, rows, rp, tmp2, rp));   // P = Q2 U2 (cols x rp)
      TTR_CHECK(E.scale_cols(c, tmp2, rp, rp, cols, sw.sig));           // P diag(s)
      Gemm v;                                                           // (P diag(s))^T H(Y_{k+1})
      v.M = rp; v.N = ncol; v.K = cols;
      v.A = tmp2; v.sam = 1; v.sak = rp;
      v.B = Y[k + 1]; v.sbk = ncol; v.sbn = 1;
      v.C = tmp; v.scm = ncol; v.scn = 1;
      TTR_CHECK(E.small_gemm(c, v));
    }
    TTR_CUDA(cudaMemcpyAsync(Y[k + 1], tmp, sizeof(double) * rp * ncol, cudaMemcpyDeviceToDevice, stream));
    r[k + 1] = rp;
  }
  TTR_CHECK(result_alloc(c, X, out));
  double* arena = (double*)out->arena;
  int64_t off = 0;
  for (int k = 0; k < d; ++k) {
    const int64_t sz = r[k] * X.n[k] * r[k + 1];
    TTR_CUDA(cudaMemcpyAsync(arena + off, Y[k], sizeof(double) * sz, cudaMemcpyDeviceToDevice, stream));
    out->cores[k] = arena + off;
    off += sz;
  }
  for (int k = 0; k <= d; ++k) out->ranks[k] = r[k];
  tm.rec(2, stream);
  TTR_CUDA(cudaStreamSynchronize(stream));
  TTR_CHECK(check_device_flags(c));
  out->tau = tau;
  out->nrmx = nrm;
  out->ms_total = tm.ms(0, 2);
  out->ms_sweep_lr = out->ms_total;
  out->kernel_launches = c.launches;
  disown(c, out->arena);
  return TTR_OK;
}

}  // namespace ttr

// ============================================================================= C ABI
using namespace ttr;

extern "C" {

void ttr_default_options(ttr_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = TTR_PREC_FP64;
  o->slices = 0;
  o->adap_r = 0;
  o->adap_r_tau_scale = 1.0;
  o->nrmx = 0.0;
  o->f_init = 0.1;
  o->f_inc = 0.05;
  o->width_hint = 0;
  o->kernel_timing = 0;
  o->max_sms = 0;
  o->est_min = 0;
  o->est_safety = 1.0;
  o->rl_percore = 0;
  o->block_loop_df = 0;
  o->block_loop_tc = 0;
  o->autotune = 0;
}

static int finish(int st, ttr_result* out, cudaStream_t s) {
  if (st != TTR_OK && out) {
    if (out->arena) cudaFreeAsync(out->arena, s);
    result_host_free(out);
    result_zero(out);
    out->status = st;
  } else if (out) {
    out->status = st;
  }
  return st;
}

int tt_round_fixed(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores, int64_t ell,
                   int64_t target, uint64_t seed, const ttr_options* opts, void* stream, ttr_result* out) {
  if (!out) return set_error("out must be non-null"), TTR_ERR_ARG;
  result_zero(out);
  ttr_options o;
  if (opts) o = *opts; else ttr_default_options(&o);
  TT X{d, n, r, cores};
  int st = validate(X);
  if (st == TTR_OK) st = round_fixed(X, ell, target, seed, o, (cudaStream_t)stream, out);
  return finish(st, out, (cudaStream_t)stream);
}

int tt_round_adaptive(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores, double tol,
                      int64_t block, uint64_t seed, const ttr_options* opts, void* stream, ttr_result* out) {
  if (!out) return set_error("out must be non-null"), TTR_ERR_ARG;
  result_zero(out);
  ttr_options o;
  if (opts) o = *opts; else ttr_default_options(&o);
  TT X{d, n, r, cores};
  int st = validate(X);
  if (st == TTR_OK) st = round_adaptive(single_sum(X), tol, block, seed, o, (cudaStream_t)stream, out);
  return finish(st, out, (cudaStream_t)stream);
}

int tt_round_adaptive_sum(int32_t s, int32_t d, const int64_t* n, const int64_t* const* r,
                          const double* const* const* cores, double tol, int64_t block, uint64_t seed,
                          const ttr_options* opts, void* stream, ttr_result* out) {
  if (!out) return set_error("out must be non-null"), TTR_ERR_ARG;
  result_zero(out);
  ttr_options o;
  if (opts) o = *opts; else ttr_default_options(&o);
  SumTT X;
  int st = make_sum(s, d, n, r, cores, X);
  if (st == TTR_OK) st = round_adaptive(X, tol, block, seed, o, (cudaStream_t)stream, out, true);
  return finish(st, out, (cudaStream_t)stream);
}

int tt_round_adaptive_matvec(int32_t d, const int64_t* n, const int64_t* m, const int64_t* p,
                             const double* const* A, const int64_t* r, const double* const* x, double tol,
                             int64_t block, uint64_t seed, const ttr_options* opts, void* stream, ttr_result* out) {
  if (!out) return set_error("out must be non-null"), TTR_ERR_ARG;
  result_zero(out);
  ttr_options o;
  if (opts) o = *opts; else ttr_default_options(&o);
  Matvec mv;
  SumTT X;
  int st = make_matvec(d, n, m, p, A, r, x, mv, X);
  if (st == TTR_OK && o.rl_percore != 0) st = (set_error("rl_percore applies to plain TTs and sums, not to y = A x"), TTR_ERR_ARG);
  if (st == TTR_OK) st = round_adaptive(X, tol, block, seed, o, (cudaStream_t)stream, out);
  return finish(st, out, (cudaStream_t)stream);
}

int tt_round_deterministic(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores, double tol,
                           void* stream, ttr_result* out) {
  if (!out) return set_error("out must be non-null"), TTR_ERR_ARG;
  result_zero(out);
  TT X{d, n, r, cores};
  int st = validate(X);
  if (st == TTR_OK) st = round_deterministic(X, tol, (cudaStream_t)stream, out);
  return finish(st, out, (cudaStream_t)stream);
}

void ttr_free(ttr_result* out, void* stream) {
  if (!out) return;
  if (out->arena) cudaFreeAsync(out->arena, (cudaStream_t)stream);
  result_host_free(out);
  result_zero(out);
}

const char* ttr_strerror(int s) {
  switch (s) {
    case TTR_OK: return "ok";
    case TTR_ERR_ARG: return "invalid argument";
    case TTR_ERR_OOM: return "out of memory";
    case TTR_ERR_NONFINITE: return "non-finite value";
    case TTR_ERR_QR_BREAKDOWN: return "CholeskyQR breakdown";
    case TTR_ERR_TIMEOUT: return "bounded device wait ran out";
    case TTR_ERR_CUDA: return "CUDA error";
    case TTR_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char* ttr_last_error(void) { return g_last_error.c_str(); }

int ttr_sketch_omega(uint64_t seed, int32_t k, int64_t n_k, int64_t col0, int64_t col1, double* dst, void* stream) {
  if (!dst || n_k < 1 || col1 < col0 || col0 < 0 || k < 1) return set_error("bad omega arguments"), TTR_ERR_ARG;
  Ctx c;
  c.stream = (cudaStream_t)stream;
  std::vector<int64_t> nn(k, n_k);
  int st = omega_fill(c, seed, k, k, nn.data(), col0, col1, dst, nullptr, 0, col1 - col0);
  if (st == TTR_OK) {
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return set_error(cudaGetErrorString(e)), TTR_ERR_CUDA;
  }
  return st;
}

int ttr_partial_contractions_percore(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores,
                                     uint64_t seed, int64_t col0, int64_t col1, int32_t t, double* const* W,
                                     void* stream) {
  TT X{d, n, r, cores};
  int st = validate(X);
  if (st != TTR_OK) return st;
  if (!W || t < 2 || t > d || col1 <= col0 || col0 < 0) return set_error("bad partial-contraction arguments"), TTR_ERR_ARG;
  for (int k = t; k <= d; ++k)
    if (!W[k - 1]) return set_error("null W buffer"), TTR_ERR_ARG;
  Ctx c;
  c.stream = (cudaStream_t)stream;
  Engine E;
  TTR_CHECK(E.init(c, TTR_PREC_FP64, 0, 0.0));
  const int64_t w = col1 - col0;
  Sketch s;
  TTR_CHECK(sketch_alloc(c, X, w, s));
  for (int k = t; k <= d; ++k) s.W[k - 1] = W[k - 1] - col0;   // caller buffers: [a][j - col0], ld w
  s.ldw = w;
  s.percore = true;
  TTR_CHECK(rl_pass(c, E, single_sum(X), seed, col0, col1, t, s));
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return set_error(cudaGetErrorString(e)), TTR_ERR_CUDA;
  return check_device_flags(c);
}

int ttr_partial_contractions_matvec(int32_t d, const int64_t* n, const int64_t* m, const int64_t* p,
                                    const double* const* A, const int64_t* r, const double* const* x, uint64_t seed,
                                    int64_t col0, int64_t col1, int32_t t, int32_t precision, int32_t slices,
                                    double* const* W, void* stream) {
  Matvec mv;
  SumTT X;
  TTR_CHECK(make_matvec(d, n, m, p, A, r, x, mv, X));
  if (!W || t < 2 || t > d || col1 <= col0 || col0 < 0) return set_error("bad partial-contraction arguments"), TTR_ERR_ARG;
  for (int k = t; k <= d; ++k)
    if (!W[k - 1]) return set_error("null W buffer"), TTR_ERR_ARG;
  Ctx c;
  c.stream = (cudaStream_t)stream;
  Engine E;
  TTR_CHECK(E.init(c, precision, slices, 0.0));
  const int64_t w = col1 - col0;
  Sketch s;
  TTR_CHECK(sketch_alloc(c, X.shape(), w, s));
  for (int k = t; k <= d; ++k) s.W[k - 1] = W[k - 1] - col0;   // caller buffers: [(a, b)][j - col0], ld w
  s.ldw = w;
  TTR_CHECK(rl_pass(c, E, X, seed, col0, col1, t, s));
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return set_error(cudaGetErrorString(e)), TTR_ERR_CUDA;
  return check_device_flags(c);
}

int ttr_selftest_rsqrt(const double* x, double* out, int64_t count, void* stream) {
  if (!x || !out || count < 0) return set_error("bad self-test arguments"), TTR_ERR_ARG;
  Ctx c;
  c.stream = (cudaStream_t)stream;
  TTR_CHECK(rsqrt_selftest(c, x, out, count));
  const cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return set_error(cudaGetErrorString(e)), TTR_ERR_CUDA;
  return TTR_OK;
}

int ttr_selftest_jacobi_rotation(const double* abg, double tiny, double* cs_sn, int64_t count, void* stream) {
  if (!abg || !cs_sn || count < 0 || !(tiny >= 0.0)) return set_error("bad self-test arguments"), TTR_ERR_ARG;
  Ctx c;
  c.stream = (cudaStream_t)stream;
  TTR_CHECK(jacobi_rotation_selftest(c, abg, tiny, cs_sn, count));
  const cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return set_error(cudaGetErrorString(e)), TTR_ERR_CUDA;
  return TTR_OK;
}

int ttr_partial_contractions(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores,
                             uint64_t seed, int64_t col0, int64_t col1, int32_t t, int32_t precision,
                             int32_t slices, double* const* W, void* stream) {
  TT X{d, n, r, cores};
  int st = validate(X);
  if (st != TTR_OK) return st;
  if (!W || t < 2 || t > d || col1 <= col0 || col0 < 0) return set_error("bad partial-contraction arguments"), TTR_ERR_ARG;
  for (int k = t; k <= d; ++k)
    if (!W[k - 1]) return set_error("null W buffer"), TTR_ERR_ARG;
  Ctx c;
  c.stream = (cudaStream_t)stream;
  Engine E;
  TTR_CHECK(E.init(c, precision, slices, 0.0));
  const int64_t w = col1 - col0;
  Sketch s;
  TTR_CHECK(sketch_alloc(c, X, w, s));
  for (int k = t; k <= d; ++k) s.W[k - 1] = W[k - 1] - col0;   // caller buffers: [a][j - col0], ld w
  s.ldw = w;
  TTR_CHECK(rl_pass(c, E, single_sum(X), seed, col0, col1, t, s));
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return set_error(cudaGetErrorString(e)), TTR_ERR_CUDA;
  return check_device_flags(c);
}

}  // extern "C"
