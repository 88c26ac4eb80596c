// ttr_partial_contractions_noalloc: the right-to-left partial contractions (FP64) with their
// scratch in a fixed, file-scope device array instead of stream-ordered allocations.
//
// Who needs it: callers that may not allocate device memory at all, because something else owns
// it (a host runtime or framework whose pool allocator holds the whole device and forbids side
// allocations through cudaMalloc / cudaMallocAsync), or because an allocation there could fail
// or block (a pool at its limit, a code path that must not wait for the allocator).  The caller
// passes the inputs and the outputs; everything else the pass needs lives in g_scratch below.
//
// The array is TTR_STATIC_SCRATCH_BYTES long.  Every GPU that loads this library's device code
// holds it until the process exits.  All calls on a device share it: a call leaves its
// contents there, and two calls that overlap on the GPU (different streams, or different host
// threads) overwrite each other's scratch and race.
#include <mutex>

#include "ttr_internal.cuh"

namespace ttr {

static_assert(TTR_STATIC_SCRATCH_BYTES % 256 == 0, "scratch size must be a multiple of 256 bytes");
constexpr int64_t kScratchDoubles = TTR_STATIC_SCRATCH_BYTES / sizeof(double);
constexpr int kMaxDevices = 64;

// In host code g_scratch names a host-side stand-in, not a device address: the device address
// comes from cudaGetSymbolAddress, once per device, with that device current.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

static std::mutex g_scratch_mu;
static void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up on the first call there).
static int scratch_base(double** out) {
  int dev = -1;
  TTR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal outside the range of the static-scratch table");
    return TTR_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
      return TTR_ERR_CUDA;
    }
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
      set_error("static scratch is not 256-byte aligned");
      return TTR_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_ptr[dev]);
  return TTR_OK;
}

}  // namespace ttr

using namespace ttr;

extern "C" {

int ttr_partial_contractions_noalloc(int32_t d, const int64_t* n, const int64_t* r, const double* const* cores,
                                     uint64_t seed, int64_t col0, int64_t col1, int32_t t, double* const* W,
                                     void* stream) {
  if (d < 2 || d > TTR_MAX_D || !n || !r || !cores || !W) return set_error("bad TT arguments"), TTR_ERR_ARG;
  if (t < 2 || t > d || col0 < 0 || col1 <= col0) return set_error("bad partial-contraction arguments"), TTR_ERR_ARG;
  if (r[0] != 1 || r[d] != 1) return set_error("r[0] and r[d] must be 1"), TTR_ERR_ARG;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || r[k + 1] < 1) return set_error("mode sizes and ranks must be >= 1"), TTR_ERR_ARG;
    if (!cores[k] || reinterpret_cast<uintptr_t>(cores[k]) % 8 != 0)
      return set_error("core pointers must be non-null and 8-byte aligned"), TTR_ERR_ARG;
  }
  for (int k = t; k <= d; ++k)
    if (!W[k - 1] || reinterpret_cast<uintptr_t>(W[k - 1]) % 8 != 0)
      return set_error("W buffers must be non-null and 8-byte aligned"), TTR_ERR_ARG;

  // scratch layout (doubles): [Omega_t..Omega_d] [T]
  const int64_t w = col1 - col0;
  const int32_t nc = d - t + 1;
  int64_t nmax = 1;
  __int128 rowsmax = 0;   // r_{k-1} n_k < 2^126
  for (int k = t; k <= d; ++k) {
    nmax = n[k - 1] > nmax ? n[k - 1] : nmax;
    const __int128 rows = (__int128)r[k - 1] * n[k - 1];
    if (k < d && rows > rowsmax) rowsmax = rows;
  }
  const bool huge = rowsmax > kScratchDoubles || nmax > kScratchDoubles || w > kScratchDoubles;
  const __int128 need = huge ? ((__int128)1 << 62) : ((__int128)nc * nmax + rowsmax) * w;
  if (need > kScratchDoubles) {
    const __int128 bytes = need * 8;
    set_error("ttr_partial_contractions_noalloc needs " +
              (huge ? std::string("far more than that") : std::to_string((long long)bytes)) +
              " bytes of scratch; the static limit is TTR_STATIC_SCRATCH_BYTES = " +
              std::to_string((long long)TTR_STATIC_SCRATCH_BYTES));
    return TTR_ERR_UNSUPPORTED;
  }

  double* base = nullptr;
  TTR_CHECK(scratch_base(&base));
  double* Om = base;
  const int64_t ostride = nmax * w;
  double* T = Om + (int64_t)nc * ostride;   // (max r_{k-1} n_k) x w

  Ctx c;   // no allocation below: every device buffer is the caller's or the static scratch
  c.stream = (cudaStream_t)stream;
  // The mode sizes go to the Omega kernels as kernel parameters (no host-to-device copy).  Every
  // scratch element read below is written earlier in this call (Omega by omega_fill_byval, T by a
  // non-accumulating GEMM), so nothing left by a previous call needs clearing.
  TTR_CHECK(omega_fill_byval(c, seed, t, nc, n + (t - 1), col0, col1, Om, ostride, w));
  {  // W_d = H(X_d) Omega_d   (Eq. (3.2))
    Gemm g;
    g.M = r[d - 1]; g.N = w; g.K = n[d - 1];
    g.A = cores[d - 1]; g.sam = n[d - 1]; g.sak = 1;
    g.B = Om + (int64_t)(d - t) * ostride; g.sbk = w; g.sbn = 1;
    g.C = W[d - 1]; g.scm = w; g.scn = 1;
    TTR_CHECK(gemm_f64(c, g));
  }
  for (int k = d - 1; k >= t; --k) {  // W_k from W_{k+1} (Eq. (3.3))
    Gemm g;
    g.M = r[k - 1] * n[k - 1]; g.N = w; g.K = r[k];
    g.A = cores[k - 1]; g.sam = r[k]; g.sak = 1;
    g.B = W[k]; g.sbk = w; g.sbn = 1;
    g.C = T; g.scm = w; g.scn = 1;
    TTR_CHECK(gemm_f64(c, g));
    TTR_CHECK(omega_reduce(c, T, w, Om + (int64_t)(k - t) * ostride, w, r[k - 1], n[k - 1], w, W[k - 1], w));
  }
  return TTR_OK;
}

}  // extern "C"
