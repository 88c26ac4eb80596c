// Tensor-core (tcgen05) sliced contractions.  Placeholder until the kernels land: every entry
// reports TTR_ERR_UNSUPPORTED so the engine uses the FP64 kernels.
#include "engine.cuh"

namespace ttr {

int tc_rl_step(Ctx&, int, const double*, int64_t, int64_t, int64_t, const double*, int64_t, const double*, int64_t,
               int64_t, double*, int64_t) {
  return TTR_ERR_UNSUPPORTED;
}
int tc_gemm_rowmajor(Ctx&, int, const double*, int64_t, int64_t, int64_t, const double*, int64_t, int64_t, double*,
                     int64_t) {
  return TTR_ERR_UNSUPPORTED;
}
int tc_project(Ctx&, int, const double*, int64_t, int64_t, int64_t, const double*, int64_t, double*) {
  return TTR_ERR_UNSUPPORTED;
}

}  // namespace ttr
