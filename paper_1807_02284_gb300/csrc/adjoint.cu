// Reverse-mode (adjoint) stepping with checkpointing.
#include "runtime.h"

using namespace lbm;

namespace lbm {
struct TapeState {
  int every = 0;
};
}  // namespace lbm

void release_tape(lbm_domain* dom) {
  delete dom->tape;
  dom->tape = nullptr;
}

lbm_status tape_before_step(lbm_domain* dom) {
  (void)dom;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_tape(lbm_domain* dom, int32_t checkpoint_every) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  (void)checkpoint_every;
  return dom->fail(LBM_ERR_UNSUPPORTED, "adjoint not built yet");
}

extern "C" lbm_status lbm_adjoint_step(lbm_domain* dom, int32_t n_steps, const float* dL_dc,
                                       const float* dL_du, float* dL_du0, float* dL_dinflow) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  (void)n_steps; (void)dL_dc; (void)dL_du; (void)dL_du0; (void)dL_dinflow;
  return dom->fail(LBM_ERR_UNSUPPORTED, "adjoint not built yet");
}
