// Continuous-scale coupling (Sec. 4.2, Algorithm 1): refined blocks, prior-/post-mapping,
// temporal alignment.
#include "runtime.h"

using namespace lbm;

lbm_status multiscale_step(lbm_domain* dom) {
  return dom->fail(LBM_ERR_UNSUPPORTED, "multi-scale stepping not built yet");
}

extern "C" lbm_status lbm_add_scale_block(lbm_domain* dom, const double origin[3], double h,
                                          const int32_t dims[3], int32_t* block_id) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  (void)origin; (void)h; (void)dims; (void)block_id;
  return dom->fail(LBM_ERR_UNSUPPORTED, "scale blocks not built yet");
}
