// Batched persistent stepping of many independent single-block domains.
#include "runtime.h"

using namespace lbm;

extern "C" lbm_status lbm_step_batch(lbm_domain* const* doms, int32_t n, int32_t steps) {
  if (!doms || n <= 0 || !doms[0]) return LBM_ERR_INVALID_ARG;
  (void)steps;
  return doms[0]->fail(LBM_ERR_UNSUPPORTED, "batched stepping not built yet");
}
