// Device helpers shared by the diagnostics reductions.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Compensated FP32 sum (Kahan): the error of a thread's partial sum stays near one FP32
// rounding of the sum whatever the number of terms, so the per-node work runs on the FP32
// pipe and only the cross-thread combination needs FP64 (whose issue rate on this part is a
// small fraction of FP32's).  No product is involved, so no FMA contraction can undo it.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace lbm
