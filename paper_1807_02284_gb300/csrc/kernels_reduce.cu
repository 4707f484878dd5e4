// Diagnostics reduction (mass, momentum, kinetic energy) over the current populations of a
// block: one pass over the 27 planes, deterministic order.
#include "lbm_internal.h"

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

template <typename T>
__global__ void __launch_bounds__(REDUCE_THREADS, 4) k_reduce(const T* d, const uint8_t* flags,
                                                              size_t N, double* partials) {
  unsigned count = 0;
  KahanF acc[5];
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    if (flags[idx] & (F_SOLID | F_GHOST)) continue;
    float dd[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) dd[k] = load_pop(d + (size_t)k * N + idx);
    float drho, jx, jy, jz;
    macros(dd, drho, jx, jy, jz);
    ++count;
    acc[0].add(drho);
    acc[1].add(jx);
    acc[2].add(jy);
    acc[3].add(jz);
    acc[4].add(0.5f * (jx * jx + jy * jy + jz * jz) / (1.0f + drho));
  }
  __shared__ double sh[REDUCE_THREADS / 32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double w = warp_sum(i == 0 ? (double)count : acc[i - 1].value());
    if (lane == 0) sh[wid][i] = w;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0;
    for (int w = 0; w < REDUCE_THREADS / 32; ++w) s += sh[w][threadIdx.x];
    partials[blockIdx.x * 6 + threadIdx.x] = s;
  }
}

// One warp per value: lane l sums partials l, l + 32, ... in order, then a fixed shuffle
// tree combines the lanes, so the result does not depend on scheduling.
__global__ void __launch_bounds__(192) k_reduce_final(const double* partials, int n, double* out) {
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < n; b += 32) s += partials[b * 6 + v];
  s = warp_sum(s);
  if (lane == 0) out[v] = s;
}

// Six columns of n partial sums (value-major): one CTA per column, thread t sums entries
// t, t + 1024, ... in order, then a fixed tree over the threads.
__global__ void __launch_bounds__(1024) k_reduce_columns(const double* partials, size_t n,
                                                         double* out) {
  __shared__ double sh[1024];
  const double* col = partials + blockIdx.x * n;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += 1024) s += col[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

cudaError_t launch_reduce_columns(const double* partials, size_t n, double* out, cudaStream_t s) {
  k_reduce_columns<<<6, 1024, 0, s>>>(partials, n, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const void* d, int storage, const uint8_t* flags, size_t N,
                          double* partials, double* out, cudaStream_t s) {
  const size_t want = (N + REDUCE_THREADS - 1) / REDUCE_THREADS;
  const int ctas = (int)(want < (size_t)REDUCE_CTAS ? (want > 0 ? want : 1) : REDUCE_CTAS);
  if (storage == ST_FP16)
    k_reduce<__half><<<ctas, REDUCE_THREADS, 0, s>>>((const __half*)d, flags, N, partials);
  else
    k_reduce<float><<<ctas, REDUCE_THREADS, 0, s>>>((const float*)d, flags, N, partials);
  k_reduce_final<<<1, 192, 0, s>>>(partials, ctas, out);
  return cudaGetLastError();
}

}  // namespace lbm
