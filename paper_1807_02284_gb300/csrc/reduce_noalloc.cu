// Mass / momentum / kinetic-energy reduction that allocates no memory.
//
// Some callers cannot allocate device memory: a process whose device memory is entirely
// reserved by another framework's pool, or a latency-critical loop that must never reach the
// driver's allocator.  For them this variant of the diagnostics reduction keeps its per-CTA
// partial sums in a file-scope device array instead of a library-allocated buffer.  The
// caller passes the populations, the flags and the output; nothing else is needed.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "reduce_util.cuh"

namespace lbm {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_NODES_PER_CTA = 16384;
constexpr int NOALLOC_MAX_CTAS = LBM_REDUCE_NOALLOC_MAX_NODES / NOALLOC_NODES_PER_CTA;
static_assert(NOALLOC_MAX_CTAS * NOALLOC_NODES_PER_CTA == LBM_REDUCE_NOALLOC_MAX_NODES,
              "node limit must be a whole number of CTA chunks");

// Scratch: 6 partial sums per CTA (192 KiB).  Every process that loads the library holds it
// on every GPU it uses until exit.  All calls share it; each call overwrites the slots of the
// CTAs it launches before reading them, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_CTAS * 6];

// f: 27 planes of unshifted populations in the paper's order; one CTA per chunk of nodes.
// Per node the deviations f - w from the lattice weights are summed in FP32 (small numbers:
// no cancellation against the weights), per thread with compensated FP32 sums, and combined
// across threads in FP64 in a fixed order.
template <typename I>
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_reduce_noalloc(const I* __restrict__ f, const uint8_t* __restrict__ flags, size_t N,
                 double* __restrict__ partials) {
  const size_t lo = (size_t)blockIdx.x * NOALLOC_NODES_PER_CTA;
  const size_t hi = lo + NOALLOC_NODES_PER_CTA < N ? lo + NOALLOC_NODES_PER_CTA : N;
  unsigned count = 0;
  KahanF acc[5];
  for (size_t idx = lo + threadIdx.x; idx < hi; idx += NOALLOC_THREADS) {
    if (flags && (flags[idx] & (F_SOLID | F_GHOST))) continue;
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int k = paper_to_cube(q);
      const float d = (float)(f[(size_t)q * N + idx] - (I)wkd(k));
      drho += d;
      if (cxk(k) > 0) jx += d; else if (cxk(k) < 0) jx -= d;
      if (cyk(k) > 0) jy += d; else if (cyk(k) < 0) jy -= d;
      if (czk(k) > 0) jz += d; else if (czk(k) < 0) jz -= d;
    }
    ++count;
    acc[0].add(drho);
    acc[1].add(jx);
    acc[2].add(jy);
    acc[3].add(jz);
    acc[4].add(0.5f * (jx * jx + jy * jy + jz * jz) / (1.0f + drho));
  }
  __shared__ double sh[NOALLOC_THREADS / 32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double w = warp_sum(i == 0 ? (double)count : acc[i - 1].value());
    if (lane == 0) sh[wid][i] = w;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0;
    for (int w = 0; w < NOALLOC_THREADS / 32; ++w) s += sh[w][threadIdx.x];
    partials[blockIdx.x * 6 + threadIdx.x] = s;
  }
}

// One warp per value: lane l sums partials l, l + 32, ... in order, a fixed shuffle tree
// combines the lanes; mass = node count + sum of (rho - 1).
__global__ void __launch_bounds__(192) k_reduce_noalloc_final(const double* __restrict__ partials,
                                                              int n_ctas, double* __restrict__ out) {
  __shared__ double tot[6];
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < n_ctas; b += 32) s += partials[b * 6 + v];
  s = warp_sum(s);
  if (lane == 0) tot[v] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = tot[0] + tot[1];
    out[1] = tot[2];
    out[2] = tot[3];
    out[3] = tot[4];
    out[4] = tot[5];
  }
}

// Device address of the scratch array, looked up once per device with that device current.
// In host code the array's name is only a host-side stand-in, so kernels get this address.
// The cached address belongs to the device's primary context: a context reset
// (cudaDeviceReset) invalidates it, and the entry point must not be called afterwards.
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};
}  // namespace

static cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace lbm

void lbm_set_global_error(const char* msg);  // runtime.cu

extern "C" lbm_status lbm_reduce_noalloc(const void* f, int32_t dtype, const uint8_t* flags,
                                         int64_t n_nodes, double* out, void* cuda_stream) {
  using namespace lbm;
  if (!f || !out) { lbm_set_global_error("lbm_reduce_noalloc: null pointer"); return LBM_ERR_INVALID_ARG; }
  if (dtype != LBM_F32 && dtype != LBM_F64) {
    lbm_set_global_error("lbm_reduce_noalloc: dtype must be LBM_F32 or LBM_F64");
    return LBM_ERR_INVALID_ARG;
  }
  if (n_nodes < 1 || n_nodes > (int64_t)LBM_REDUCE_NOALLOC_MAX_NODES) {
    lbm_set_global_error("lbm_reduce_noalloc: n_nodes must be in [1, LBM_REDUCE_NOALLOC_MAX_NODES]"
                         " (the fixed scratch holds that many nodes' partial sums)");
    return LBM_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    lbm_set_global_error(cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  const size_t N = (size_t)n_nodes;
  const int n_ctas = (int)((N + NOALLOC_NODES_PER_CTA - 1) / NOALLOC_NODES_PER_CTA);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (dtype == LBM_F64)
    k_reduce_noalloc<double><<<n_ctas, NOALLOC_THREADS, 0, s>>>(static_cast<const double*>(f),
                                                                flags, N, scratch);
  else
    k_reduce_noalloc<float><<<n_ctas, NOALLOC_THREADS, 0, s>>>(static_cast<const float*>(f),
                                                               flags, N, scratch);
  k_reduce_noalloc_final<<<1, 192, 0, s>>>(scratch, n_ctas, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    lbm_set_global_error(cudaGetErrorString(e));
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
