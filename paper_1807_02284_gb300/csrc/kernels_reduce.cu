// Diagnostics reduction (mass, momentum, kinetic energy) over the current populations of a
// block: one pass over the 27 planes, deterministic order.
#include "lbm_internal.h"
#include "reduce_util.cuh"

namespace lbm {

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
// tree combines the lanes, so the result does not depend on scheduling.  out5 (optional)
// also receives the five diagnostics in the lbm_reduce layout (mass = out[0] + out[1]).
__global__ void __launch_bounds__(192) k_reduce_final(const double* partials, int n, double* out,
                                                      double* out5) {
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0;
  for (int b = lane; b < n; b += 32) s += partials[b * 6 + v];
  s = warp_sum(s);
  if (lane == 0) out[v] = s;
  if (out5 != nullptr) {
    __syncthreads();
    if (threadIdx.x < 5) out5[threadIdx.x] = threadIdx.x == 0 ? out[0] + out[1] : out[threadIdx.x + 1];
  }
}

// n records of 8 doubles (6 sums + 2 unused), summed in two fixed-order stages so that many
// SMs share the reads: CTA s of stage 1 sums slice s of the records (thread t: records
// t, t + 256, ... of the slice, in order, then a fixed tree per value) into
// stage[s * 6 + value]; stage 2 is k_reduce_final over those partials.
constexpr int COL_SLICES = 128;

__global__ void __launch_bounds__(256) k_reduce_records(const double* rec, size_t n,
                                                        double* stage) {
  __shared__ double sh[6][256];
  const int sl = blockIdx.x;
  const size_t per = (n + COL_SLICES - 1) / COL_SLICES;
  const size_t lo = per * sl, hi = lo + per < n ? lo + per : n;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (size_t i = lo + threadIdx.x; i < hi; i += 256) {
#pragma unroll
    for (int v = 0; v < 6; ++v) s[v] += rec[i * 8 + v];
  }
#pragma unroll
  for (int v = 0; v < 6; ++v) sh[v][threadIdx.x] = s[v];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int v = 0; v < 6; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) stage[sl * 6 + threadIdx.x] = sh[threadIdx.x][0];
}

// `partials` holds 8 n + 6 COL_SLICES doubles: the records, then the stage-1 sums.
cudaError_t launch_reduce_columns(double* partials, size_t n, double* out, cudaStream_t s,
                                  double* out5) {
  double* stage = partials + 8 * n;
  k_reduce_records<<<COL_SLICES, 256, 0, s>>>(partials, n, stage);
  k_reduce_final<<<1, 192, 0, s>>>(stage, COL_SLICES, out, out5);
  return cudaGetLastError();
}

// Diagnostics of many domains in one launch (lbm_reduce_batch): a list of chunks, each of
// one member's nodes; every CTA takes chunks in turn (per-thread compensated FP32 sums, FP64
// across the CTA, in the order of k_reduce) and writes one record of 8 doubles per chunk.
template <typename T>
__global__ void __launch_bounds__(REDUCE_THREADS) k_reduce_items(const RedItem* items, int n_items,
                                                                 const RedMember* members,
                                                                 double* records) {
  __shared__ double sh[REDUCE_THREADS / 32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
    const RedItem it = items[w];
    const RedMember m = members[it.member];
    const T* d = static_cast<const T*>(m.f);
    unsigned count = 0;
    KahanF acc[5];
    for (size_t idx = it.start + threadIdx.x; idx < it.start + it.len; idx += blockDim.x) {
      if (m.flags[idx] & (F_SOLID | F_GHOST)) continue;
      float dd[27];
#pragma unroll
      for (int k = 0; k < 27; ++k) dd[k] = load_pop(d + (size_t)k * m.N + idx);
      float drho, jx, jy, jz;
      macros(dd, drho, jx, jy, jz);
      ++count;
      acc[0].add(drho);
      acc[1].add(jx);
      acc[2].add(jy);
      acc[3].add(jz);
      acc[4].add(0.5f * (jx * jx + jy * jy + jz * jz) / (1.0f + drho));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double v = warp_sum(i == 0 ? (double)count : acc[i - 1].value());
      if (lane == 0) sh[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
      double s = 0;
      for (int k = 0; k < REDUCE_THREADS / 32; ++k) s += sh[k][threadIdx.x];
      records[(size_t)w * 8 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// One warp per member: its chunks' records (contiguous in the list) in order, then the
// shuffle tree; the member's device error word rides along in slot 6.
__global__ void __launch_bounds__(256) k_reduce_items_final(const double* records,
                                                            const RedMember* members, int n,
                                                            double* out) {
  const int m = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (m >= n) return;
  const RedMember mb = members[m];
  for (int v = 0; v < 6; ++v) {
    double s = 0;
    for (int c = lane; c < mb.n_items; c += 32) s += records[(size_t)(mb.first_item + c) * 8 + v];
    s = warp_sum(s);
    if (lane == 0) out[(size_t)m * 8 + v] = s;
  }
  if (lane == 0) out[(size_t)m * 8 + 6] = (double)*mb.err;
}

cudaError_t launch_reduce_item_records(const double* records, const RedMember* members, int n,
                                      double* out, cudaStream_t s) {
  k_reduce_items_final<<<(n + 7) / 8, 256, 0, s>>>(records, members, n, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_items(int storage, const RedItem* items, int n_items,
                                const RedMember* members, int n_members, double* records,
                                double* out, cudaStream_t s) {
  const int ctas = n_items < REDUCE_CTAS ? n_items : REDUCE_CTAS;
  if (storage == ST_FP16)
    k_reduce_items<__half><<<ctas, REDUCE_THREADS, 0, s>>>(items, n_items, members, records);
  else
    k_reduce_items<float><<<ctas, REDUCE_THREADS, 0, s>>>(items, n_items, members, records);
  k_reduce_items_final<<<(n_members + 7) / 8, 256, 0, s>>>(records, members, n_members, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const void* d, int storage, const uint8_t* flags, size_t N,
                          double* partials, double* out, cudaStream_t s, double* out5) {
  const size_t want = (N + REDUCE_THREADS - 1) / REDUCE_THREADS;
  const int ctas = (int)(want < (size_t)REDUCE_CTAS ? (want > 0 ? want : 1) : REDUCE_CTAS);
  if (storage == ST_FP16)
    k_reduce<__half><<<ctas, REDUCE_THREADS, 0, s>>>((const __half*)d, flags, N, partials);
  else
    k_reduce<float><<<ctas, REDUCE_THREADS, 0, s>>>((const float*)d, flags, N, partials);
  k_reduce_final<<<1, 192, 0, s>>>(partials, ctas, out, out5);
  return cudaGetLastError();
}

}  // namespace lbm
