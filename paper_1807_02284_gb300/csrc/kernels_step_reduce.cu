// The collide-stream step with the block diagnostics fused in (lbm_step_reduce): the same
// per-node update as k_step, plus the sums that lbm_reduce would take in a second pass.
#include "lbm_cell.cuh"

namespace lbm {

// End of a fused-diagnostics CTA: each warp has written the sums of its gpw 32-node groups to
// swarp (lane 0); the last warp to get here (shared-memory counter `done`, zeroed before
// any warp counts) adds the nwarps * gpw group sums in order and stores the CTA's record of
// 8 doubles (6 sums, 2 zeros).  No warp waits for the others' updates.
__device__ __forceinline__ void finish_cta_record(float (*swarp)[6], unsigned& done, int lane,
                                                  int nwarps, int gpw, double* partials) {
  unsigned last = 0u;
  if (lane == 0) {
    __threadfence_block();
    last = atomicAdd(&done, 1u) == (unsigned)(nwarps - 1);
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last && lane < 8) {
    __threadfence_block();
    const volatile float* sv = &swarp[0][0];
    float s = 0.0f;
    if (lane < 6)
      for (int k = 0; k < nwarps * gpw; ++k) s += sv[k * 6 + lane];
    const size_t cta = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    partials[cta * 8 + lane] = (double)s;
  }
}

// A step that also sums the diagnostics of the state it stores (lbm_step_reduce): every node
// writes its moments into its warp's shared-memory columns as soon as they are known, so
// nothing is held through the collision; after the update each warp reads its nodes' six
// values back and sums them with a shuffle tree (six independent chains, a short tail at
// the end of every warp's life), and the last warp to finish adds the warps' sums in order
// and stores one record of 8 doubles (6 sums, 2 unused: two whole 32-byte sectors) at
// partials[cta * 8 + value].  All of it in FP32 (FP64's issue rate on this part
// is a small fraction of FP32's); the records are summed in FP64 afterwards, in a fixed
// order.  Same populations, velocity and scalar as k_step.
template <typename T, int MINB, bool WALLS>
__global__ void __launch_bounds__(256, MINB) k_step_reduce(BlockView v, double* partials) {
  __shared__ float snm[8][6][32];
  __shared__ float swarp[8][6];
  __shared__ unsigned done;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  float(*col)[32] = snm[w];
#pragma unroll
  for (int i = 0; i < 6; ++i) col[i][lane] = 0.0f;
  if (t == 0) done = 0u;
  __syncthreads();                          // the counter is set before any warp counts
  const NodeMomentsOut out{&col[0][lane], 32};
  if (x < v.nx && y < v.ny) cell_update<T, uint32_t, false, WALLS, true>(v, x, y, z, &out);
  __syncwarp();
  float val[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) val[i] = col[i][lane];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 6; ++i) val[i] += __shfl_xor_sync(0xffffffffu, val[i], o);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) swarp[w][i] = val[i];
  }
  finish_cta_record(swarp, done, lane, (blockDim.x * blockDim.y + 31) >> 5, 1, partials);
}

// k_step_reduce with two nodes per thread (k_step2's update): the CTA covers the same bx x by
// nodes as k_step_reduce's and every node's moments go to the shared-memory column of the
// one-node thread that would own it (t = row * bx + x offset = 2 * thread + 0 or 1), so warp
// w holds exactly the 32-node groups 2w and 2w + 1 and sums them with the same shuffle
// tree after a warp barrier only; the last warp to finish (a shared-memory counter) adds
// the eight group sums in order.  The CTA records, and the diagnostics, are bit-identical
// to k_step_reduce's on the same node tile, and no warp waits for the others' collision.
template <typename T, int MINB, bool WALLS>
__global__ void __launch_bounds__(128, MINB) k_step2_reduce(BlockView v, double* partials) {
  __shared__ float snm[8][6][32];
  __shared__ float swarp[8][6];
  __shared__ unsigned done;
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  const int t0 = 2 * t, t1 = t0 + 1;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    snm[t0 >> 5][i][t0 & 31] = 0.0f;
    snm[t1 >> 5][i][t1 & 31] = 0.0f;
  }
  if (t == 0) done = 0u;
  __syncthreads();                          // the counter is set before any warp counts
  const NodeMomentsOut out0{&snm[t0 >> 5][0][t0 & 31], 32};
  const NodeMomentsOut out1{&snm[t1 >> 5][0][t1 & 31], 32};
  if (x < v.nx && y < v.ny) {
    if constexpr (pair_corners_async<T>()) {
      __shared__ float corners[16][128];
      cell_update_pair<T, uint32_t, WALLS, true>(v, x, y, z, &corners[0][t], 128, &out0, &out1);
    } else {
      cell_update_pair<T, uint32_t, WALLS, true>(v, x, y, z, nullptr, 0, &out0, &out1);
    }
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int g = 2 * w + h;
    float val[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) val[i] = snm[g][i][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < 6; ++i) val[i] += __shfl_xor_sync(0xffffffffu, val[i], o);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) swarp[g][i] = val[i];
    }
  }
  finish_cta_record(swarp, done, lane, (blockDim.x * blockDim.y + 31) >> 5, 2, partials);
}

// records written by one k_step_reduce launch (one per CTA)
size_t step_reduce_ctas(const BlockView& v, int bx, int by) {
  return (size_t)((v.nx + bx - 1) / bx) * ((v.ny + by - 1) / by) * v.nz;
}

// The register bound the step's autotuner chose for the block (the diagnostics add no live
// values through the collision: both bounds compile without spills).
template <typename T>
static void launch_step_reduce_t(const BlockView& v, dim3 grid, dim3 block, int minb,
                                 double* partials, cudaStream_t s) {
  if (step_scalar_bound(minb) >= 4) {
    if (v.walls) k_step_reduce<T, 4, true><<<grid, block, 0, s>>>(v, partials);
    else k_step_reduce<T, 4, false><<<grid, block, 0, s>>>(v, partials);
  } else {
    if (v.walls) k_step_reduce<T, 3, true><<<grid, block, 0, s>>>(v, partials);
    else k_step_reduce<T, 3, false><<<grid, block, 0, s>>>(v, partials);
  }
}

template <typename T, int MINB>
static void launch_step2_reduce_b(const BlockView& v, dim3 grid, dim3 block, double* partials,
                                  cudaStream_t s) {
  if (v.walls) k_step2_reduce<T, MINB, true><<<grid, block, 0, s>>>(v, partials);
  else k_step2_reduce<T, MINB, false><<<grid, block, 0, s>>>(v, partials);
}

template <typename T>
static void launch_step2_reduce_t(const BlockView& v, dim3 grid, dim3 block, int b,
                                  double* partials, cudaStream_t s) {
  if (b >= 6) launch_step2_reduce_b<T, 6>(v, grid, block, partials, s);
  else if (b == 5) launch_step2_reduce_b<T, 5>(v, grid, block, partials, s);
  else launch_step2_reduce_b<T, 4>(v, grid, block, partials, s);
}

// 32-bit indexing only (27 N < 2^32): the caller checks fits_32bit_index.  A two-node bound
// code runs k_step2_reduce (same CTA grid and records) where the block allows pairs and the
// CTA is whole warps (its warp w owns the 32-node groups 2w and 2w + 1).
cudaError_t launch_step_reduce(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                               int minb, double* partials, double* out, double* out5) {
  if (step_is_pair(minb) && step_pair_ok(v, storage, bx, by) && bx * by <= 256 &&
      ((bx / 2) * by) % 32 == 0) {
    dim3 block(bx / 2, by, 1);
    dim3 grid((v.nx + bx - 1) / bx, (v.ny + by - 1) / by, v.nz);
    if (storage == ST_FP16) launch_step2_reduce_t<__half>(v, grid, block, minb - STEP_PAIR, partials, s);
    else launch_step2_reduce_t<float>(v, grid, block, minb - STEP_PAIR, partials, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_columns(partials, step_reduce_ctas(v, bx, by), out, s, out5);
  }
  dim3 block(bx, by, 1);
  dim3 grid((v.nx + bx - 1) / bx, (v.ny + by - 1) / by, v.nz);
  if (storage == ST_FP16) launch_step_reduce_t<__half>(v, grid, block, minb, partials, s);
  else launch_step_reduce_t<float>(v, grid, block, minb, partials, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_columns(partials, step_reduce_ctas(v, bx, by), out, s, out5);
}

}  // namespace lbm
