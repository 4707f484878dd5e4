// The collide-stream step with the block diagnostics fused in (lbm_step_reduce): the same
// per-node update as k_step, plus the sums that lbm_reduce would take in a second pass.
#include "lbm_cell.cuh"

namespace lbm {

// A step that also sums the diagnostics of the state it stores (lbm_step_reduce): every node
// writes its moments into its warp's shared-memory columns as soon as they are known, so
// nothing is held through the collision; after the update each warp reads its nodes' six
// values back and sums them with a shuffle tree (six independent chains, a short tail at
// the end of every warp's life), and once every warp is done warp 0 adds the warps' sums in
// order and stores one record of 8 doubles (6 sums, 2 unused: two whole 32-byte sectors) at
// partials[cta * 8 + value].  All of it in FP32 (FP64's issue rate on this part
// is a small fraction of FP32's); the records are summed in FP64 afterwards, in a fixed
// order.  Same populations, velocity and scalar as k_step.
template <typename T, int MINB, bool WALLS>
__global__ void __launch_bounds__(256, MINB) k_step_reduce(BlockView v, double* partials) {
  __shared__ float snm[8][6][32];
  __shared__ float swarp[8][6];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  float(*col)[32] = snm[w];
#pragma unroll
  for (int i = 0; i < 6; ++i) col[i][lane] = 0.0f;
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
  __syncthreads();
  if (t < 8) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    float s = 0.0f;
    if (t < 6)
      for (int k = 0; k < nw; ++k) s += swarp[k][t];
    const size_t cta = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    partials[cta * 8 + t] = (double)s;
  }
}

// k_step_reduce with two nodes per thread (k_step2's update): the CTA covers the same bx x by
// nodes as k_step_reduce's, every node's moments go to the shared-memory column of the
// one-node thread that would own it (t = row * bx + x offset), and each warp sums two of
// the eight 32-column groups with the same shuffle tree, so the CTA records (and the
// diagnostics) are bit-identical to k_step_reduce's.
template <typename T, int MINB, bool WALLS>
__global__ void __launch_bounds__(128, MINB) k_step2_reduce(BlockView v, double* partials) {
  __shared__ float snm[8][6][32];
  __shared__ float swarp[8][6];
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  const int bx = 2 * blockDim.x;
  const int t0 = threadIdx.y * bx + 2 * threadIdx.x, t1 = t0 + 1;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    snm[t0 >> 5][i][t0 & 31] = 0.0f;
    snm[t1 >> 5][i][t1 & 31] = 0.0f;
  }
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
  __syncthreads();
  const int lane = t & 31, w = t >> 5;
  const int nv = (bx * blockDim.y + 31) >> 5;     // 32-node groups of the tile
  for (int g = w; g < nv; g += (blockDim.x * blockDim.y + 31) >> 5) {
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
  __syncthreads();
  if (t < 8) {
    float s = 0.0f;
    if (t < 6)
      for (int k = 0; k < nv; ++k) s += swarp[k][t];
    const size_t cta = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    partials[cta * 8 + t] = (double)s;
  }
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
// code runs k_step2_reduce (same CTA grid and records) where the block allows pairs.
cudaError_t launch_step_reduce(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                               int minb, double* partials, double* out, double* out5) {
  if (step_is_pair(minb) && step_pair_ok(v, storage, bx, by) && bx * by <= 256) {
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
