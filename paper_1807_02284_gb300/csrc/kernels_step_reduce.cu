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

// 32-bit indexing only (27 N < 2^32): the caller checks fits_32bit_index.
cudaError_t launch_step_reduce(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                               int minb, double* partials, double* out, double* out5) {
  dim3 block(bx, by, 1);
  dim3 grid((v.nx + bx - 1) / bx, (v.ny + by - 1) / by, v.nz);
  if (storage == ST_FP16) launch_step_reduce_t<__half>(v, grid, block, minb, partials, s);
  else launch_step_reduce_t<float>(v, grid, block, minb, partials, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_columns(partials, step_reduce_ctas(v, bx, by), out, s, out5);
}

}  // namespace lbm
