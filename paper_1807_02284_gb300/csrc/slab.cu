// Halo planes for a domain split into slabs along z (no counterpart in the paper): one
// z-plane of block 0's current state — population rows as stored, the velocity, the scalar
// and the node flags — copied to or from a packed device buffer, so that neighbouring slabs
// (on other devices or in other processes) can exchange their edge planes before every step.
// A node next to a cut pulls from the halo plane only the 9 populations whose c_z points
// into the slab (slots 18..26 from the plane below, 0..8 from the plane above, in cube
// order), so a directed plane carries those 9 rows; the lagged velocity (central
// differences), the scalar (departure point at most one node away) and the flags (bounce-back
// and wall unknowns) are read in full.  The flags travel with the state because the derived
// bits of a halo node (obstacle surface, inflow) depend on nodes beyond the slab.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "runtime.h"

namespace lbm {

// Packed layout of one plane of P = nx * ny nodes: nk population rows (slots k0 .. k0+nk-1,
// element size of the storage), padded to a multiple of 16 bytes, then 3 velocity rows and
// 1 scalar row (FP32), then 1 flag row (bytes).  dir +1: slots with c_z = +1 (k0 18), dir -1:
// c_z = -1 (k0 0), dir 0: all 27.
static inline int plane_rows(int dir) { return dir == 0 ? 27 : 9; }
static inline int plane_first(int dir) { return dir > 0 ? 18 : 0; }
static inline size_t pop_rows_bytes(size_t P, size_t elem, int dir) {
  return ((size_t)plane_rows(dir) * P * elem + 15) / 16 * 16;
}

template <typename T, bool PACK>
__global__ void k_plane(T* f, float* u, float* c, uint8_t* flags, size_t N, size_t base,
                        size_t P, int k0, int nk, size_t pop_bytes, unsigned char* buf) {
  T* bf = reinterpret_cast<T*>(buf);
  float* bu = reinterpret_cast<float*>(buf + pop_bytes);
  uint8_t* bfl = reinterpret_cast<uint8_t*>(bu + 4 * P);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t idx = base + i;
    for (int j = 0; j < nk; ++j) {
      const size_t k = (size_t)(k0 + j);
      if (PACK) bf[j * P + i] = f[k * N + idx];
      else f[k * N + idx] = bf[j * P + i];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (PACK) bu[a * P + i] = u[a * N + idx];
      else u[a * N + idx] = bu[a * P + i];
    }
    if (PACK) bu[3 * P + i] = c[idx];
    else c[idx] = bu[3 * P + i];
    if (PACK) bfl[i] = flags[idx];
    else flags[idx] = bfl[i];
  }
}

// Plane z of level `level` of block 0 to (PACK) or from the buffer, on stream s.
template <bool PACK>
static cudaError_t launch_plane(lbm_domain* dom, int level, int z, int dir, void* buf,
                                cudaStream_t s) {
  Block& B = dom->blocks[0];
  const size_t P = (size_t)B.nx * B.ny, base = (size_t)z * P;
  const int grid = (int)std::min<size_t>((P + 255) / 256, 4096);
  Level& L = B.lv[level];
  unsigned char* b = static_cast<unsigned char*>(buf);
  const int k0 = plane_first(dir), nk = plane_rows(dir);
  if (dom->desc.storage == LBM_FP16_SHIFTED)
    k_plane<__half, PACK><<<grid, 256, 0, s>>>(static_cast<__half*>(L.f), L.u, L.c, B.flags, B.N,
                                               base, P, k0, nk, pop_rows_bytes(P, 2, dir), b);
  else
    k_plane<float, PACK><<<grid, 256, 0, s>>>(static_cast<float*>(L.f), L.u, L.c, B.flags, B.N,
                                              base, P, k0, nk, pop_rows_bytes(P, 4, dir), b);
  return cudaGetLastError();
}

}  // namespace lbm

using namespace lbm;

extern "C" size_t lbm_plane_bytes(const lbm_domain* dom, int32_t dir) {
  if (!dom || dir < -1 || dir > 1) return 0;
  const Block& B = dom->blocks[0];
  const size_t P = (size_t)B.nx * B.ny;
  return pop_rows_bytes(P, dom->desc.storage == LBM_FP16_SHIFTED ? 2 : 4, dir) +
         P * (4 * sizeof(float) + 1);
}

static lbm_status plane_args(lbm_domain* dom, int32_t z, int32_t dir, const void* buf) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (dir < -1 || dir > 1) return dom->fail(LBM_ERR_INVALID_ARG, "plane direction is -1, 0 or +1");
  if (!buf || reinterpret_cast<uintptr_t>(buf) % 16)
    return dom->fail(LBM_ERR_INVALID_ARG, "plane buffer null or not 16-byte aligned");
  if (dom->blocks.size() != 1) return dom->fail(LBM_ERR_UNSUPPORTED, "slab planes need a single-block domain");
  if (dom->tape) return dom->fail(LBM_ERR_STATE, "planes cannot be exchanged while a tape records");
  if (z < 0 || z >= dom->blocks[0].nz) return dom->fail(LBM_ERR_INVALID_ARG, "plane index out of range");
  return LBM_OK;
}

extern "C" lbm_status lbm_pack_plane(lbm_domain* dom, int32_t z, int32_t dir, void* dev_buf) {
  lbm_status st = plane_args(dom, z, dir, dev_buf);
  if (st != LBM_OK) return st;
  const cudaError_t e = launch_plane<true>(dom, dom->blocks[0].cur, z, dir, dev_buf, dom->stream);
  return e == cudaSuccess ? LBM_OK : dom->cuda_fail(e, "pack plane");
}

extern "C" lbm_status lbm_unpack_plane(lbm_domain* dom, int32_t z, int32_t dir,
                                       const void* dev_buf) {
  lbm_status st = plane_args(dom, z, dir, dev_buf);
  if (st != LBM_OK) return st;
  const cudaError_t e = launch_plane<false>(dom, dom->blocks[0].cur, z, dir,
                                            const_cast<void*>(dev_buf), dom->stream);
  return e == cudaSuccess ? LBM_OK : dom->cuda_fail(e, "unpack plane");
}

// One step of a slab whose halo exchange overlaps its work: the owned planes next to the
// halos (the planes the neighbours need next) are stepped first, packed on pack_stream as soon
// as they are written, while the remaining owned planes are stepped on the domain's stream;
// halo planes are not stepped (the next unpack overwrites what the pull reads of them).
extern "C" lbm_status lbm_step_slab(lbm_domain* dom, int32_t lo, int32_t hi, void* send_lo,
                                    void* send_hi, void* pack_stream) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (dom->blocks.size() != 1) return dom->fail(LBM_ERR_UNSUPPORTED, "slab steps need a single-block domain");
  if (dom->tape) return dom->fail(LBM_ERR_STATE, "slab steps do not record an adjoint tape");
  Block& B = dom->blocks[0];
  const int zlo = lo ? 1 : 0, zhi = hi ? B.nz - 2 : B.nz - 1;   // first and last owned plane
  if (zhi - zlo < 1) return dom->fail(LBM_ERR_INVALID_ARG, "a slab step needs at least two owned planes");
  auto bad = [](const void* b) { return !b || reinterpret_cast<uintptr_t>(b) % 16 != 0; };
  if ((lo && bad(send_lo)) || (hi && bad(send_hi)))
    return dom->fail(LBM_ERR_INVALID_ARG, "send buffer null or not 16-byte aligned");
  if (*dom->h_err & 1) return dom->fail(LBM_ERR_DIVERGED, "divergence recorded by an earlier step");
  lbm_status st = dom->autotune_tiles(0);
  if (st != LBM_OK) return st;
  cudaStream_t ps = static_cast<cudaStream_t>(pack_stream);
  if (!ps) {
    st = dom->aux(&ps);
    if (st != LBM_OK) return st;
  }
  cudaEvent_t ev = dom->event(7);
  if (!ev) return dom->fail(LBM_ERR_CUDA, "cudaEventCreate");
  const int nxt = B.cur ^ 1;
  const BlockView v = dom->view(0, B.cur, nxt);
  const int storage = dom->desc.storage;
  cudaError_t e = cudaSuccess;
  if (lo) e = launch_step_planes(v, storage, B.bx, B.by, dom->stream, B.minb, zlo, 1);
  if (hi && e == cudaSuccess) e = launch_step_planes(v, storage, B.bx, B.by, dom->stream, B.minb, zhi, 1);
  if ((lo || hi) && e == cudaSuccess) {
    e = cudaEventRecord(ev, dom->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ps, ev, 0);
    if (lo && e == cudaSuccess) e = launch_plane<true>(dom, nxt, zlo, -1, send_lo, ps);
    if (hi && e == cudaSuccess) e = launch_plane<true>(dom, nxt, zhi, +1, send_hi, ps);
  }
  const int i0 = zlo + (lo ? 1 : 0), i1 = zhi - (hi ? 1 : 0);
  if (e == cudaSuccess) e = launch_step_planes(v, storage, B.bx, B.by, dom->stream, B.minb, i0, i1 - i0 + 1);
  if (e != cudaSuccess) return dom->cuda_fail(e, "slab step");
  B.cur = nxt;
  ++dom->steps;
  return LBM_OK;
}
