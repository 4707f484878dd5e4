// Dynamic scale construction (Sec. 5): detection of the samples that need a finer scale,
// placement of a box block around them, and the start of a new block from the coarser scale
// it is overlaid on.
//
// Detection keeps the nodes whose gradient magnitude (the Frobenius norm of the
// central-difference Jacobian of the stored velocity, the quantity of the adaptive factor)
// reaches g_threshold and whose velocity magnitude reaches u_threshold; obstacle and ghost
// nodes never count.  Count and bounding box are order-independent reductions (sum, min,
// max), so the result is deterministic.  A new block is placed around the box widened by a
// margin and clipped to the reference block; its obstacle and scalar-source bits come from
// the nearest node of its prior-mapping source, and every other node is started from that
// source by the Sec. 3.2 mapping at the current time.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "lbm_cell.cuh"
#include "runtime.h"

namespace lbm {

struct RegionOut {
  unsigned long long count;
  int lo[3];
  int hi[3];
};

__global__ void k_detect_init(RegionOut* out) {
  out->count = 0ull;
  for (int a = 0; a < 3; ++a) {
    out->lo[a] = INT_MAX;
    out->hi[a] = -1;
  }
}

// Persistent over the (y, z) rows of the block, threads along x; per-CTA reduction, then
// one atomic per quantity and CTA.
__global__ void __launch_bounds__(256) k_detect(BlockView v, float g_thr, float u_thr,
                                                RegionOut* out) {
  const uint32_t N = (uint32_t)v.N;
  unsigned cnt = 0;
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
  const int rows = v.ny * v.nz;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int y = r % v.ny, z = r / v.ny;
    for (int x = threadIdx.x; x < v.nx; x += blockDim.x) {
      const uint32_t idx = ((uint32_t)z * (uint32_t)v.ny + (uint32_t)y) * (uint32_t)v.nx + (uint32_t)x;
      if (v.flags[idx] & (F_SOLID | F_GHOST)) continue;
      const Nbr<uint32_t> n = neighbours<uint32_t>(v, x, y, z);
      const float g = grad_norm<uint32_t>(v.u_in, N, n);
      const float ux = v.u_in[idx], uy = v.u_in[N + idx], uz = v.u_in[2 * N + idx];
      const float um = sqrtf(ux * ux + uy * uy + uz * uz);
      if (g >= g_thr && um >= u_thr) {
        ++cnt;
        lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
        lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
        lo[2] = min(lo[2], z); hi[2] = max(hi[2], z);
      }
    }
  }
  const unsigned full = 0xffffffffu;
  cnt = __reduce_add_sync(full, cnt);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(full, lo[a]);
    hi[a] = __reduce_max_sync(full, hi[a]);
  }
  __shared__ unsigned s_cnt[8];
  __shared__ int s_lo[8][3], s_hi[8][3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_cnt[w] = cnt;
    for (int a = 0; a < 3; ++a) { s_lo[w][a] = lo[a]; s_hi[w][a] = hi[a]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned c = 0;
    int l[3] = {INT_MAX, INT_MAX, INT_MAX}, h[3] = {-1, -1, -1};
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      c += s_cnt[i];
      for (int a = 0; a < 3; ++a) { l[a] = min(l[a], s_lo[i][a]); h[a] = max(h[a], s_hi[i][a]); }
    }
    if (c) {
      atomicAdd(&out->count, (unsigned long long)c);
      for (int a = 0; a < 3; ++a) {
        atomicMin(&out->lo[a], l[a]);
        atomicMax(&out->hi[a], h[a]);
      }
    }
  }
}

// Count and bounding box of the nodes carrying any of `mask` (per-CTA reduction, one atomic
// per quantity and CTA).
__global__ void __launch_bounds__(256) k_flag_box(const uint8_t* __restrict__ flags, int nx, int ny,
                                                  int nz, uint8_t mask, RegionOut* out) {
  unsigned cnt = 0;
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
  for (int r = blockIdx.x; r < ny * nz; r += gridDim.x) {
    const int y = r % ny, z = r / ny;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      if (!(flags[((size_t)z * ny + y) * nx + x] & mask)) continue;
      ++cnt;
      lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
      lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
      lo[2] = min(lo[2], z); hi[2] = max(hi[2], z);
    }
  }
  const unsigned full = 0xffffffffu;
  cnt = __reduce_add_sync(full, cnt);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = __reduce_min_sync(full, lo[a]);
    hi[a] = __reduce_max_sync(full, hi[a]);
  }
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(&out->count, (unsigned long long)cnt);
    for (int a = 0; a < 3; ++a) {
      atomicMin(&out->lo[a], lo[a]);
      atomicMax(&out->hi[a], hi[a]);
    }
  }
}

// Obstacle and scalar-source bits of a block from the nearest node of another block (index
// floor(q + 1/2) of the node's position q in the source's node units, clamped); the ghost
// bit of the destination is kept, every other bit cleared.
__global__ void k_nearest_flags(uint8_t* dflags, int dnx, int dny, int dnz, double o0, double o1,
                                double o2, double dh, const uint8_t* sflags, int snx, int sny,
                                int snz, double s0, double s1, double s2, double sh) {
  const size_t N = (size_t)dnx * dny * dnz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int node[3] = {(int)(idx % dnx), (int)((idx / dnx) % dny), (int)(idx / ((size_t)dnx * dny))};
    const double od[3] = {o0, o1, o2}, os[3] = {s0, s1, s2};
    const int sn[3] = {snx, sny, snz};
    int j[3];
    for (int a = 0; a < 3; ++a) {
      const double p = __dadd_rn(od[a], __dmul_rn((double)node[a], dh));
      const double q = __ddiv_rn(__dsub_rn(p, os[a]), sh);
      j[a] = max(0, min((int)floor(q + 0.5), sn[a] - 1));
    }
    const uint8_t src = sflags[((size_t)j[2] * sny + j[1]) * snx + j[0]];
    dflags[idx] = (uint8_t)((dflags[idx] & F_GHOST) | (src & (F_SOLID | F_SCALAR_SRC)));
  }
}

// Soft-shadow wake of the static scale construction (Sec. 5): every non-obstacle node of the
// slab a0 <= coordinate <= a1 along `axis` counts the light samples (lights: M points, 3
// ints each) whose segment to it crosses no obstacle voxel.  The segment is walked in 2 m
// steps (m its largest coordinate difference), step k checked at the nearest voxel of
// p + d k / (2 m) in integer arithmetic (end points not checked).  A node that sees c samples
// belongs to the wake of refined scale s = 1 .. nsc - 1 when c (nsc - 1) <= (nsc - 1 - s) M;
// out[s - 1] receives the count and bounding box of those nodes (per-thread, then per-warp
// reductions, then one atomic per warp and value: the result does not depend on order).
constexpr int SHADOW_MAX_SCALES = 8;

__global__ void __launch_bounds__(256) k_shadow(const uint8_t* __restrict__ flags, int nx, int ny,
                                                int nz, int axis, int a0, int a1,
                                                const int* __restrict__ lights, int M, int nsc,
                                                RegionOut* out) {
  int ext[3] = {nx, ny, nz}, org[3] = {0, 0, 0};
  ext[axis] = a1 - a0 + 1;
  org[axis] = a0;
  const long long total = (long long)ext[0] * ext[1] * ext[2];
  unsigned cnt[SHADOW_MAX_SCALES - 1];
  int lo[SHADOW_MAX_SCALES - 1][3], hi[SHADOW_MAX_SCALES - 1][3];
#pragma unroll
  for (int s = 0; s < SHADOW_MAX_SCALES - 1; ++s) {
    cnt[s] = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) { lo[s][a] = INT_MAX; hi[s][a] = -1; }
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p[3] = {org[0] + (int)(i % ext[0]), org[1] + (int)((i / ext[0]) % ext[1]),
                      org[2] + (int)(i / ((long long)ext[0] * ext[1]))};
    if (flags[((size_t)p[2] * ny + p[1]) * nx + p[0]] & F_SOLID) continue;
    int c = 0;
    for (int j = 0; j < M; ++j) {
      const long long d[3] = {(long long)lights[3 * j] - p[0], (long long)lights[3 * j + 1] - p[1],
                              (long long)lights[3 * j + 2] - p[2]};
      long long m = d[0] < 0 ? -d[0] : d[0];
      for (int a = 1; a < 3; ++a) m = max(m, d[a] < 0 ? -d[a] : d[a]);
      const long long n = 2 * m;
      bool blocked = false;
      for (long long k = 1; k < n && !blocked; ++k) {
        long long v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = (2 * (p[a] * n + d[a] * k) + n) / (2 * n);
        blocked = (flags[((size_t)v[2] * ny + v[1]) * nx + v[0]] & F_SOLID) != 0;
      }
      c += blocked ? 0 : 1;
    }
#pragma unroll
    for (int s = 1; s < SHADOW_MAX_SCALES; ++s) {
      if (s < nsc && (long long)c * (nsc - 1) <= (long long)(nsc - 1 - s) * M) {
        ++cnt[s - 1];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lo[s - 1][a] = min(lo[s - 1][a], p[a]);
          hi[s - 1][a] = max(hi[s - 1][a], p[a]);
        }
      }
    }
  }
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int s = 0; s < SHADOW_MAX_SCALES - 1; ++s) {
    const unsigned cs = __reduce_add_sync(full, cnt[s]);
    int l[3], h[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      l[a] = __reduce_min_sync(full, lo[s][a]);
      h[a] = __reduce_max_sync(full, hi[s][a]);
    }
    if ((threadIdx.x & 31) == 0 && cs && s + 1 < nsc) {
      atomicAdd(&out[s].count, (unsigned long long)cs);
      for (int a = 0; a < 3; ++a) {
        atomicMin(&out[s].lo[a], l[a]);
        atomicMax(&out[s].hi[a], h[a]);
      }
    }
  }
}

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_detect_region(lbm_domain* dom, int32_t block_id, double g_threshold,
                                        double u_threshold, int64_t* count, int32_t box[6]) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  if (!count || !box) return dom->fail(LBM_ERR_INVALID_ARG, "null output");
  if (!std::isfinite(g_threshold) || !std::isfinite(u_threshold))
    return dom->fail(LBM_ERR_INVALID_ARG, "thresholds must be finite");
  const Block& B = dom->blocks[block_id];
  if (27ull * B.N >= 0xFFFFFFFFull) return dom->fail(LBM_ERR_UNSUPPORTED, "block too large for detection");
  // the result area reuses the reduction's read-back buffers (both calls synchronise)
  RegionOut* d_out = reinterpret_cast<RegionOut*>(dom->d_red);
  BlockView v = dom->view(block_id, B.cur, B.cur);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dom->desc.device);
  const int rows = B.ny * B.nz;
  const int grid = std::max(1, std::min(rows, 8 * std::max(sms, 1)));
  k_detect_init<<<1, 1, 0, dom->stream>>>(d_out);
  k_detect<<<grid, 256, 0, dom->stream>>>(v, (float)g_threshold, (float)u_threshold, d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dom->h_red, d_out, sizeof(RegionOut), cudaMemcpyDeviceToHost, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "region detection");
  st = dom->sync_and_check();
  if (st != LBM_OK) return st;
  RegionOut r;
  std::memcpy(&r, dom->h_red, sizeof(RegionOut));
  *count = (int64_t)r.count;
  for (int a = 0; a < 3; ++a) {
    box[a] = r.count ? r.lo[a] : 0;
    box[3 + a] = r.count ? r.hi[a] : -1;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_init_block_from_parent(lbm_domain* dom, int32_t block_id) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  lbm_status st = dom->check_block(block_id);
  if (st != LBM_OK) return st;
  if (block_id == 0) return dom->fail(LBM_ERR_INVALID_ARG, "the reference block has no parent");
  if (dom->blocks[block_id].far) return dom->fail(LBM_ERR_INVALID_ARG, "far-field blocks are started with lbm_init_macro");
  if (dom->walls & WALLS_OBSTACLES)
    return dom->fail(LBM_ERR_UNSUPPORTED, "blocks started from their parent do not take obstacle-surface walls");
  Block& B = dom->blocks[block_id];
  const Block& P = dom->blocks[B.prior.src];
  cudaError_t e;
  {
    const size_t g = std::min<size_t>((B.N + 255) / 256, 65535);
    k_nearest_flags<<<(int)g, 256, 0, dom->stream>>>(
        B.flags, B.nx, B.ny, B.nz, B.origin[0], B.origin[1], B.origin[2], B.h, P.flags, P.nx,
        P.ny, P.nz, P.origin[0], P.origin[1], P.origin[2], P.h);
    e = cudaGetLastError();
  }
  const int per[3] = {0, 0, 0};
  if (e == cudaSuccess) e = launch_near_solid(B.flags, B.nx, B.ny, B.nz, per, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "block flags");
  st = dom->clear_block(block_id);   // rest state everywhere (obstacle nodes keep it)
  if (st != LBM_OK) return st;
  MapArgs a{};
  a.table = nullptr;
  a.n = (int)B.N;
  a.f_lo = a.f_hi = P.lv[P.cur].f;
  a.c_lo = a.c_hi = P.lv[P.cur].c;
  a.theta = 0.0f;
  a.src_flags = P.flags;
  a.snx = P.nx; a.sny = P.ny; a.snz = P.nz; a.sN = P.N;
  a.f_dst = B.lv[B.cur].f;
  a.u_dst = B.lv[B.cur].u;
  a.c_dst = B.lv[B.cur].c;
  a.dst_flags = B.flags;
  a.skip_mask = F_SOLID;
  a.dN = B.N;
  a.khat = B.prior.khat;
  for (int k = 0; k < 3; ++k) { a.o_dst[k] = B.origin[k]; a.o_src[k] = P.origin[k]; }
  a.h_dst = B.h;
  a.h_src = P.h;
  a.dnx = B.nx; a.dny = B.ny;
  e = launch_map(a, dom->desc.storage, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "block start mapping");
  dom->invalidate_graphs();
  return LBM_OK;
}

extern "C" lbm_status lbm_build_dynamic_scale(lbm_domain* dom, int32_t src_block, double h,
                                              double g_threshold, double u_threshold,
                                              int32_t margin, int32_t replace_last,
                                              int32_t* block_id) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (!block_id) return dom->fail(LBM_ERR_INVALID_ARG, "null block_id");
  if (dom->walls & WALLS_OBSTACLES)
    return dom->fail(LBM_ERR_UNSUPPORTED, "dynamic scales do not take obstacle-surface walls");
  *block_id = -1;
  lbm_status st = dom->check_block(src_block);
  if (st != LBM_OK) return st;
  if (margin < 0) return dom->fail(LBM_ERR_INVALID_ARG, "margin must be >= 0");
  if (!(h > 0.0 && h < 1.0)) return dom->fail(LBM_ERR_INVALID_ARG, "h must be in (0, 1)");
  {
    const Block& B0 = dom->blocks[0];
    const int m = std::max(B0.nx, std::max(B0.ny, B0.nz));
    if ((double)m / h > 65535.0) return dom->fail(LBM_ERR_INVALID_ARG, "h too small for this reference block");
  }
  const int last = (int)dom->blocks.size() - 1;
  if (replace_last && (last < 1 || src_block == last || dom->blocks[last].far))
    return dom->fail(LBM_ERR_INVALID_ARG, "replace_last needs a refined last block other than the source");
  int64_t count = 0;
  int32_t box[6];
  st = lbm_detect_region(dom, src_block, g_threshold, u_threshold, &count, box);
  if (st != LBM_OK) return st;
  // geometry of the source block, read before any removal
  const Block& S = dom->blocks[src_block];
  const double so[3] = {S.origin[0], S.origin[1], S.origin[2]};
  const double sh = S.h;
  const int ref[3] = {dom->blocks[0].nx, dom->blocks[0].ny, dom->blocks[0].nz};
  if (replace_last) {
    st = lbm_remove_scale_block(dom, last);
    if (st != LBM_OK) return st;
  }
  if (count == 0) return LBM_OK;
  double origin[3];
  int32_t dims[3];
  for (int a = 0; a < 3; ++a) {
    const double top = (double)(ref[a] - 1);
    double lo = std::max(so[a] + (box[a] - margin) * sh, 0.0);
    const double hi = std::min(so[a] + (box[3 + a] + margin) * sh, top);
    const int n = std::max((int)std::floor((hi - lo) / h + 1e-9) + 1, 4);
    if (lo + (n - 1) * h > top + 1e-9) lo = std::max(0.0, top - (n - 1) * h);
    origin[a] = lo;
    dims[a] = n;
  }
  int32_t id = -1;
  st = lbm_add_scale_block(dom, origin, h, dims, &id);
  if (st != LBM_OK) return st;
  st = lbm_init_block_from_parent(dom, id);
  if (st != LBM_OK) {
    lbm_remove_scale_block(dom, id);
    return st;
  }
  *block_id = id;
  return LBM_OK;
}

// Static scale construction (Sec. 5); n_light > 0 shapes each scale's wake as a soft shadow
// (k_shadow), n_light == 0 extends every box straight downstream by `wake`.
static lbm_status static_scales(lbm_domain* dom, int32_t n_scales, double h_min, double d_max,
                                double wake, int32_t flow_axis, int32_t n_light,
                                int32_t* n_added) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (!n_added) return dom->fail(LBM_ERR_INVALID_ARG, "null n_added");
  *n_added = 0;
  if (dom->walls & WALLS_OBSTACLES)
    return dom->fail(LBM_ERR_UNSUPPORTED, "static scales do not take obstacle-surface walls");
  if (n_scales < 2 || !(h_min > 0.0 && h_min < 1.0) || !(d_max >= 0.0) || !(wake >= 0.0) ||
      flow_axis < 0 || flow_axis > 2)
    return dom->fail(LBM_ERR_INVALID_ARG, "need n_scales >= 2, 0 < h_min < 1, d_max, wake >= 0, axis 0..2");
  if (n_light < 0 || (n_light > 0 && n_scales > SHADOW_MAX_SCALES))
    return dom->fail(LBM_ERR_INVALID_ARG, "a shadow-shaped wake needs n_light >= 1 and n_scales <= 8");
  const Block& B0 = dom->blocks[0];
  RegionOut* d_out = reinterpret_cast<RegionOut*>(dom->d_red);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dom->desc.device);
  const int grid = std::max(1, std::min(B0.ny * B0.nz, 8 * std::max(sms, 1)));
  k_detect_init<<<1, 1, 0, dom->stream>>>(d_out);
  k_flag_box<<<grid, 256, 0, dom->stream>>>(B0.flags, B0.nx, B0.ny, B0.nz, F_SOLID, d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dom->h_red, d_out, sizeof(RegionOut), cudaMemcpyDeviceToHost, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "obstacle box");
  lbm_status st = dom->sync_and_check();
  if (st != LBM_OK) return st;
  RegionOut r;
  std::memcpy(&r, dom->h_red, sizeof(RegionOut));
  if (r.count == 0) return LBM_OK;
  const int ref[3] = {B0.nx, B0.ny, B0.nz};
  // the wake of every refined scale: a straight extension, or the soft shadow's boxes
  std::vector<RegionOut> shadow;
  if (n_light > 0) {
    // light samples: the inflow nodes (every ceil(count / n_light)-th in index order), or the
    // nodes of the upstream face without inflow nodes
    std::vector<uint8_t> fl(B0.N);
    e = cudaMemcpyAsync(fl.data(), B0.flags, B0.N, cudaMemcpyDeviceToHost, dom->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(dom->stream);
    if (e != cudaSuccess) return dom->cuda_fail(e, "flags read-back");
    std::vector<int> pts;
    for (int pass = 0; pass < 2 && pts.empty(); ++pass)
      for (size_t i = 0; i < B0.N; ++i) {
        const int x = (int)(i % B0.nx), y = (int)((i / B0.nx) % B0.ny), z = (int)(i / ((size_t)B0.nx * B0.ny));
        const int c[3] = {x, y, z};
        if (pass == 0 ? (fl[i] & F_INFLOW) != 0 : c[flow_axis] == 0) {
          pts.push_back(x); pts.push_back(y); pts.push_back(z);
        }
      }
    const size_t count = pts.size() / 3, stride = (count + n_light - 1) / n_light;
    std::vector<int> lights;
    for (size_t j = 0; j < count; j += stride)
      for (int a = 0; a < 3; ++a) lights.push_back(pts[3 * j + a]);
    const int M = (int)(lights.size() / 3);
    const int a0 = r.lo[flow_axis];
    const int a1 = std::min((int)std::floor(r.hi[flow_axis] + wake), ref[flow_axis] - 1);
    int* d_lights = static_cast<int*>(dom->dev_alloc(lights.size() * sizeof(int)));
    RegionOut* d_sh = static_cast<RegionOut*>(dom->dev_alloc((SHADOW_MAX_SCALES - 1) * sizeof(RegionOut)));
    if (!d_lights || !d_sh) {
      dom->dev_free(d_lights);
      dom->dev_free(d_sh);
      return dom->fail(LBM_ERR_OOM, "shadow buffers");
    }
    shadow.resize(SHADOW_MAX_SCALES - 1);
    e = cudaMemcpyAsync(d_lights, lights.data(), lights.size() * sizeof(int), cudaMemcpyHostToDevice, dom->stream);
    for (int s = 0; s < SHADOW_MAX_SCALES - 1 && e == cudaSuccess; ++s) {
      k_detect_init<<<1, 1, 0, dom->stream>>>(d_sh + s);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_shadow<<<std::max(sms, 1) * 8, 256, 0, dom->stream>>>(B0.flags, B0.nx, B0.ny, B0.nz, flow_axis, a0, a1,
                                                          d_lights, M, n_scales, d_sh);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(shadow.data(), d_sh, (SHADOW_MAX_SCALES - 1) * sizeof(RegionOut),
                          cudaMemcpyDeviceToHost, dom->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(dom->stream);
    dom->dev_free(d_lights);
    dom->dev_free(d_sh);
    if (e != cudaSuccess) return dom->cuda_fail(e, "shadow");
  }
  for (int i = 1; i < n_scales; ++i) {
    const double h = 1.0 + (h_min - 1.0) * i / (n_scales - 1);
    const double d = d_max * (n_scales - 1 - i) / (n_scales - 1);
    double origin[3];
    int32_t dims[3];
    for (int a = 0; a < 3; ++a) {
      const double top = (double)(ref[a] - 1);
      double lo = r.lo[a] - d, hi = r.hi[a] + d;
      if (n_light > 0) {
        if (shadow[i - 1].count) {
          lo = std::min(lo, (double)shadow[i - 1].lo[a]);
          hi = std::max(hi, (double)shadow[i - 1].hi[a]);
        }
      } else if (a == flow_axis) {
        hi += wake;
      }
      lo = std::max(lo, 0.0);
      hi = std::min(hi, top);
      const int n = std::max((int)std::floor((hi - lo) / h + 1e-9) + 1, 4);
      if (lo + (n - 1) * h > top + 1e-9) lo = std::max(0.0, top - (n - 1) * h);
      origin[a] = lo;
      dims[a] = n;
    }
    int32_t id = -1;
    st = lbm_add_scale_block(dom, origin, h, dims, &id);
    if (st != LBM_OK) return st;
    st = lbm_init_block_from_parent(dom, id);
    if (st != LBM_OK) {
      lbm_remove_scale_block(dom, id);
      return st;
    }
    ++*n_added;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_build_static_scales(lbm_domain* dom, int32_t n_scales, double h_min,
                                              double d_max, double wake, int32_t flow_axis,
                                              int32_t* n_added) {
  return static_scales(dom, n_scales, h_min, d_max, wake, flow_axis, 0, n_added);
}

extern "C" lbm_status lbm_build_static_scales_shadow(lbm_domain* dom, int32_t n_scales,
                                                     double h_min, double d_max, double wake,
                                                     int32_t flow_axis, int32_t n_light,
                                                     int32_t* n_added) {
  if (dom && n_light < 1) return dom->fail(LBM_ERR_INVALID_ARG, "n_light must be >= 1");
  return static_scales(dom, n_scales, h_min, d_max, wake, flow_axis, n_light, n_added);
}

