// Internal (non-ABI) declarations shared by the runtime and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

enum Storage : int { ST_FP32 = 0, ST_FP16 = 1 };

// Everything one collide-stream launch needs about one block of nodes.
struct BlockView {
  const void* d_in;    // shifted populations at time t, 27 planes of N (cube order)
  void* d_out;         // same at t + dt
  const float* u_in;   // velocity stored at t (lagged field for |grad u|), 3 planes
  float* u_out;
  const float* c_in;   // passive scalar
  float* c_out;
  const uint8_t* flags;
  int nx, ny, nz;
  int per[3];
  size_t N;
  RelaxParams rp;
  float c_src;
  int* err;            // device error word (bit 0: non-finite or non-positive density)
  int walls = 0;       // no-slip wall faces, bits x-, x+, y-, y+, z-, z+ (nodes flagged F_WALL),
                       // and WALLS_OBSTACLES: obstacle surfaces are walls (F_OBST_WALL)
  // temporal alignment fused into the last sub-step of a refined block (Sec. 4.2.4): the
  // stored state is L0 f(t_n) + L1 f(t_n+(l-1)h) + L2 f(t_n+lh), with f(t_n+(l-1)h) = d_in
  const void* f_al0 = nullptr;   // populations at t_n
  const float* c_al0 = nullptr;  // scalar at t_n
  float al0 = 0.f, al1 = 0.f, al2 = 0.f;
  int z_first = 0;     // plane of the launch's first z index (a launch over some planes only)
};

// One node mapped between scales: destination node index, index of the source cell's
// lower corner (i0, j0, k0) and the trilinear fractions along x, y, z.
struct MapEntry {
  uint32_t dst;
  uint32_t src;
  float tx, ty, tz;
};

// Arguments of one prior- or post-mapping launch (Sec. 3.2 / 4.2).
struct MapArgs {
  const MapEntry* table;
  int n;
  // source block: populations at the two time levels mixed with weight theta (prior-mapping
  // interpolates the source in time; post-mapping uses lo only, theta = 0)
  const void* f_lo;
  const void* f_hi;
  const float* c_lo;
  const float* c_hi;
  float theta;
  const uint8_t* src_flags;
  int snx, sny;
  size_t sN;
  // destination block level
  void* f_dst;
  float* u_dst;
  float* c_dst;
  const uint8_t* dst_flags;
  uint8_t skip_mask;   // destination nodes with any of these flags are left alone
  size_t dN;
  float khat;          // K_hat factor of moments 4..8 (1 for all others)
  // a destination whose 8 source corners are all obstacle voxels: rest state (scale
  // boundaries, which have no update of their own) or left unchanged (post-mapped nodes)
  int rest_if_empty;
  // table == nullptr: entry e is destination node e of a whole block, its source cell
  // computed from the two blocks' geometry (reference units) instead of read from a table
  double o_dst[3], h_dst;
  double o_src[3], h_src;
  int dnx, dny;
  int snz;
  // ghost layers of refined blocks (k_map modes 4 and 5): the trilinear interpolant of the
  // gathered source level is also stored here (GHOST_PLANES planes of n floats), and mode 4
  // blends it in time with the interpolant `ghost_blend` of the source's earlier level
  float* ghost_store;
  const float* ghost_blend;
};

// One tile of the batched work list: a BX x BY patch of one z-plane of one simulation.
struct WorkItem {
  int view;            // index into the BlockView array
  int x0, y0, z;
};

// ---- kernels_step.cu
// Register-bound code of the collide-stream launch (chosen by autotuning with the tile
// bx x by of nodes): 3 or 4 = CTAs of bx by one-node threads per SM; STEP_PAIR + b = the
// two-node kernel k_step2 (bx / 2 x by threads per CTA, b = 4, 5 or 6 CTAs per SM), which
// needs an even nx and falls back to the one-node kernel (bound 4) otherwise.  Kernels
// without a two-node form (fused diagnostics, fused alignment) take step_scalar_bound.
constexpr int STEP_PAIR = 16;
inline bool step_is_pair(int minb) { return minb >= STEP_PAIR; }
inline int step_scalar_bound(int minb) { return minb >= STEP_PAIR ? 4 : minb; }
// Whether the two-node kernels can run this view with the node tile bx x by (even nx,
// pair-aligned arrays, at most 128 threads).
bool step_pair_ok(const BlockView& v, int storage, int bx, int by);
cudaError_t launch_step(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                        int minb = 3);
cudaError_t launch_step_align(const BlockView& v, int bx, int by, cudaStream_t s, int minb = 3);
cudaError_t launch_init(const BlockView& v, int storage, const float* rho, const float* u,
                        const float* c, cudaStream_t s);
cudaError_t launch_merge_user_flags(uint8_t* flags, const uint8_t* user, size_t N,
                                    cudaStream_t s);
cudaError_t launch_mark_walls(uint8_t* flags, int nx, int ny, int nz, int walls, cudaStream_t s);
cudaError_t launch_obstacle_walls(uint8_t* flags, int nx, int ny, int nz, const int per[3], int on,
                                  cudaStream_t s);
cudaError_t launch_near_solid(uint8_t* flags, int nx, int ny, int nz, const int per[3],
                              cudaStream_t s);
// one member of lbm_set_inflow_batch: its flags, velocity levels (up to 3, unused null),
// dims and error word
struct InflowMember {
  uint8_t* flags;
  float* u[3];
  int nx, ny, nz, pad;
  size_t N;
  int* err;
};
cudaError_t launch_inflow_records_multi(const void* rec, int n, const int* member_of,
                                        const InflowMember* members, cudaStream_t s);
cudaError_t launch_inflow_records(const void* rec, int n, uint8_t* flags, float* const* u_levels,
                                  int n_levels, int nx, int ny, int nz, size_t N, int* err,
                                  cudaStream_t s);
// fields: 0 = populations f (27 planes, paper order), 1 = u, 2 = scalar, 3 = rho
cudaError_t launch_read_f(const void* d, int storage, size_t N, void* out, int out_f64,
                          cudaStream_t s);
cudaError_t launch_write_f(void* d, int storage, size_t N, const void* in, int in_f64,
                           cudaStream_t s);
cudaError_t launch_read_rho(const void* d, int storage, size_t N, float* out, cudaStream_t s);
cudaError_t launch_convert(const void* in, int in_f64, void* out, int out_f64, size_t n,
                           cudaStream_t s);
// deterministic reduction of mass, momentum and kinetic energy over non-solid, non-ghost
// nodes (per-thread compensated FP32 sums of per-node FP32 values, combined in FP64 in a
// fixed order):
// writes per-CTA partials into `partials` (REDUCE_CTAS * 6 doubles) and the
// final six doubles {count, sum drho, sum jx, sum jy, sum jz, sum |j|^2/(2 rho)} into `out`.
constexpr int REDUCE_CTAS = 608;   // 4 CTAs on each of 152 SMs
constexpr int REDUCE_THREADS = 256;
// out: the 6 sums; out5 (optional, device): the 5 diagnostics in the lbm_reduce layout
cudaError_t launch_reduce(const void* d, int storage, const uint8_t* flags, size_t N,
                          double* partials, double* out, cudaStream_t s, double* out5 = nullptr);
// 27 N < 2^32: every array index of the block fits 32 bits
bool fits_32bit_index(size_t N);
// diagnostics of several domains in one launch: chunks of members' nodes
struct RedMember {
  const void* f;          // current populations (27 planes)
  const uint8_t* flags;
  const int* err;         // the member's device error word
  size_t N;
  int first_item, n_items;
};
struct RedItem {
  int member, pad;
  size_t start, len;
};
// records: 8 doubles per item; out: 8 doubles per member (the six launch_reduce sums, then
// the member's error word)
cudaError_t launch_reduce_items(int storage, const RedItem* items, int n_items,
                                const RedMember* members, int n_members, double* records,
                                double* out, cudaStream_t s);
// the per-member sums of item records written by another kernel (the batched step's fused
// diagnostics): member i's items are records first_item .. first_item + n_items - 1
cudaError_t launch_reduce_item_records(const double* records, const RedMember* members, int n,
                                      double* out, cudaStream_t s);
// the six sums over `n` per-CTA records of 8 doubles (partials[8 i + value]); the buffer
// holds 8 n + 6 * 128 doubles (the records, then the first stage's sums)
cudaError_t launch_reduce_columns(double* partials, size_t n, double* out, cudaStream_t s,
                                  double* out5 = nullptr);
// one collide-stream step of a block (32-bit indexing) that also leaves the diagnostics of
// the stored state in `out` (same six doubles as launch_reduce); `partials` holds
// 8 * step_reduce_ctas(v, bx, by) + 6 * 128 doubles
size_t step_reduce_ctas(const BlockView& v, int bx, int by);
cudaError_t launch_step_reduce(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                               int minb, double* partials, double* out, double* out5 = nullptr);

// ---- coupling.cu
cudaError_t launch_map(const MapArgs& a, int storage, cudaStream_t s);
cudaError_t launch_step_planes(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                               int minb, int z0, int count);
// ghost layer of a refined block that also keeps the source's trilinear interpolant
// (a.ghost_store): first = true maps level a.f_lo at t_n; first = false maps level a.f_hi
// blended at a.theta with the interpolant a.ghost_blend of the earlier level (FP32)
cudaError_t launch_ghost_map(const MapArgs& a, bool first, cudaStream_t s);
// ghost layer at t_n + theta dt_0 from the two interpolant buffers, K_hat rescaled
cudaError_t launch_ghost_finish(const MapEntry* table, int n, const float* slo, const float* shi,
                                float theta, float khat, float* f_dst, float* u_dst,
                                float* c_dst, size_t dN, cudaStream_t s);
cudaError_t launch_set_ghost_layer(uint8_t* flags, int nx, int ny, int nz, cudaStream_t s);
// outer layer of a block surrounded by a far-field block: GHOST on (except obstacle and
// inflow nodes, which keep their own update) or off
cudaError_t launch_outer_ghost(uint8_t* flags, int nx, int ny, int nz, int on, cudaStream_t s);

// ---- kernels_batch.cu
cudaError_t launch_step_batch(const BlockView* views_dev, const WorkItem* items, int n_items,
                              int storage, int bx, int by, int grid, cudaStream_t s);

}  // namespace lbm
