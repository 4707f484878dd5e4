// Single-block kernels: collide-stream step, equilibrium initialisation, flag derivation and
// field conversion.
#include "lbm_cell.cuh"

namespace lbm {

// Paper velocity index q (Appendix list, index 13 read as (1,0,-1)) -> cube slot k.
__constant__ int c_paper_to_cube[27] = {13, 14, 12, 16, 10, 22, 4,  17, 15, 11, 9,  23, 21, 5,
                                        3,  25, 19, 7,  1,  26, 24, 20, 18, 8,  6,  2,  0};

// MINB: CTAs of 256 threads per SM the registers are bounded for (3: 80 registers, no
// spills; 4: 64 registers with a small spill, more loads in flight); chosen by autotuning.
template <typename T, typename IT, bool ALIGN, int MINB, bool WALLS>
__global__ void __launch_bounds__(256, MINB) k_step(BlockView v) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + v.z_first;
  if (x >= v.nx || y >= v.ny) return;
  cell_update<T, IT, ALIGN, WALLS>(v, x, y, z);
}

// Two nodes (x, x + 1) per thread, x = 2 (thread's column): MINB CTAs of at most 128 threads
// per SM (128 registers per thread at 4; 96 at 5 and 80 at 6, with small spills).
template <typename T, typename IT, int MINB, bool WALLS>
__global__ void __launch_bounds__(128, MINB) k_step2(BlockView v) {
  const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z + v.z_first;
  if (x >= v.nx || y >= v.ny) return;
  if constexpr (pair_corners_async<T>()) {
    __shared__ float corners[16][128];     // each thread's scalar corners, column t
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    cell_update_pair<T, IT, WALLS>(v, x, y, z, &corners[0][t], 128);
  } else {
    cell_update_pair<T, IT, WALLS>(v, x, y, z, nullptr, 0);
  }
}

bool fits_32bit_index(size_t N) { return 27ull * (unsigned long long)N < 0xFFFFFFFFull; }

template <typename T, typename IT, int MINB>
static void launch_step2_b(const BlockView& v, dim3 grid, dim3 block, cudaStream_t s) {
  if (v.walls) k_step2<T, IT, MINB, true><<<grid, block, 0, s>>>(v);
  else k_step2<T, IT, MINB, false><<<grid, block, 0, s>>>(v);
}

template <typename T, typename IT>
static void launch_step2_t(const BlockView& v, dim3 grid, dim3 block, int b, cudaStream_t s) {
  if (b >= 6) launch_step2_b<T, IT, 6>(v, grid, block, s);
  else if (b == 5) launch_step2_b<T, IT, 5>(v, grid, block, s);
  else launch_step2_b<T, IT, 4>(v, grid, block, s);
}

static bool aligned_to(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// The two-node kernel reads and writes aligned pairs of every array: it needs an even nx
// (then every row, plane and level starts on an even node) and pair-aligned base pointers.
bool step_pair_ok(const BlockView& v, int storage, int bx, int by) {
  const size_t pe = storage == ST_FP16 ? 4 : 8;
  return (v.nx % 2) == 0 && bx % 2 == 0 && (bx / 2) * by <= 128 && aligned_to(v.d_in, pe) &&
         aligned_to(v.d_out, pe) && aligned_to(v.u_in, 8) && aligned_to(v.u_out, 8) &&
         aligned_to(v.c_in, 8) && aligned_to(v.c_out, 8) && aligned_to(v.flags, 2);
}

// grid.z = planes; the tile bx x by of nodes becomes bx / 2 x by threads.
static void launch_step2(const BlockView& v, int storage, int bx, int by, int b, unsigned planes,
                         cudaStream_t s) {
  const int tx = bx / 2;
  dim3 block(tx, by, 1);
  dim3 grid((v.nx / 2 + tx - 1) / tx, (v.ny + by - 1) / by, planes);
  const bool i32 = fits_32bit_index(v.N);
  if (storage == ST_FP16) {
    if (i32) launch_step2_t<__half, uint32_t>(v, grid, block, b, s);
    else launch_step2_t<__half, uint64_t>(v, grid, block, b, s);
  } else {
    if (i32) launch_step2_t<float, uint32_t>(v, grid, block, b, s);
    else launch_step2_t<float, uint64_t>(v, grid, block, b, s);
  }
}

template <typename T, typename IT, bool ALIGN>
static void launch_step_t(const BlockView& v, dim3 grid, dim3 block, int minb, cudaStream_t s) {
  minb = step_scalar_bound(minb);
  if (v.walls) {
    if (minb >= 4) k_step<T, IT, ALIGN, 4, true><<<grid, block, 0, s>>>(v);
    else k_step<T, IT, ALIGN, 3, true><<<grid, block, 0, s>>>(v);
  } else {
    if (minb >= 4) k_step<T, IT, ALIGN, 4, false><<<grid, block, 0, s>>>(v);
    else k_step<T, IT, ALIGN, 3, false><<<grid, block, 0, s>>>(v);
  }
}

cudaError_t launch_step(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                        int minb) {
  if (step_is_pair(minb) && step_pair_ok(v, storage, bx, by)) {
    launch_step2(v, storage, bx, by, minb - STEP_PAIR, (unsigned)v.nz, s);
    return cudaGetLastError();
  }
  dim3 block(bx, by, 1);
  dim3 grid((v.nx + bx - 1) / bx, (v.ny + by - 1) / by, v.nz);
  const bool i32 = fits_32bit_index(v.N);
  if (storage == ST_FP16) {
    if (i32) launch_step_t<__half, uint32_t, false>(v, grid, block, minb, s);
    else launch_step_t<__half, uint64_t, false>(v, grid, block, minb, s);
  } else {
    if (i32) launch_step_t<float, uint32_t, false>(v, grid, block, minb, s);
    else launch_step_t<float, uint64_t, false>(v, grid, block, minb, s);
  }
  return cudaGetLastError();
}

// The step of planes [z0, z0 + count) only (a slab's send planes before its other planes).
cudaError_t launch_step_planes(const BlockView& v, int storage, int bx, int by, cudaStream_t s,
                               int minb, int z0, int count) {
  if (count <= 0) return cudaSuccess;
  BlockView w = v;
  w.z_first = z0;
  if (step_is_pair(minb) && step_pair_ok(w, storage, bx, by)) {
    launch_step2(w, storage, bx, by, minb - STEP_PAIR, (unsigned)count, s);
    return cudaGetLastError();
  }
  dim3 block(bx, by, 1);
  dim3 grid((v.nx + bx - 1) / bx, (v.ny + by - 1) / by, count);
  const bool i32 = fits_32bit_index(v.N);
  if (storage == ST_FP16) {
    if (i32) launch_step_t<__half, uint32_t, false>(w, grid, block, minb, s);
    else launch_step_t<__half, uint64_t, false>(w, grid, block, minb, s);
  } else {
    if (i32) launch_step_t<float, uint32_t, false>(w, grid, block, minb, s);
    else launch_step_t<float, uint64_t, false>(w, grid, block, minb, s);
  }
  return cudaGetLastError();
}

// Last sub-step of a refined block with the temporal alignment fused in (FP32 storage,
// 32-bit indexing: refined blocks are limited to 27 N < 2^32).
cudaError_t launch_step_align(const BlockView& v, int bx, int by, cudaStream_t s, int minb) {
  dim3 block(bx, by, 1);
  dim3 grid((v.nx + bx - 1) / bx, (v.ny + by - 1) / by, v.nz);
  launch_step_t<float, uint32_t, true>(v, grid, block, minb, s);
  return cudaGetLastError();
}

// f_0 = f^eq(rho_0, u_0) (Algorithm 1 initialisation); obstacle voxels hold the rest state.
template <typename T>
__global__ void k_init(BlockView v, const float* rho, const float* u, const float* c) {
  const size_t N = v.N;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    T* dout = static_cast<T*>(v.d_out);
    const bool solid = v.flags[idx] & (F_SOLID | F_OBST_WALL);   // obstacle voxels start at rest
    const float r = (rho && !solid) ? rho[idx] : 1.0f;
    const float ux = solid ? 0.f : u[idx], uy = solid ? 0.f : u[N + idx],
                uz = solid ? 0.f : u[2 * N + idx];
    float d[27];
    equilibrium(d, r, ux, uy, uz);
#pragma unroll
    for (int k = 0; k < 27; ++k) store_pop(dout + (size_t)k * N + idx, d[k]);
    v.u_out[idx] = ux; v.u_out[N + idx] = uy; v.u_out[2 * N + idx] = uz;
    v.c_out[idx] = (solid || !c) ? 0.0f : c[idx];
  }
}

cudaError_t launch_init(const BlockView& v, int storage, const float* rho, const float* u,
                        const float* c, cudaStream_t s) {
  const int threads = 256;
  const size_t want = (v.N + threads - 1) / threads;
  const int grid = (int)(want < 65535 ? want : 65535);
  if (storage == ST_FP16) k_init<__half><<<grid, threads, 0, s>>>(v, rho, u, c);
  else k_init<float><<<grid, threads, 0, s>>>(v, rho, u, c);
  return cudaGetLastError();
}

// User bits (obstacle, inflow, scalar source) replace the node's; library bits are kept.
__global__ void k_merge_user_flags(uint8_t* flags, const uint8_t* user, size_t N) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const uint8_t keep = flags[i] & (F_GHOST | F_WALL);
    flags[i] = keep | (user[i] & (F_SOLID | F_INFLOW | F_SCALAR_SRC));
  }
}

// F_WALL on the nodes of the wall faces (bits x-, x+, y-, y+, z-, z+), off elsewhere.
__global__ void k_mark_walls(uint8_t* flags, int nx, int ny, int nz, int walls) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((size_t)nx * ny));
    const bool w = ((walls & 1) && x == 0) || ((walls & 2) && x == nx - 1) ||
                   ((walls & 4) && y == 0) || ((walls & 8) && y == ny - 1) ||
                   ((walls & 16) && z == 0) || ((walls & 32) && z == nz - 1);
    flags[i] = w ? (uint8_t)(flags[i] | F_WALL) : (uint8_t)(flags[i] & ~F_WALL);
  }
}

cudaError_t launch_mark_walls(uint8_t* flags, int nx, int ny, int nz, int walls, cudaStream_t s) {
  const size_t g = ((size_t)nx * ny * nz + 255) / 256;
  k_mark_walls<<<(int)(g < 8192 ? g : 8192), 256, 0, s>>>(flags, nx, ny, nz, walls);
  return cudaGetLastError();
}

// Obstacle surfaces as walls: an obstacle voxel (F_SOLID or F_OBST_WALL) with a non-obstacle
// pull source is a surface voxel; with `on` it becomes an active wall node (F_OBST_WALL, not
// F_SOLID), otherwise every obstacle voxel is F_SOLID again.  The obstacle predicate is the
// same before and after, so the update runs in place.
__global__ void k_obstacle_walls(uint8_t* flags, int nx, int ny, int nz, int px, int py, int pz,
                                 int on) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const uint8_t f = flags[idx];
    if (!(f & (F_SOLID | F_OBST_WALL))) continue;
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((size_t)nx * ny));
    bool surface = false;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int sx = nbr(x, dx, nx, px), sy = nbr(y, dy, ny, py), sz = nbr(z, dz, nz, pz);
          surface |= !(flags[((size_t)sz * ny + sy) * nx + sx] & (F_SOLID | F_OBST_WALL));
        }
    const uint8_t base = f & (uint8_t)~(F_SOLID | F_OBST_WALL);
    flags[idx] = (on && surface) ? (uint8_t)(base | F_OBST_WALL) : (uint8_t)(base | F_SOLID);
  }
}

cudaError_t launch_obstacle_walls(uint8_t* flags, int nx, int ny, int nz, const int per[3], int on,
                                  cudaStream_t s) {
  const size_t N = (size_t)nx * ny * nz;
  const int grid = (int)((N + 255) / 256 < 65535 ? (N + 255) / 256 : 65535);
  k_obstacle_walls<<<grid, 256, 0, s>>>(flags, nx, ny, nz, per[0], per[1], per[2], on);
  return cudaGetLastError();
}

cudaError_t launch_merge_user_flags(uint8_t* flags, const uint8_t* user, size_t N,
                                    cudaStream_t s) {
  const size_t g = (N + 255) / 256;
  k_merge_user_flags<<<(int)(g < 8192 ? g : 8192), 256, 0, s>>>(flags, user, N);
  return cudaGetLastError();
}

// Derived flag: F_NEAR_SOLID when any pull source of a non-solid node is an obstacle voxel.
__global__ void k_near_solid(uint8_t* flags, int nx, int ny, int nz, int px, int py, int pz) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((size_t)nx * ny));
    bool near = false;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          const int sx = nbr(x, dx, nx, px), sy = nbr(y, dy, ny, py), sz = nbr(z, dz, nz, pz);
          near |= (flags[((size_t)sz * ny + sy) * nx + sx] & F_SOLID) != 0;
        }
    uint8_t f = flags[idx];
    f = near ? (f | F_NEAR_SOLID) : (f & ~F_NEAR_SOLID);
    flags[idx] = f;
  }
}

cudaError_t launch_near_solid(uint8_t* flags, int nx, int ny, int nz, const int per[3],
                              cudaStream_t s) {
  const size_t N = (size_t)nx * ny * nz;
  const int grid = (int)((N + 255) / 256 < 65535 ? (N + 255) / 256 : 65535);
  k_near_solid<<<grid, 256, 0, s>>>(flags, nx, ny, nz, per[0], per[1], per[2]);
  return cudaGetLastError();
}

struct InflowRec {
  int x, y, z;
  float ux, uy, uz;
};

__global__ void k_inflow_records(const InflowRec* rec, int n, uint8_t* flags, float* u0, float* u1,
                                 float* u2, int nx, int ny, int nz, size_t N, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const InflowRec r = rec[i];
  if (r.x < 0 || r.y < 0 || r.z < 0 || r.x >= nx || r.y >= ny || r.z >= nz) {
    atomicOr(err, 4);  // bad record: ignored, reported
    return;
  }
  const size_t idx = ((size_t)r.z * ny + r.y) * nx + r.x;
  if (flags[idx] & (F_SOLID | F_OBST_WALL | F_GHOST)) {
    atomicOr(err, 4);  // obstacle voxels and ghost nodes cannot become inflow nodes
    return;
  }
  flags[idx] |= F_INFLOW;
  float* lv[3] = {u0, u1, u2};
  for (int l = 0; l < 3; ++l)
    if (lv[l]) { lv[l][idx] = r.ux; lv[l][N + idx] = r.uy; lv[l][2 * N + idx] = r.uz; }
}

// Records of several domains in one launch (lbm_set_inflow_batch): record i belongs to
// member member_of[i]; the same checks and writes as k_inflow_records.
__global__ void k_inflow_records_multi(const InflowRec* rec, int n, const int* member_of,
                                       const InflowMember* members) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const InflowMember m = members[member_of[i]];
  const InflowRec r = rec[i];
  if (r.x < 0 || r.y < 0 || r.z < 0 || r.x >= m.nx || r.y >= m.ny || r.z >= m.nz) {
    atomicOr(m.err, 4);
    return;
  }
  const size_t idx = ((size_t)r.z * m.ny + r.y) * m.nx + r.x;
  if (m.flags[idx] & (F_SOLID | F_OBST_WALL | F_GHOST)) {
    atomicOr(m.err, 4);
    return;
  }
  m.flags[idx] |= F_INFLOW;
  for (int l = 0; l < 3; ++l)
    if (m.u[l]) { m.u[l][idx] = r.ux; m.u[l][m.N + idx] = r.uy; m.u[l][2 * m.N + idx] = r.uz; }
}

cudaError_t launch_inflow_records_multi(const void* rec, int n, const int* member_of,
                                        const InflowMember* members, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_inflow_records_multi<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const InflowRec*>(rec), n,
                                                        member_of, members);
  return cudaGetLastError();
}

cudaError_t launch_inflow_records(const void* rec, int n, uint8_t* flags, float* const* u_levels,
                                  int n_levels, int nx, int ny, int nz, size_t N, int* err,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  float* u0 = n_levels > 0 ? u_levels[0] : nullptr;
  float* u1 = n_levels > 1 ? u_levels[1] : nullptr;
  float* u2 = n_levels > 2 ? u_levels[2] : nullptr;
  k_inflow_records<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const InflowRec*>(rec), n, flags,
                                                  u0, u1, u2, nx, ny, nz, N, err);
  return cudaGetLastError();
}

// ---- field conversion ------------------------------------------------------------------

template <typename T, typename O>
__global__ void k_read_f(const T* d, size_t N, O* out) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int k = c_paper_to_cube[q];
      const double val = wkd(k) + (double)load_pop(d + (size_t)k * N + idx);
      out[(size_t)q * N + idx] = (O)val;
    }
  }
}

template <typename T, typename I>
__global__ void k_write_f(T* d, size_t N, const I* in) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int k = c_paper_to_cube[q];
      const double dev = (double)in[(size_t)q * N + idx] - wkd(k);
      if constexpr (sizeof(T) == 2) d[(size_t)k * N + idx] = __double2half(dev);
      else d[(size_t)k * N + idx] = (float)dev;
    }
  }
}

static int grid_for(size_t n) {
  const size_t g = (n + 255) / 256;
  return (int)(g < 8192 ? (g ? g : 1) : 8192);
}

cudaError_t launch_read_f(const void* d, int storage, size_t N, void* out, int out_f64,
                          cudaStream_t s) {
  const int g = grid_for(N);
  if (storage == ST_FP16) {
    if (out_f64) k_read_f<__half, double><<<g, 256, 0, s>>>((const __half*)d, N, (double*)out);
    else k_read_f<__half, float><<<g, 256, 0, s>>>((const __half*)d, N, (float*)out);
  } else {
    if (out_f64) k_read_f<float, double><<<g, 256, 0, s>>>((const float*)d, N, (double*)out);
    else k_read_f<float, float><<<g, 256, 0, s>>>((const float*)d, N, (float*)out);
  }
  return cudaGetLastError();
}

cudaError_t launch_write_f(void* d, int storage, size_t N, const void* in, int in_f64,
                           cudaStream_t s) {
  const int g = grid_for(N);
  if (storage == ST_FP16) {
    if (in_f64) k_write_f<__half, double><<<g, 256, 0, s>>>((__half*)d, N, (const double*)in);
    else k_write_f<__half, float><<<g, 256, 0, s>>>((__half*)d, N, (const float*)in);
  } else {
    if (in_f64) k_write_f<float, double><<<g, 256, 0, s>>>((float*)d, N, (const double*)in);
    else k_write_f<float, float><<<g, 256, 0, s>>>((float*)d, N, (const float*)in);
  }
  return cudaGetLastError();
}

template <typename T>
__global__ void k_read_rho(const T* d, size_t N, float* out) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 27; ++k) s += load_pop(d + (size_t)k * N + idx);
    out[idx] = 1.0f + s;
  }
}

cudaError_t launch_read_rho(const void* d, int storage, size_t N, float* out, cudaStream_t s) {
  const int g = grid_for(N);
  if (storage == ST_FP16) k_read_rho<__half><<<g, 256, 0, s>>>((const __half*)d, N, out);
  else k_read_rho<float><<<g, 256, 0, s>>>((const float*)d, N, out);
  return cudaGetLastError();
}

template <typename I, typename O>
__global__ void k_convert(const I* in, O* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (O)in[i];
}

cudaError_t launch_convert(const void* in, int in_f64, void* out, int out_f64, size_t n,
                           cudaStream_t s) {
  const int g = grid_for(n);
  if (in_f64 && out_f64) k_convert<double, double><<<g, 256, 0, s>>>((const double*)in, (double*)out, n);
  else if (in_f64) k_convert<double, float><<<g, 256, 0, s>>>((const double*)in, (float*)out, n);
  else if (out_f64) k_convert<float, double><<<g, 256, 0, s>>>((const float*)in, (double*)out, n);
  else k_convert<float, float><<<g, 256, 0, s>>>((const float*)in, (float*)out, n);
  return cudaGetLastError();
}

}  // namespace lbm
