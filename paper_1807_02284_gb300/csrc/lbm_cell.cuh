// Per-node collide-and-stream update shared by the single-block, batched and adjoint-recompute
// kernels, so that every launch shape computes bit-identical results.
//
// IT is the index type: 32-bit when every array of the block has fewer than 2^32 elements
// (27 N < 2^32), which halves the address arithmetic, 64-bit otherwise.
#pragma once
#include "lbm_internal.h"

namespace lbm {

template <typename IT>
struct Nbr {
  IT xm, x0, xp;            // x - 1, x, x + 1 (wrapped or clamped)
  IT rm, r0, rp;            // row offsets (y - 1, y, y + 1) * nx
  IT pm, p0, pp;            // plane offsets (z - 1, z, z + 1) * nx * ny
};

template <typename IT>
__device__ __forceinline__ Nbr<IT> neighbours(const BlockView& v, int x, int y, int z) {
  Nbr<IT> n;
  const IT nx = (IT)v.nx, nxy = (IT)v.nx * (IT)v.ny;
  n.xm = (IT)nbr(x, -1, v.nx, v.per[0]);
  n.x0 = (IT)x;
  n.xp = (IT)nbr(x, 1, v.nx, v.per[0]);
  n.rm = nx * (IT)nbr(y, -1, v.ny, v.per[1]);
  n.r0 = nx * (IT)y;
  n.rp = nx * (IT)nbr(y, 1, v.ny, v.per[1]);
  n.pm = nxy * (IT)nbr(z, -1, v.nz, v.per[2]);
  n.p0 = nxy * (IT)z;
  n.pp = nxy * (IT)nbr(z, 1, v.nz, v.per[2]);
  return n;
}

// A node whose y and z neighbours need no wrap or clamp (1 <= y <= ny - 2, 1 <= z <= nz - 2):
// its rows and planes are plain offsets, the same for a whole warp of an x-row, so every
// pull source is a warp-uniform offset plus the lane's x source.  The x neighbours keep the
// face rules (wrap or clamp).  Same indices, loads and values as the general path.
__device__ __forceinline__ bool inner_yz(const BlockView& v, int y, int z) {
  return (unsigned)(y - 1) < (unsigned)(v.ny - 2) && (unsigned)(z - 1) < (unsigned)(v.nz - 2);
}

template <typename IT>
__device__ __forceinline__ Nbr<IT> neighbours_inner(const BlockView& v, int x, int y, int z) {
  Nbr<IT> n;
  const IT nx = (IT)v.nx, nxy = (IT)v.nx * (IT)v.ny;
  n.xm = (IT)nbr(x, -1, v.nx, v.per[0]);
  n.x0 = (IT)x;
  n.xp = (IT)nbr(x, 1, v.nx, v.per[0]);
  n.r0 = nx * (IT)y;
  n.rm = n.r0 - nx;
  n.rp = n.r0 + nx;
  n.p0 = nxy * (IT)z;
  n.pm = n.p0 - nxy;
  n.pp = n.p0 + nxy;
  return n;
}

// Pull of an inner_yz node: plane K at rows y - c_y, z - c_z is the offset
// K N - c_z nx ny - c_y nx from the lane's row (uniform over the warp); am, a0, ap are the
// lane's row index plus its x source for c_x = +1, 0, -1.
template <typename T, typename IT, int K = 0>
__device__ __forceinline__ void pull_inner(float (&d)[27], const T* __restrict__ din, IT N,
                                           IT nx, IT nxy, IT am, IT a0, IT ap) {
  if constexpr (K < 27) {
    constexpr int cx = cxk(K), cy = cyk(K), cz = czk(K);
    const IT off = (IT)K * N - (IT)cz * nxy - (IT)cy * nx;
    const IT a = cx > 0 ? am : cx < 0 ? ap : a0;
    d[K] = load_pop(din + (off + a));
    pull_inner<T, IT, K + 1>(d, din, N, nx, nxy, am, a0, ap);
  }
}

// Source node of the pull for velocity slot k: x - c_k.
template <int K, typename IT>
__device__ __forceinline__ IT pull_src(const Nbr<IT>& n) {
  constexpr int cx = cxk(K), cy = cyk(K), cz = czk(K);
  const IT sx = cx > 0 ? n.xm : cx < 0 ? n.xp : n.x0;
  const IT sy = cy > 0 ? n.rm : cy < 0 ? n.rp : n.r0;
  const IT sz = cz > 0 ? n.pm : cz < 0 ? n.pp : n.p0;
  return sz + sy + sx;
}

template <typename T, typename IT, int K = 0>
__device__ __forceinline__ void pull_all(float (&d)[27], const T* __restrict__ din, IT N,
                                         const Nbr<IT>& n) {
  if constexpr (K < 27) {
    d[K] = load_pop(din + ((IT)K * N + pull_src<K>(n)));
    pull_all<T, IT, K + 1>(d, din, N, n);
  }
}

// Halfway bounce-back: a population whose source node is an obstacle voxel is replaced by
// the opposite population of this node (wall at rest).
template <typename T, typename IT, int K = 0>
__device__ __forceinline__ void bounce_back(float (&d)[27], const T* __restrict__ din, IT N,
                                            const uint8_t* __restrict__ flags,
                                            const Nbr<IT>& n, IT idx) {
  if constexpr (K < 27) {
    if constexpr (K != 13) {
      if (__ldg(flags + pull_src<K>(n)) & F_SOLID)
        d[K] = load_pop(din + ((IT)(26 - K) * N + idx));
    }
    bounce_back<T, IT, K + 1>(d, din, N, flags, n, idx);
  }
}

// grad_norm of an inner_yz node (same loads and arithmetic order as grad_norm).
template <typename IT>
__device__ __forceinline__ float grad_norm_inner(const float* __restrict__ U, IT N, IT nx, IT nxy,
                                                 IT idx, IT im, IT ip) {
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* Ua = U + (IT)a * N;
    const float dx = __ldg(Ua + ip) - __ldg(Ua + im);
    const float dy = __ldg(Ua + (idx + nx)) - __ldg(Ua + (idx - nx));
    const float dz = __ldg(Ua + (idx + nxy)) - __ldg(Ua + (idx - nxy));
    s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, s)));
  }
  return 0.5f * sqrtf(s);
}

template <typename IT>
__device__ __forceinline__ float grad_norm(const float* __restrict__ U, IT N, const Nbr<IT>& n) {
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* Ua = U + (IT)a * N;
    const float dx = __ldg(Ua + (n.p0 + n.r0 + n.xp)) - __ldg(Ua + (n.p0 + n.r0 + n.xm));
    const float dy = __ldg(Ua + (n.p0 + n.rp + n.x0)) - __ldg(Ua + (n.p0 + n.rm + n.x0));
    const float dz = __ldg(Ua + (n.pp + n.r0 + n.x0)) - __ldg(Ua + (n.pm + n.r0 + n.x0));
    s = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, s)));
  }
  return 0.5f * sqrtf(s);
}

// The eight corner values of the departure cell and the interpolation weights.
struct ScalarCell {
  float c[8];
  float tx, ty, tz;
};

template <typename IT>
__device__ __forceinline__ ScalarCell scalar_corners(const BlockView& v, int x, int y, int z,
                                                     float ux, float uy, float uz) {
  const Axis1 ax = sl_axis(x, ux, v.nx, v.per[0]);
  const Axis1 ay = sl_axis(y, uy, v.ny, v.per[1]);
  const Axis1 az = sl_axis(z, uz, v.nz, v.per[2]);
  const IT nx = (IT)v.nx, nxy = (IT)v.nx * (IT)v.ny;
  const float* __restrict__ c = v.c_in;
  const IT z0 = nxy * (IT)az.i0, z1 = nxy * (IT)az.i1, y0 = nx * (IT)ay.i0, y1 = nx * (IT)ay.i1;
  const IT x0 = (IT)ax.i0, x1 = (IT)ax.i1;
  ScalarCell s;
  s.c[0] = __ldg(c + (z0 + y0 + x0)); s.c[1] = __ldg(c + (z0 + y0 + x1));
  s.c[2] = __ldg(c + (z0 + y1 + x0)); s.c[3] = __ldg(c + (z0 + y1 + x1));
  s.c[4] = __ldg(c + (z1 + y0 + x0)); s.c[5] = __ldg(c + (z1 + y0 + x1));
  s.c[6] = __ldg(c + (z1 + y1 + x0)); s.c[7] = __ldg(c + (z1 + y1 + x1));
  s.tx = ax.t; s.ty = ay.t; s.tz = az.t;
  return s;
}

__device__ __forceinline__ float scalar_value(const ScalarCell& s) {
  const float a00 = fmaf(s.tx, s.c[1] - s.c[0], s.c[0]);
  const float a01 = fmaf(s.tx, s.c[3] - s.c[2], s.c[2]);
  const float a10 = fmaf(s.tx, s.c[5] - s.c[4], s.c[4]);
  const float a11 = fmaf(s.tx, s.c[7] - s.c[6], s.c[6]);
  const float b0 = fmaf(s.ty, a01 - a00, a00);
  const float b1 = fmaf(s.ty, a11 - a10, a10);
  return fmaf(s.tz, b1 - b0, b0);
}

// Non-positive or non-finite density, or a velocity far outside the lattice's range.
__device__ __forceinline__ bool unphysical(float drho, float ux, float uy, float uz) {
  return !(1.0f + drho > 0.0f) || !(fabsf(ux) + fabsf(uy) + fabsf(uz) < 3.0f);
}

__device__ __forceinline__ void flag_error(int* err, bool bad) {
  const unsigned m = __ballot_sync(__activemask(), bad);
  if (m && (threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicOr(err, 1);
}

// Bits k of the populations of a node whose pull source is an inner obstacle voxel.
template <typename IT, int K = 0>
__device__ __forceinline__ unsigned solid_sources(const uint8_t* __restrict__ flags,
                                                  const Nbr<IT>& n) {
  if constexpr (K < 27) {
    unsigned b = 0u;
    if constexpr (K != 13) b = (__ldg(flags + pull_src<K>(n)) & F_SOLID) ? (1u << K) : 0u;
    return b | solid_sources<IT, K + 1>(flags, n);
  } else {
    return 0u;
  }
}

// No-slip wall node (the second-order wall of Sec. 6.1, read as the regularized on-node
// wall) on a flat face of the block or, with obstacle walls, on an obstacle's surface voxel:
// populations pulled from beyond the wall (through a wall face, or from an inner obstacle
// voxel) are completed by bounce-back from their opposite (wall at rest); where both of a
// pair come from beyond the wall (edges, corners) they take the rest equilibrium; rho is the
// mass of the completed set and every population is rebuilt as
// w_i rho + (w_i / (2 c_s^4)) Q_i : Pi from the non-equilibrium stress Pi of the completed
// set.  On shifted populations d = f - w.
template <typename IT>
__device__ __forceinline__ void wall_regularize(float (&d)[27], const BlockView& v, int x, int y,
                                                int z, uint8_t fl, const Nbr<IT>& n) {
  const bool lo[3] = {(v.walls & 1) && x == 0, (v.walls & 4) && y == 0, (v.walls & 16) && z == 0};
  const bool hi[3] = {(v.walls & 2) && x == v.nx - 1, (v.walls & 8) && y == v.ny - 1,
                      (v.walls & 32) && z == v.nz - 1};
  unsigned unk = 0u;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int c[3] = {cxk(k), cyk(k), czk(k)};
    bool u = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) u |= (lo[a] && c[a] == 1) || (hi[a] && c[a] == -1);
    if (u) unk |= 1u << k;
  }
  if (fl & F_OBST_WALL) unk |= solid_sources<IT>(v.flags, n);
  float s = 0.0f, wb = 0.0f;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const bool uk = (unk >> k) & 1u, uo = (unk >> (26 - k)) & 1u;
    if (uk && uo) {
      wb += wk(k);
    } else {
      if (uk) d[k] = d[26 - k];          // the opposite's source is inside: it is known
      s += d[k];
    }
  }
  const float drho = s / (1.0f - wb);
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const bool both = ((unk >> k) & 1u) && ((unk >> (26 - k)) & 1u);
    const float neq = both ? 0.0f : d[k] - wk(k) * drho;
    const float cx = (float)cxk(k), cy = (float)cyk(k), cz = (float)czk(k);
    pxx = fmaf(cx * cx, neq, pxx); pyy = fmaf(cy * cy, neq, pyy); pzz = fmaf(cz * cz, neq, pzz);
    pxy = fmaf(cx * cy, neq, pxy); pxz = fmaf(cx * cz, neq, pxz); pyz = fmaf(cy * cz, neq, pyz);
  }
  const float tr = (pxx + pyy + pzz) * (1.0f / 3.0f);
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const float cx = (float)cxk(k), cy = (float)cyk(k), cz = (float)czk(k);
    const float qp = cx * cx * pxx + cy * cy * pyy + cz * cz * pzz +
                     2.0f * (cx * cy * pxy + cx * cz * pxz + cy * cz * pyz) - tr;
    d[k] = wk(k) * fmaf(4.5f, qp, drho);
  }
}

// Where a node writes the moments of the state it stores, for the diagnostics fused into
// the step (the quantities lbm_reduce sums: node count, rho - 1, j, |j|^2 / (2 rho)): six
// floats at nm[0], nm[stride], ..., nm[5 stride] (shared memory, one column per thread).
struct NodeMomentsOut {
  float* nm;
  int stride;
  __device__ __forceinline__ void put(float drho, float jx, float jy, float jz, float inv_rho) const {
    nm[0] = 1.0f;
    nm[stride] = drho;
    nm[2 * stride] = jx;
    nm[3 * stride] = jy;
    nm[4 * stride] = jz;
    const float jj = __fmaf_rn(jz, jz, __fmaf_rn(jy, jy, __fmul_rn(jx, jx)));
    nm[5 * stride] = __fmul_rn(__fmul_rn(0.5f, jj), inv_rho);   // explicit: one value per node
  }
};

// One node of one block: pull (with bounce-back and face handling), macroscopic moments,
// adaptive rates from the lagged velocity, CMR collision, store of f~, u and the scalar.
// Scale-boundary (ghost) nodes of refined blocks are not written: their next values come
// from the coarse-to-fine mapping, which can therefore run concurrently with this update.
// ALIGN: last sub-step of a refined block, storing the temporal alignment (see BlockView).
// WALLS: the block has no-slip wall faces (an instance without them carries no wall code).
// RED: also write the moments of the stored state through *nm (the caller zeroes them first:
// obstacle voxels and ghost nodes write nothing).  Collision conserves rho and j, so a fluid
// node's are those of its pulled set, written as soon as they are known, so that nothing
// is held through the collision.
template <typename T, typename IT, bool ALIGN = false, bool WALLS = false, bool RED = false>
__device__ __forceinline__ void cell_update(const BlockView& v, int x, int y, int z,
                                            const NodeMomentsOut* nm = nullptr) {
  const IT N = (IT)v.N;
  const T* __restrict__ din = static_cast<const T*>(v.d_in);
  T* __restrict__ dout = static_cast<T*>(v.d_out);
  const bool inner = inner_yz(v, y, z);
  const Nbr<IT> n = inner ? neighbours_inner<IT>(v, x, y, z) : neighbours<IT>(v, x, y, z);
  const IT idx = n.p0 + n.r0 + n.x0;
  const uint8_t fl = __ldg(v.flags + idx);
  float d[27];

  if (fl & (F_SOLID | F_INFLOW | F_GHOST)) {
    float ux = 0.f, uy = 0.f, uz = 0.f, cval = 0.f;
    if (fl & F_SOLID) {
#pragma unroll
      for (int k = 0; k < 27; ++k) d[k] = 0.0f;
    } else if (fl & F_GHOST) {
      return;
    } else {  // Dirichlet inflow: equilibrium at rho = 1 and the stored inflow velocity
      ux = v.u_in[idx]; uy = v.u_in[N + idx]; uz = v.u_in[2 * N + idx];
      equilibrium(d, 1.0f, ux, uy, uz);
      if constexpr (RED) nm->put(0.0f, ux, uy, uz, 1.0f);
      cval = (fl & F_SCALAR_SRC) ? v.c_src
                                 : scalar_value(scalar_corners<IT>(v, x, y, z, ux, uy, uz));
    }
#pragma unroll
    for (int k = 0; k < 27; ++k) store_pop(dout + ((IT)k * N + idx), d[k]);
    v.u_out[idx] = ux; v.u_out[N + idx] = uy; v.u_out[2 * N + idx] = uz;
    v.c_out[idx] = cval;
    return;
  }

  // all independent loads first: the pull and the lagged velocity neighbourhood
  const IT nxI = (IT)v.nx, nxyI = (IT)v.nx * (IT)v.ny;
  const IT row = n.p0 + n.r0;
  if (inner) pull_inner<T, IT>(d, din, N, nxI, nxyI, row + n.xm, idx, row + n.xp);
  else pull_all<T, IT>(d, din, N, n);
  // an obstacle wall node completes what comes from inside the obstacle itself
  if ((fl & F_NEAR_SOLID) && !(WALLS && (fl & F_OBST_WALL)))
    bounce_back<T, IT>(d, din, N, v.flags, n, idx);
  if constexpr (WALLS) {
    if (fl & (F_WALL | F_OBST_WALL)) wall_regularize<IT>(d, v, x, y, z, fl, n);
  }
  float g_lag = 0.0f;
  if (v.rp.adaptive && !v.rp.local)
    g_lag = inner ? grad_norm_inner<IT>(v.u_in, N, nxI, nxyI, idx, row + n.xm, row + n.xp)
                  : grad_norm<IT>(v.u_in, N, n);

  raw_moments(d);
  const float drho = d[kap(0, 0, 0)];
  const float inv = fast_rcp(__fadd_rn(1.0f, drho));
  const float ux = __fmul_rn(d[kap(1, 0, 0)], inv), uy = __fmul_rn(d[kap(0, 1, 0)], inv),
              uz = __fmul_rn(d[kap(0, 0, 1)], inv);
  flag_error(v.err, unphysical(drho, ux, uy, uz));
  if constexpr (RED) {
    static_assert(!ALIGN, "the fused diagnostics cover plain steps");
    nm->put(drho, d[kap(1, 0, 0)], d[kap(0, 1, 0)], d[kap(0, 0, 1)], inv);
  }

  // departure-cell scalar loads go out before the collision arithmetic
  ScalarCell sc;
  const bool src = (fl & F_SCALAR_SRC) != 0;
  if (!src) sc = scalar_corners<IT>(v, x, y, z, ux, uy, uz);

  central_from_raw(d, ux, uy, uz);
  const float g = (v.rp.adaptive && v.rp.local) ? local_strain(d, drho, ux, uy, uz, v.rp.s_nu)
                                                : g_lag;
  const Keep kf = keep_factors(v.rp, g);
  collide_from_central(d, drho, ux, uy, uz, kf);

  if constexpr (ALIGN) {
    // three-point Lagrange interpolation to t_n + dt_0 of this node's states at t_n, at
    // t_n + (l-1)h (the sub-step's input) and at t_n + l h (just computed)
    // (a far-field block's linear alignment has al0 = 0: its t_n level is not read)
    const T* __restrict__ f0 = static_cast<const T*>(v.f_al0);
    const bool use0 = v.al0 != 0.0f;
    float s = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      const IT i = (IT)k * N + idx;
      const float rest = fmaf(v.al1, load_pop(din + i), v.al2 * d[k]);
      const float val = use0 ? fmaf(v.al0, load_pop(f0 + i), rest) : rest;
      d[k] = val;
      s += val;
      if (cxk(k) > 0) jx += val; else if (cxk(k) < 0) jx -= val;
      if (cyk(k) > 0) jy += val; else if (cyk(k) < 0) jy -= val;
      if (czk(k) > 0) jz += val; else if (czk(k) < 0) jz -= val;
    }
    const float ia = 1.0f / (1.0f + s);
    const float cnew = src ? v.c_src : scalar_value(sc);
    const float crest = fmaf(v.al1, v.c_in[idx], v.al2 * cnew);
    const float cal = use0 ? fmaf(v.al0, v.c_al0[idx], crest) : crest;
#pragma unroll
    for (int k = 0; k < 27; ++k) store_pop(dout + ((IT)k * N + idx), d[k]);
    __stcs(v.u_out + idx, jx * ia);
    __stcs(v.u_out + (N + idx), jy * ia);
    __stcs(v.u_out + (2 * N + idx), jz * ia);
    __stcs(v.c_out + idx, cal);
  } else {
#pragma unroll
    for (int k = 0; k < 27; ++k) store_pop(dout + ((IT)k * N + idx), d[k]);
    __stcs(v.u_out + idx, ux);
    __stcs(v.u_out + (N + idx), uy);
    __stcs(v.u_out + (2 * N + idx), uz);
    __stcs(v.c_out + idx, src ? v.c_src : scalar_value(sc));
  }
}


// ---- two nodes per thread (k_step2): nodes x and x + 1 of one row, x even, nx even, so that
// their stored values are aligned pairs.  The pair path covers inner_yz fluid nodes without
// bounce-back, walls or inflow (almost all nodes of a block); any other pair takes
// cell_update node by node.  Every value equals cell_update's for the same node: the loads,
// the lane arithmetic (float2 forms of the same rounded operations) and the stores are the
// per-node ones, only issued two at a time.

// Pull of the pair: c_x = 0 planes are one aligned pair load; c_x = +1 reads (x - 1, x),
// c_x = -1 reads (x + 1, x + 2), as two single loads (am0: node x's source x - 1, ap1: node
// x + 1's source x + 2, both with the face rules; a0: the pair's own index).
template <typename T, typename IT, int K = 0>
__device__ __forceinline__ void pull_pair(float2 (&d)[27], const T* __restrict__ din, IT N, IT nx,
                                          IT nxy, IT am0, IT a0, IT ap1) {
  if constexpr (K < 27) {
    constexpr int cx = cxk(K), cy = cyk(K), cz = czk(K);
    const IT off = (IT)K * N - (IT)cz * nxy - (IT)cy * nx;
    if constexpr (cx == 0) {
      d[K] = load_pop2(din + (off + a0));
    } else if constexpr (cx > 0) {
      d[K] = make_float2(load_pop(din + (off + am0)), load_pop(din + (off + a0)));
    } else {
      d[K] = make_float2(load_pop(din + (off + a0 + 1)), load_pop(din + (off + ap1)));
    }
    pull_pair<T, IT, K + 1>(d, din, N, nx, nxy, am0, a0, ap1);
  }
}

// grad_norm_inner of both nodes (the y and z differences as aligned pair loads).
template <typename IT>
__device__ __forceinline__ float2 grad_norm_pair(const float* __restrict__ U, IT N, IT nx, IT nxy,
                                                 IT a0, IT am0, IT ap1) {
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* Ua = U + (IT)a * N;
    const float2 c = __ldg(reinterpret_cast<const float2*>(Ua + a0));
    const float2 dx = vsub(make_float2(c.y, __ldg(Ua + ap1)), make_float2(__ldg(Ua + am0), c.x));
    const float2 dy = vsub(__ldg(reinterpret_cast<const float2*>(Ua + (a0 + nx))),
                           __ldg(reinterpret_cast<const float2*>(Ua + (a0 - nx))));
    const float2 dz = vsub(__ldg(reinterpret_cast<const float2*>(Ua + (a0 + nxy))),
                           __ldg(reinterpret_cast<const float2*>(Ua + (a0 - nxy))));
    s = vfma(dx, dx, vfma(dy, dy, vfma(dz, dz, s)));
  }
  return make_float2(0.5f * sqrtf(s.x), 0.5f * sqrtf(s.y));
}

// The departure cell's eight scalar corners of one node, copied asynchronously (cp.async,
// 4 bytes each, through L1) into this thread's shared-memory slots slot[i * stride]: the
// values are in flight through the collision without holding registers.
template <typename IT>
__device__ __forceinline__ void scalar_corners_async(const BlockView& v, int x, int y, int z,
                                                     float ux, float uy, float uz, float* slot,
                                                     int stride) {
  const Axis1 ax = sl_axis(x, ux, v.nx, v.per[0]);
  const Axis1 ay = sl_axis(y, uy, v.ny, v.per[1]);
  const Axis1 az = sl_axis(z, uz, v.nz, v.per[2]);
  const IT nx = (IT)v.nx, nxy = (IT)v.nx * (IT)v.ny;
  const IT z0 = nxy * (IT)az.i0, z1 = nxy * (IT)az.i1, y0 = nx * (IT)ay.i0, y1 = nx * (IT)ay.i1;
  const IT x0 = (IT)ax.i0, x1 = (IT)ax.i1;
  const IT src[8] = {z0 + y0 + x0, z0 + y0 + x1, z0 + y1 + x0, z0 + y1 + x1,
                     z1 + y0 + x0, z1 + y0 + x1, z1 + y1 + x0, z1 + y1 + x1};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(slot + i * stride);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(v.c_in + src[i])
                 : "memory");
  }
}

// scalar_value of the corners copied by scalar_corners_async (after cp.async.wait_group);
// the weights are recomputed from the same velocity.
__device__ __forceinline__ float scalar_value_slots(const BlockView& v, int x, int y, int z,
                                                    float ux, float uy, float uz,
                                                    const float* slot, int stride) {
  ScalarCell s;
#pragma unroll
  for (int i = 0; i < 8; ++i) s.c[i] = slot[i * stride];
  s.tx = sl_axis(x, ux, v.nx, v.per[0]).t;
  s.ty = sl_axis(y, uy, v.ny, v.per[1]).t;
  s.tz = sl_axis(z, uz, v.nz, v.per[2]).t;
  return scalar_value(s);
}

// FP16 storage takes the scalar corners through shared memory: its pair kernel is bound by
// the registers that hold loads in flight (occupancy), and without the corners' 22 live
// registers it runs at 5 CTAs per SM without spills (256^3 plume: 26.7 -> 27.4 GLUPS).  The
// FP32 pair kernel is bound by DRAM bandwidth and runs faster with the corners in registers
// (24.9 against 23.8 GLUPS).
template <typename T>
constexpr bool pair_corners_async() { return sizeof(T) == 2; }

// slot: this thread's 16 shared-memory floats (slot[i * stride], i < 16) for the corners
// when pair_corners_async<T>(), unused otherwise.  RED: the two nodes' moments go through
// nm0 and nm1 as cell_update's RED form writes them.
template <typename T, typename IT, bool WALLS, bool RED = false>
__device__ __forceinline__ void cell_update_pair(const BlockView& v, int x, int y, int z,
                                                 float* slot, int stride,
                                                 const NodeMomentsOut* nm0 = nullptr,
                                                 const NodeMomentsOut* nm1 = nullptr) {
  const IT N = (IT)v.N;
  const IT nxI = (IT)v.nx, nxyI = (IT)v.nx * (IT)v.ny;
  const IT row = nxyI * (IT)z + nxI * (IT)y;
  const IT a0 = row + (IT)x;
  const unsigned fl2 = __ldg(reinterpret_cast<const unsigned short*>(v.flags + a0));
  const uint8_t fl0 = (uint8_t)(fl2 & 0xffu), fl1 = (uint8_t)(fl2 >> 8);
  constexpr uint8_t kNodeWise = F_SOLID | F_INFLOW | F_GHOST | F_NEAR_SOLID | F_WALL | F_OBST_WALL;
  if (!inner_yz(v, y, z) || ((fl0 | fl1) & kNodeWise)) {
    cell_update<T, IT, false, WALLS, RED>(v, x, y, z, nm0);
    cell_update<T, IT, false, WALLS, RED>(v, x + 1, y, z, nm1);
    return;
  }
  const T* __restrict__ din = static_cast<const T*>(v.d_in);
  T* __restrict__ dout = static_cast<T*>(v.d_out);
  const IT am0 = row + (IT)nbr(x, -1, v.nx, v.per[0]);
  const IT ap1 = row + (IT)nbr(x + 1, 1, v.nx, v.per[0]);
  float2 d[27];
  pull_pair<T, IT>(d, din, N, nxI, nxyI, am0, a0, ap1);
  float2 g_lag = make_float2(0.0f, 0.0f);
  if (v.rp.adaptive && !v.rp.local) g_lag = grad_norm_pair<IT>(v.u_in, N, nxI, nxyI, a0, am0, ap1);

  raw_moments(d);
  const float2 drho = d[kap(0, 0, 0)];
  const float2 inv = make_float2(fast_rcp(__fadd_rn(1.0f, drho.x)), fast_rcp(__fadd_rn(1.0f, drho.y)));
  const float2 ux = vmul(d[kap(1, 0, 0)], inv), uy = vmul(d[kap(0, 1, 0)], inv),
               uz = vmul(d[kap(0, 0, 1)], inv);
  flag_error(v.err, unphysical(drho.x, ux.x, uy.x, uz.x) || unphysical(drho.y, ux.y, uy.y, uz.y));
  if constexpr (RED) {
    const float2 jx = d[kap(1, 0, 0)], jy = d[kap(0, 1, 0)], jz = d[kap(0, 0, 1)];
    nm0->put(drho.x, jx.x, jy.x, jz.x, inv.x);
    nm1->put(drho.y, jx.y, jy.y, jz.y, inv.y);
  }

  const bool src0 = (fl0 & F_SCALAR_SRC) != 0, src1 = (fl1 & F_SCALAR_SRC) != 0;
  constexpr bool kAsync = pair_corners_async<T>();
  ScalarCell sc0, sc1;
  if constexpr (kAsync) {
    if (!src0) scalar_corners_async<IT>(v, x, y, z, ux.x, uy.x, uz.x, slot, stride);
    if (!src1) scalar_corners_async<IT>(v, x + 1, y, z, ux.y, uy.y, uz.y, slot + 8 * stride, stride);
    asm volatile("cp.async.commit_group;" ::: "memory");
  } else {
    if (!src0) sc0 = scalar_corners<IT>(v, x, y, z, ux.x, uy.x, uz.x);
    if (!src1) sc1 = scalar_corners<IT>(v, x + 1, y, z, ux.y, uy.y, uz.y);
  }

  central_from_raw(d, ux, uy, uz);
  float2 g = g_lag;
  if (v.rp.adaptive && v.rp.local) {
    const float2 ss = local_strain_sq(d, drho, ux, uy, uz);
    g = make_float2(strain_from_sq(ss.x, drho.x, v.rp.s_nu), strain_from_sq(ss.y, drho.y, v.rp.s_nu));
  }
  const KeepT<float2> kf = pair_keep(keep_factors(v.rp, g.x), keep_factors(v.rp, g.y));
  collide_from_central(d, drho, ux, uy, uz, kf);

#pragma unroll
  for (int k = 0; k < 27; ++k) store_pop2(dout + ((IT)k * N + a0), d[k]);
  __stcs(reinterpret_cast<float2*>(v.u_out + a0), ux);
  __stcs(reinterpret_cast<float2*>(v.u_out + (N + a0)), uy);
  __stcs(reinterpret_cast<float2*>(v.u_out + (2 * N + a0)), uz);
  float c0 = v.c_src, c1 = v.c_src;
  if constexpr (kAsync) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!src0) c0 = scalar_value_slots(v, x, y, z, ux.x, uy.x, uz.x, slot, stride);
    if (!src1) c1 = scalar_value_slots(v, x + 1, y, z, ux.y, uy.y, uz.y, slot + 8 * stride, stride);
  } else {
    if (!src0) c0 = scalar_value(sc0);
    if (!src1) c1 = scalar_value(sc1);
  }
  __stcs(reinterpret_cast<float2*>(v.c_out + a0), make_float2(c0, c1));
}

}  // namespace lbm
