// Per-node collide-and-stream update shared by the single-block, batched and adjoint-recompute
// kernels, so that every launch shape computes bit-identical results.
#pragma once
#include "lbm_internal.h"

namespace lbm {

struct Nbr {
  int xm, xp;               // x - 1, x + 1 (wrapped or clamped)
  size_t rm, r0, rp;        // row offsets (y - 1, y, y + 1) * nx
  size_t pm, p0, pp;        // plane offsets (z - 1, z, z + 1) * nx * ny
};

__device__ __forceinline__ Nbr neighbours(const BlockView& v, int x, int y, int z) {
  Nbr n;
  const size_t nx = (size_t)v.nx, nxy = (size_t)v.nx * v.ny;
  n.xm = nbr(x, -1, v.nx, v.per[0]);
  n.xp = nbr(x, 1, v.nx, v.per[0]);
  n.rm = nx * nbr(y, -1, v.ny, v.per[1]);
  n.r0 = nx * y;
  n.rp = nx * nbr(y, 1, v.ny, v.per[1]);
  n.pm = nxy * nbr(z, -1, v.nz, v.per[2]);
  n.p0 = nxy * z;
  n.pp = nxy * nbr(z, 1, v.nz, v.per[2]);
  return n;
}

// Source node of the pull for velocity slot k: x - c_k.
template <int K>
__device__ __forceinline__ size_t pull_src(const Nbr& n, int x) {
  constexpr int cx = cxk(K), cy = cyk(K), cz = czk(K);
  const size_t sx = cx > 0 ? (size_t)n.xm : cx < 0 ? (size_t)n.xp : (size_t)x;
  const size_t sy = cy > 0 ? n.rm : cy < 0 ? n.rp : n.r0;
  const size_t sz = cz > 0 ? n.pm : cz < 0 ? n.pp : n.p0;
  return sz + sy + sx;
}

template <typename T, int K = 0>
__device__ __forceinline__ void pull_all(float (&d)[27], const T* din, size_t N, const Nbr& n,
                                         int x) {
  if constexpr (K < 27) {
    d[K] = load_pop(din + (size_t)K * N + pull_src<K>(n, x));
    pull_all<T, K + 1>(d, din, N, n, x);
  }
}

// Halfway bounce-back: a population whose source node is an obstacle voxel is replaced by
// the opposite population of this node (wall at rest).
template <typename T, int K = 0>
__device__ __forceinline__ void bounce_back(float (&d)[27], const T* din, size_t N,
                                            const uint8_t* flags, const Nbr& n, int x,
                                            size_t idx) {
  if constexpr (K < 27) {
    if constexpr (K != 13) {
      if (flags[pull_src<K>(n, x)] & F_SOLID) d[K] = load_pop(din + (size_t)(26 - K) * N + idx);
    }
    bounce_back<T, K + 1>(d, din, N, flags, n, x, idx);
  }
}

__device__ __forceinline__ float grad_norm(const float* U, size_t N, const Nbr& n, int x) {
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* Ua = U + (size_t)a * N;
    const float dx = __ldg(Ua + n.p0 + n.r0 + n.xp) - __ldg(Ua + n.p0 + n.r0 + n.xm);
    const float dy = __ldg(Ua + n.p0 + n.rp + x) - __ldg(Ua + n.p0 + n.rm + x);
    const float dz = __ldg(Ua + n.pp + n.r0 + x) - __ldg(Ua + n.pm + n.r0 + x);
    s += dx * dx + dy * dy + dz * dz;
  }
  return 0.5f * sqrtf(s);
}

__device__ __forceinline__ float sample_scalar(const BlockView& v, int x, int y, int z, float ux,
                                               float uy, float uz) {
  const Axis1 ax = sl_axis(x, ux, v.nx, v.per[0]);
  const Axis1 ay = sl_axis(y, uy, v.ny, v.per[1]);
  const Axis1 az = sl_axis(z, uz, v.nz, v.per[2]);
  const size_t nx = (size_t)v.nx, nxy = (size_t)v.nx * v.ny;
  const float* c = v.c_in;
  const size_t z0 = nxy * az.i0, z1 = nxy * az.i1, y0 = nx * ay.i0, y1 = nx * ay.i1;
  const float c000 = __ldg(c + z0 + y0 + ax.i0), c001 = __ldg(c + z0 + y0 + ax.i1);
  const float c010 = __ldg(c + z0 + y1 + ax.i0), c011 = __ldg(c + z0 + y1 + ax.i1);
  const float c100 = __ldg(c + z1 + y0 + ax.i0), c101 = __ldg(c + z1 + y0 + ax.i1);
  const float c110 = __ldg(c + z1 + y1 + ax.i0), c111 = __ldg(c + z1 + y1 + ax.i1);
  const float tx = ax.t, ty = ay.t, tz = az.t;
  const float a00 = c000 + tx * (c001 - c000), a01 = c010 + tx * (c011 - c010);
  const float a10 = c100 + tx * (c101 - c100), a11 = c110 + tx * (c111 - c110);
  const float b0 = a00 + ty * (a01 - a00), b1 = a10 + ty * (a11 - a10);
  return b0 + tz * (b1 - b0);
}

__device__ __forceinline__ void flag_error(int* err, bool bad) {
  const unsigned m = __ballot_sync(__activemask(), bad);
  if (m && (threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicOr(err, 1);
}

// One node of one block: pull (with bounce-back and face handling), macroscopic moments,
// adaptive rates from the lagged velocity, CMR collision, store of f~, u and the scalar.
template <typename T>
__device__ __forceinline__ void cell_update(const BlockView& v, int x, int y, int z) {
  const size_t N = v.N;
  const size_t idx = ((size_t)z * v.ny + y) * v.nx + x;
  const T* din = static_cast<const T*>(v.d_in);
  T* dout = static_cast<T*>(v.d_out);
  const uint8_t fl = v.flags[idx];
  const Nbr n = neighbours(v, x, y, z);
  float d[27];

  if (fl & (F_SOLID | F_INFLOW | F_GHOST)) {
    float ux = 0.f, uy = 0.f, uz = 0.f, cval = 0.f;
    if (fl & F_SOLID) {
#pragma unroll
      for (int k = 0; k < 27; ++k) d[k] = 0.0f;
    } else if (fl & F_GHOST) {
#pragma unroll
      for (int k = 0; k < 27; ++k) d[k] = load_pop(din + (size_t)k * N + idx);
      ux = v.u_in[idx]; uy = v.u_in[N + idx]; uz = v.u_in[2 * N + idx];
      cval = v.c_in[idx];
    } else {  // Dirichlet inflow: equilibrium at rho = 1 and the stored inflow velocity
      ux = v.u_in[idx]; uy = v.u_in[N + idx]; uz = v.u_in[2 * N + idx];
      equilibrium(d, 1.0f, ux, uy, uz);
      cval = (fl & F_SCALAR_SRC) ? v.c_src : sample_scalar(v, x, y, z, ux, uy, uz);
    }
#pragma unroll
    for (int k = 0; k < 27; ++k) store_pop(dout + (size_t)k * N + idx, d[k]);
    v.u_out[idx] = ux; v.u_out[N + idx] = uy; v.u_out[2 * N + idx] = uz;
    v.c_out[idx] = cval;
    return;
  }

  pull_all<T>(d, din, N, n, x);
  if (fl & F_NEAR_SOLID) bounce_back<T>(d, din, N, v.flags, n, x, idx);

  float drho, jx, jy, jz;
  macros(d, drho, jx, jy, jz);
  const float rho = 1.0f + drho;
  const float inv = 1.0f / rho;
  const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
  flag_error(v.err, !(rho > 0.0f) || !(fabsf(ux) + fabsf(uy) + fabsf(uz) < 3.0f));

  const float g = v.rp.adaptive ? grad_norm(v.u_in, N, n, x) : 0.0f;
  const Keep kf = keep_factors(v.rp, g);
  collide(d, drho, ux, uy, uz, kf);

#pragma unroll
  for (int k = 0; k < 27; ++k) store_pop(dout + (size_t)k * N + idx, d[k]);
  v.u_out[idx] = ux; v.u_out[N + idx] = uy; v.u_out[2 * N + idx] = uz;
  v.c_out[idx] = (fl & F_SCALAR_SRC) ? v.c_src : sample_scalar(v, x, y, z, ux, uy, uz);
}

}  // namespace lbm
