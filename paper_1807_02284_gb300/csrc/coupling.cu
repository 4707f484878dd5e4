// Continuous-scale coupling (Sec. 3.2, Sec. 4.2, Algorithm 1): refined blocks at arbitrary
// spacing ratios, prior-mapping of their scale boundary from the nearest coarser block,
// temporal alignment of their sub-cycled states, and post-mapping of their interior into
// every coarser block.
//
// Mapping of post-collision populations from scale s_i to s_j (Sec. 3.2):
//   f^{s_j} = T (m^eq + K_hat (m - m^eq)),  K_hat = (I - S^{s_j}) K (I - S^{s_i})^{-1},
//   diag K = S^{s_i} / (alpha S^{s_j}) on moments 4..8 and 1 elsewhere, alpha = dx_i / dx_j.
// With the same high-order rates on both scales K_hat is 1 outside moments 4..8, so the
// mapping scales only the non-equilibrium shear and deviatoric stress moments: it is the
// relaxation routine with keep factor K_hat on those moments and 1 on every other one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm_cell.cuh"
#include "runtime.h"

namespace lbm {

// ------------------------------------------------------------------------------ kernels

// One CTA maps MAP_D consecutive table entries in three phases, so that the gathers of a
// small mapping (a ghost layer of a few ten thousand nodes) still keep every SM busy:
//   0. one thread per entry: source corners, obstacle-dropped trilinear weights;
//   1. one thread per (entry, population) pair, lanes over consecutive entries: the 8 (or
//      16, when mixing two time levels) gathered loads of one population, into shared memory;
//   2. one thread per entry: moments, K_hat rescale, back to populations (Sec. 3.2);
//   3. one thread per (entry, population) pair: the stores.
// MODE 0: source level lo only; 1: level hi only; 2: (1 - theta) lo + theta hi.  Ghost layers
// of refined blocks also keep the normalised trilinear interpolant of the gathered level in
// a.ghost_store (GHOST_PLANES planes of a.n floats, see k_ghost_finish): MODE 5 maps level lo
// (the ghost layer at t_n), MODE 4 maps level hi blended with the stored interpolant of the
// earlier level, a.ghost_blend, at weight theta (the ghost layer after the first sub-step).
// Entry of destination node e of a whole block: the source cell containing the node's
// position and the fractions inside it, in the same double-precision steps as the host
// tables (cell_of), so both give identical entries.
__device__ __forceinline__ MapEntry geometric_entry(const MapArgs& a, uint32_t e) {
  const uint32_t x = e % (uint32_t)a.dnx, r = e / (uint32_t)a.dnx;
  const uint32_t y = r % (uint32_t)a.dny, z = r / (uint32_t)a.dny;
  const uint32_t node[3] = {x, y, z};
  const int sn[3] = {a.snx, a.sny, a.snz};
  int i0[3];
  MapEntry m;
  float t[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double p = __dadd_rn(a.o_dst[k], __dmul_rn((double)node[k], a.h_dst));  // no FMA
    const double q = __ddiv_rn(__dsub_rn(p, a.o_src[k]), a.h_src);
    int i = (int)floor(q);
    i = max(0, min(i, max(sn[k] - 2, 0)));
    i0[k] = i;
    t[k] = (float)(q - (double)i);
  }
  m.dst = e;
  m.src = (uint32_t)(((size_t)i0[2] * a.sny + i0[1]) * a.snx + i0[0]);
  m.tx = t[0]; m.ty = t[1]; m.tz = t[2];
  return m;
}

// K_hat rescale of interpolated shifted populations (Sec. 3.2): K_hat differs from 1 only on
// moments 4..8 (the shear and deviatoric second moments), so the mapping adds to the
// populations the inverse transform of (K_hat - 1) times their non-equilibrium deviatoric
// second central moments: the same linear map as relaxing every central moment with keep
// factor K_hat on moments 4..8 and 1 elsewhere, without transforming the 21 moments it leaves
// unchanged.  acc holds the populations on entry (it is overwritten), dk receives the
// correction to add to them and u the velocity of the interpolated populations.
__device__ __forceinline__ void khat_delta(float (&acc)[27], float khat, float (&dk)[27],
                                           float (&u)[3]) {
  raw_moments(acc);
  const float drho = acc[kap(0, 0, 0)];
  const float inv = 1.0f / (1.0f + drho);
  const float X = acc[kap(1, 0, 0)] * inv, Y = acc[kap(0, 1, 0)] * inv,
              Z = acc[kap(0, 0, 1)] * inv;
  // second central moments of the shifted populations about u, from the raw ones
  const float R0 = drho, Rx = acc[kap(1, 0, 0)], Ry = acc[kap(0, 1, 0)], Rz = acc[kap(0, 0, 1)];
  const float kxx = acc[kap(2, 0, 0)] + X * fmaf(X, R0, -2.0f * Rx);
  const float kyy = acc[kap(0, 2, 0)] + Y * fmaf(Y, R0, -2.0f * Ry);
  const float kzz = acc[kap(0, 0, 2)] + Z * fmaf(Z, R0, -2.0f * Rz);
  const float kxy = acc[kap(1, 1, 0)] - X * Ry - Y * Rx + X * Y * R0;
  const float kxz = acc[kap(1, 0, 1)] - X * Rz - Z * Rx + X * Z * R0;
  const float kyz = acc[kap(0, 1, 1)] - Y * Rz - Z * Ry + Y * Z * R0;
  // non-equilibrium parts (equilibrium offsets as in relax_to_equilibrium) scaled by K - 1
  const float km1 = khat - 1.0f;
  const float dr3 = drho * (1.0f / 3.0f);
  const float A = kxx - (dr3 - X * X), B = kyy - (dr3 - Y * Y), Cc = kzz - (dr3 - Z * Z);
#pragma unroll
  for (int k = 0; k < 27; ++k) dk[k] = 0.0f;
  dk[kap(1, 1, 0)] = km1 * (kxy + X * Y);
  dk[kap(1, 0, 1)] = km1 * (kxz + X * Z);
  dk[kap(0, 1, 1)] = km1 * (kyz + Y * Z);
  dk[kap(2, 0, 0)] = km1 * (1.0f / 3.0f) * (2.0f * A - B - Cc);
  dk[kap(0, 2, 0)] = km1 * (1.0f / 3.0f) * (2.0f * B - A - Cc);
  dk[kap(0, 0, 2)] = km1 * (1.0f / 3.0f) * (2.0f * Cc - A - B);
  inv_axis<9>(dk, Z);
  inv_axis<3>(dk, Y);
  inv_axis<1>(dk, X);
  u[0] = X;
  u[1] = Y;
  u[2] = Z;
}

constexpr int MAP_THREADS = 128;
constexpr int MAP_LD = 29;         // shared-memory row stride (odd: no bank conflicts)

// MAP_D entries per CTA: 32 for small mappings (a ghost layer of a few ten thousand nodes
// still spreads over every SM), 128 for large ones (one entry per thread: the moment
// transform of phase 2 runs on every warp instead of one).
template <typename T, int MODE, int MAP_D>
__global__ void __launch_bounds__(MAP_THREADS) k_map(MapArgs a) {
  __shared__ float sv[MAP_D * MAP_LD];   // 27 populations + scalar per entry
  __shared__ uint32_t scorner[8][MAP_D];
  __shared__ float sweight[8][MAP_D];
  __shared__ float sinv[MAP_D];          // 1 / sum of weights, 0 for an inactive entry
  __shared__ uint32_t sdst[MAP_D];
  __shared__ float su[3][MAP_D];
  const int t = threadIdx.x;
  const int e0 = blockIdx.x * MAP_D;
  const int nloc = min(MAP_D, a.n - e0);
  const uint32_t sN = (uint32_t)a.sN;
  if (t < MAP_D) {
    // inactive entries keep weight 0 on corner 0, so the gather phase needs no branch
    float inv = 0.0f;
    uint32_t sc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    float w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (t < nloc) {
      const MapEntry m = a.table ? a.table[e0 + t] : geometric_entry(a, (uint32_t)(e0 + t));
      sdst[t] = m.dst;
      if (!(a.dst_flags[m.dst] & a.skip_mask)) {
        const uint32_t sy = (uint32_t)a.snx, sz = (uint32_t)a.snx * (uint32_t)a.sny;
        float wsum = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          sc[c] = m.src + (c & 1) + ((c >> 1) & 1) * sy + (c >> 2) * sz;
          const float wc = ((c & 1) ? m.tx : 1.0f - m.tx) * (((c >> 1) & 1) ? m.ty : 1.0f - m.ty) *
                           ((c >> 2) ? m.tz : 1.0f - m.tz);
          // obstacle corners are dropped (inner voxels, and surface voxels taken as walls)
          w[c] = (__ldg(a.src_flags + sc[c]) & (F_SOLID | F_OBST_WALL)) ? 0.0f : wc;
          wsum += w[c];
        }
        if (wsum > 0.0f) inv = 1.0f / wsum;
        else if (a.rest_if_empty) inv = -1.0f; // every corner an obstacle: rest state
        // (otherwise the node is left unchanged)
      }
    }
    if (!(inv > 0.0f)) {
#pragma unroll
      for (int c = 0; c < 8; ++c) { sc[c] = 0; w[c] = 0.0f; }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) { scorner[c][t] = sc[c]; sweight[c][t] = w[c]; }
    sinv[t] = inv;
  }
  __syncthreads();
  const T* __restrict__ lo = static_cast<const T*>(MODE == 1 || MODE == 4 ? a.f_hi : a.f_lo);
  const T* __restrict__ hi = static_cast<const T*>(a.f_hi);
  const float* __restrict__ clo = MODE == 1 || MODE == 4 ? a.c_hi : a.c_lo;
  const float th = a.theta;
  // every (entry, population) pair of this thread has entry d = lane: corners read once, and
  // the unrolled pairs issue all their loads before the first sum is needed.  A corner of
  // weight 0 (a fraction of 0 on an axis, where the grids line up, or an obstacle corner)
  // is not loaded: its term would add exactly 0.
  static_assert((MAP_D == 32 || MAP_D == 128) && (MAP_D * 28) % MAP_THREADS == 0, "gather layout");
  constexpr int PAIRS = MAP_D * 28 / MAP_THREADS;
  constexpr int KSTEP = MAP_THREADS / MAP_D;   // populations apart of one thread's pairs
  const int d = t % MAP_D;
  uint32_t sc[8];
  float w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) { sc[c] = scorner[c][d]; w[c] = sweight[c][d]; }
  float vals[PAIRS];
#pragma unroll
  for (int i = 0; i < PAIRS; ++i) {
    const int k = t / MAP_D + i * KSTEP;
    float v = 0.0f;
    if (k < 27) {
      const T* pl = lo + (uint32_t)k * sN;
      if (MODE == 2) {
        const T* ph = hi + (uint32_t)k * sN;
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (w[c] != 0.0f)
            v = fmaf(w[c], fmaf(th, load_pop(ph + sc[c]) - load_pop(pl + sc[c]), load_pop(pl + sc[c])), v);
      } else {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (w[c] != 0.0f) v = fmaf(w[c], load_pop(pl + sc[c]), v);
      }
    } else if (MODE == 2) {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (w[c] != 0.0f) {
          v = fmaf(w[c] * (1.0f - th), __ldg(clo + sc[c]), v);
          v = fmaf(w[c] * th, __ldg(a.c_hi + sc[c]), v);
        }
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (w[c] != 0.0f) v = fmaf(w[c], __ldg(clo + sc[c]), v);
    }
    vals[i] = v;
  }
  const float inv_d = sinv[d] > 0.0f ? sinv[d] : 0.0f;     // rest state: all zero
  if constexpr (MODE >= 4) {
    float* S = a.ghost_store;
    const size_t n = (size_t)a.n;
    if (d < nloc) {
#pragma unroll
      for (int i = 0; i < PAIRS; ++i) {
        const int k = t / MAP_D + i * KSTEP;
        if (k < 28) S[(size_t)k * n + e0 + d] = vals[i] * inv_d;
      }
    }
    if (t < nloc) S[(size_t)28 * n + e0 + t] = sinv[t] > 0.0f ? 1.0f : (sinv[t] < 0.0f ? -1.0f : 0.0f);
  }
  {
#pragma unroll
    for (int i = 0; i < PAIRS; ++i) {
      float v = vals[i] * inv_d;
      if constexpr (MODE == 4) {   // (1 - theta) earlier interpolant + theta this one
        const int k = t / MAP_D + i * KSTEP;
        if (k < 28 && d < nloc) {
          const float vlo = a.ghost_blend[(size_t)k * a.n + e0 + d];
          v = fmaf(th, v - vlo, vlo);
        }
      }
      sv[d * MAP_LD + t / MAP_D + i * KSTEP] = v;
    }
    __syncthreads();
    if (t < MAP_D && sinv[t] < 0.0f) {   // rest state: shifted populations, u and scalar 0
      su[0][t] = su[1][t] = su[2][t] = 0.0f;
    }
    if (t < MAP_D && sinv[t] > 0.0f) {
      float acc[27], dk[27], u[3];
#pragma unroll
      for (int k = 0; k < 27; ++k) acc[k] = sv[t * MAP_LD + k];
      khat_delta(acc, a.khat, dk, u);
#pragma unroll
      for (int k = 0; k < 27; ++k) sv[t * MAP_LD + k] += dk[k];
      su[0][t] = u[0];
      su[1][t] = u[1];
      su[2][t] = u[2];
    }
    __syncthreads();
    T* out = static_cast<T*>(a.f_dst);
    const size_t dN = a.dN;
    if (sinv[d] == 0.0f) return;
    const uint32_t dst = sdst[d];
#pragma unroll
    for (int i = 0; i < (31 + KSTEP - 1) / KSTEP; ++i) {
      const int k = t / MAP_D + i * KSTEP;
      if (k < 27) store_pop(out + (size_t)k * dN + dst, sv[d * MAP_LD + k]);
      else if (k < 30) a.u_dst[(size_t)(k - 27) * dN + dst] = su[k - 27][d];
      else if (k == 30) a.c_dst[dst] = sv[d * MAP_LD + 27];
    }
  }
}

// A refined block's ghost layer at t_n + theta dt_0 from the trilinear interpolants of its
// source at t_n (slo) and at t_n + dt_0 (shi), kept by k_map<MODE 5 / 4> once per source
// level and reference step: MODE 0 takes slo, 1 shi, 2 (1 - theta) slo + theta shi (the trilinear
// map is linear, so this equals interpolating the time-blended source), then the K_hat rescale
// (Sec. 3.2).  Buffer layout: planes 0..26 the shifted populations, 27 the scalar, 28 the
// entry's status (1 mapped, -1 every corner an obstacle: rest state, 0 destination left
// alone), each plane a.n floats in table order.  One thread per entry.
template <int MODE>
__global__ void __launch_bounds__(128) k_ghost_finish(const MapEntry* __restrict__ table, int n,
                                                      const float* __restrict__ slo,
                                                      const float* __restrict__ shi, float theta,
                                                      float khat, float* __restrict__ f_dst,
                                                      float* __restrict__ u_dst,
                                                      float* __restrict__ c_dst, size_t dN) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const size_t nn = (size_t)n;
  const float* __restrict__ s0 = MODE == 1 ? shi : slo;
  const float status = s0[28 * nn + e];
  if (status == 0.0f) return;
  const uint32_t dst = table[e].dst;
  // the blended interpolant of plane k (read again for the stores: L1 / L2 hits)
  auto value = [&](int k) {
    const float lo = s0[(size_t)k * nn + e];
    return MODE == 2 ? fmaf(theta, shi[(size_t)k * nn + e] - lo, lo) : lo;
  };
  float dk[27], u[3] = {0.0f, 0.0f, 0.0f}, c = 0.0f;
  if (status > 0.0f) {
    float acc[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) acc[k] = value(k);
    c = value(27);
    khat_delta(acc, khat, dk, u);
  }
#pragma unroll
  for (int k = 0; k < 27; ++k) f_dst[(size_t)k * dN + dst] = status > 0.0f ? value(k) + dk[k] : 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) u_dst[(size_t)a * dN + dst] = u[a];
  c_dst[dst] = c;
}

cudaError_t launch_ghost_map(const MapArgs& a, bool first, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const bool big = a.n >= 152 * 8 * 128;
  if (first) {
    if (big) k_map<float, 5, 128><<<(a.n + 127) / 128, MAP_THREADS, 0, s>>>(a);
    else k_map<float, 5, 32><<<(a.n + 31) / 32, MAP_THREADS, 0, s>>>(a);
  } else {
    if (big) k_map<float, 4, 128><<<(a.n + 127) / 128, MAP_THREADS, 0, s>>>(a);
    else k_map<float, 4, 32><<<(a.n + 31) / 32, MAP_THREADS, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_ghost_finish(const MapEntry* table, int n, const float* slo, const float* shi,
                                float theta, float khat, float* f_dst, float* u_dst,
                                float* c_dst, size_t dN, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (n + 127) / 128;
  if (theta <= 0.0f)
    k_ghost_finish<0><<<grid, 128, 0, s>>>(table, n, slo, shi, theta, khat, f_dst, u_dst, c_dst, dN);
  else if (theta >= 1.0f)
    k_ghost_finish<1><<<grid, 128, 0, s>>>(table, n, slo, shi, theta, khat, f_dst, u_dst, c_dst, dN);
  else
    k_ghost_finish<2><<<grid, 128, 0, s>>>(table, n, slo, shi, theta, khat, f_dst, u_dst, c_dst, dN);
  return cudaGetLastError();
}

template <typename T, int D>
static void launch_map_t(const MapArgs& a, cudaStream_t s) {
  const int grid = (a.n + D - 1) / D;
  if (a.theta <= 0.0f) k_map<T, 0, D><<<grid, MAP_THREADS, 0, s>>>(a);
  else if (a.theta >= 1.0f) k_map<T, 1, D><<<grid, MAP_THREADS, 0, s>>>(a);
  else k_map<T, 2, D><<<grid, MAP_THREADS, 0, s>>>(a);
}

cudaError_t launch_map(const MapArgs& a, int storage, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  // 128 entries per CTA once that still gives every SM about 8 CTAs
  const bool big = a.n >= 152 * 8 * 128;
  if (storage == ST_FP16) {
    if (big) launch_map_t<__half, 128>(a, s);
    else launch_map_t<__half, 32>(a, s);
  } else {
    if (big) launch_map_t<float, 128>(a, s);
    else launch_map_t<float, 32>(a, s);
  }
  return cudaGetLastError();
}

__global__ void k_outer_ghost(uint8_t* flags, int nx, int ny, int nz, int on) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((size_t)nx * ny));
    const bool edge = x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 || z == nz - 1;
    if (!edge) continue;
    const uint8_t f = flags[idx];
    const bool ghost = on && !(f & (F_SOLID | F_OBST_WALL | F_INFLOW));
    flags[idx] = ghost ? (uint8_t)(f | F_GHOST) : (uint8_t)(f & ~F_GHOST);
  }
}

cudaError_t launch_outer_ghost(uint8_t* flags, int nx, int ny, int nz, int on, cudaStream_t s) {
  const size_t N = (size_t)nx * ny * nz;
  const int grid = (int)std::min<size_t>((N + 255) / 256, 65535);
  k_outer_ghost<<<grid, 256, 0, s>>>(flags, nx, ny, nz, on);
  return cudaGetLastError();
}

__global__ void k_set_ghost_layer(uint8_t* flags, int nx, int ny, int nz) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((size_t)nx * ny));
    const bool edge = x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 || z == nz - 1;
    if (edge) flags[idx] |= F_GHOST;
  }
}

cudaError_t launch_set_ghost_layer(uint8_t* flags, int nx, int ny, int nz, cudaStream_t s) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t g = (N + 255) / 256;
  k_set_ghost_layer<<<(int)(g < 8192 ? g : 8192), 256, 0, s>>>(flags, nx, ny, nz);
  return cudaGetLastError();
}

}  // namespace lbm

using namespace lbm;

// --------------------------------------------------------------------------- host side

namespace {

double shear_rate(double nu) { return 1.0 / (3.0 * nu + 0.5); }

// K_hat on moments 4..8 for src -> dst (Sec. 3.2); alpha = dx_src / dx_dst.
double khat(const Block& src, const Block& dst) {
  const double Ss = shear_rate(src.nu), Sd = shear_rate(dst.nu);
  const double alpha = src.h / dst.h;
  return (1.0 - Sd) * (Ss / (alpha * Sd)) / (1.0 - Ss);
}

// Trilinear cell of a reference-unit point p in block B: lower corner index and fractions.
void cell_of(const Block& B, const double p[3], uint32_t* base, float t[3]) {
  const int n[3] = {B.nx, B.ny, B.nz};
  int i0[3];
  for (int a = 0; a < 3; ++a) {
    const double q = (p[a] - B.origin[a]) / B.h;
    int i = (int)std::floor(q);
    i = std::max(0, std::min(i, std::max(n[a] - 2, 0)));
    i0[a] = i;
    t[a] = (float)(q - i);
  }
  *base = (uint32_t)(((size_t)i0[2] * B.ny + i0[1]) * B.nx + i0[0]);
}

bool contains(const Block& outer, const Block& inner) {
  for (int a = 0; a < 3; ++a) {
    const int no = a == 0 ? outer.nx : a == 1 ? outer.ny : outer.nz;
    const int ni = a == 0 ? inner.nx : a == 1 ? inner.ny : inner.nz;
    const double lo = inner.origin[a], hi = inner.origin[a] + (ni - 1) * inner.h;
    const double olo = outer.origin[a], ohi = outer.origin[a] + (no - 1) * outer.h;
    if (lo < olo - 1e-9 || hi > ohi + 1e-9) return false;
  }
  return true;
}

}  // namespace

// The table's entry count is set only once its device copy exists, so a failed upload can
// never leave a launchable table without storage.
static lbm_status upload_table(lbm_domain* dom, const std::vector<MapEntry>& h, MapTable* t) {
  t->n = 0;
  t->d = nullptr;
  if (h.empty()) return LBM_OK;
  MapEntry* d = static_cast<MapEntry*>(dom->dev_alloc(h.size() * sizeof(MapEntry)));
  if (!d) return dom->fail(LBM_ERR_OOM, "mapping table allocation failed");
  cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(MapEntry),
                                  cudaMemcpyHostToDevice, dom->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(dom->stream);
  if (e != cudaSuccess) {
    dom->dev_free(d);
    return dom->cuda_fail(e, "mapping table upload");
  }
  t->d = d;
  t->n = (int)h.size();
  return LBM_OK;
}

// Frees every device buffer of a block that is not (or no longer) part of the domain.
static void release_block(lbm_domain* dom, Block& B) {
  for (Level& L : B.lv) {
    dom->dev_free(L.f);
    dom->dev_free(L.u);
    dom->dev_free(L.c);
    L = Level();
  }
  dom->dev_free(B.flags);
  B.flags = nullptr;
  dom->dev_free(B.prior.d);
  B.prior.d = nullptr;
  B.prior.n = 0;
  for (float*& g : B.gs) {
    dom->dev_free(g);
    g = nullptr;
  }
  for (MapTable& t : B.post) dom->dev_free(t.d);
  B.post.clear();
  dom->dev_free(B.far_in.d);
  dom->dev_free(B.far_out.d);
  B.far_in = MapTable();
  B.far_out = MapTable();
}

// Table of the nodes of block T that lie in block S's interior span [o + h, o + (n-2) h] on
// every axis, with their source cells in S (prior-mapping regions of refined blocks' post
// maps, and of far blocks' overlap).
// Index box of the nodes of block T inside block S's interior span [o + h, o + (n-2) h] on
// every axis; false if it is empty.
static bool interior_box(const Block& S, const Block& T, int lo[3], int hi[3]) {
  const int nT[3] = {T.nx, T.ny, T.nz};
  const int nS[3] = {S.nx, S.ny, S.nz};
  for (int a = 0; a < 3; ++a) {
    const double plo = S.origin[a] + S.h, phi = S.origin[a] + (nS[a] - 2) * S.h;
    lo[a] = std::max(0, (int)std::ceil((plo - 1e-9 - T.origin[a]) / T.h));
    hi[a] = std::min(nT[a] - 1, (int)std::floor((phi + 1e-9 - T.origin[a]) / T.h));
    while (lo[a] <= hi[a] && T.origin[a] + lo[a] * T.h < plo - 1e-9) ++lo[a];
    while (hi[a] >= lo[a] && T.origin[a] + hi[a] * T.h > phi + 1e-9) --hi[a];
    if (lo[a] > hi[a]) return false;
  }
  return true;
}

static std::vector<MapEntry> interior_table(const Block& S, const Block& T) {
  std::vector<MapEntry> tab;
  int lo[3], hi[3];
  if (!interior_box(S, T, lo, hi)) return tab;
  tab.reserve((size_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1));
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const double p[3] = {T.origin[0] + x * T.h, T.origin[1] + y * T.h, T.origin[2] + z * T.h};
        MapEntry m;
        m.dst = (uint32_t)(((size_t)z * T.ny + y) * T.nx + x);
        float t[3];
        cell_of(S, p, &m.src, t);
        m.tx = t[0]; m.ty = t[1]; m.tz = t[2];
        tab.push_back(m);
      }
  return tab;
}

// Table of the outer-layer nodes of block T with their source cells in block S.
static std::vector<MapEntry> outer_table(const Block& S, const Block& T) {
  std::vector<MapEntry> tab;
  for (int z = 0; z < T.nz; ++z)
    for (int y = 0; y < T.ny; ++y)
      for (int x = 0; x < T.nx; ++x) {
        const bool edge = x == 0 || y == 0 || z == 0 || x == T.nx - 1 || y == T.ny - 1 ||
                          z == T.nz - 1;
        if (!edge) continue;
        const double p[3] = {T.origin[0] + x * T.h, T.origin[1] + y * T.h, T.origin[2] + z * T.h};
        MapEntry m;
        m.dst = (uint32_t)(((size_t)z * T.ny + y) * T.nx + x);
        float t[3];
        cell_of(S, p, &m.src, t);
        m.tx = t[0]; m.ty = t[1]; m.tz = t[2];
        tab.push_back(m);
      }
  return tab;
}

// Index of the block a new far-field block has to surround: the last far block, else s0.
static int outermost(const lbm_domain* dom) {
  int c = 0;
  for (size_t i = 1; i < dom->blocks.size(); ++i)
    if (dom->blocks[i].far) c = (int)i;
  return c;
}

static lbm_status add_far_block(lbm_domain* dom, const double origin[3], double h,
                                const int32_t dims[3], int32_t* block_id) {
  for (int a = 0; a < 3; ++a)
    if (dom->desc.periodic[a])
      return dom->fail(LBM_ERR_UNSUPPORTED, "far-field blocks need a reference block without periodic faces");
  if (dom->walls & ~WALLS_OBSTACLES)
    return dom->fail(LBM_ERR_UNSUPPORTED, "wall faces and far-field blocks exclude each other");
  Block F;
  F.nx = dims[0]; F.ny = dims[1]; F.nz = dims[2];
  F.N = (size_t)F.nx * F.ny * F.nz;
  for (int a = 0; a < 3; ++a) F.origin[a] = origin[a];
  F.h = h;
  F.nu = dom->desc.nu / h;
  F.substeps = 1;
  F.integer_ratio = false;
  F.rp = dom->relax_params(F.nu);
  F.far = true;
  F.child = outermost(dom);
  const Block& C = dom->blocks[F.child];
  if (!contains(F, C)) return dom->fail(LBM_ERR_INVALID_ARG, "a far-field block must contain the outermost block");
  if (std::fabs(1.0 - shear_rate(F.nu)) < 1e-12)
    return dom->fail(LBM_ERR_INVALID_ARG, "K_hat is undefined for S = 1 (nu = 1/6 on this block)");
  const int id = (int)dom->blocks.size();
  lbm_status st = dom->alloc_block_levels(F, 2);
  if (st != LBM_OK) {
    release_block(dom, F);
    return st;
  }
  dom->blocks.push_back(F);
  auto abandon = [dom](lbm_status s) {
    cudaStreamSynchronize(dom->stream);
    release_block(dom, dom->blocks.back());
    dom->blocks.pop_back();
    return s;
  };
  st = dom->clear_block(id);
  if (st != LBM_OK) return abandon(st);
  Block& NF = dom->blocks.back();
  const Block& CC = dom->blocks[NF.child];
  NF.far_in.src = NF.child;
  NF.far_in.dst = id;
  NF.far_in.khat = (float)khat(CC, NF);
  st = upload_table(dom, interior_table(CC, NF), &NF.far_in);
  if (st != LBM_OK) return abandon(st);
  NF.far_out.src = id;
  NF.far_out.dst = NF.child;
  NF.far_out.khat = (float)khat(NF, CC);
  st = upload_table(dom, outer_table(NF, CC), &NF.far_out);
  if (st != LBM_OK) return abandon(st);
  Block& CW = dom->blocks[NF.child];
  const cudaError_t e = launch_outer_ghost(CW.flags, CW.nx, CW.ny, CW.nz, 1, dom->stream);
  if (e != cudaSuccess) return abandon(dom->cuda_fail(e, "scale-boundary flags"));
  dom->pick_tiles(id);
  dom->invalidate_graphs();
  *block_id = id;
  return LBM_OK;
}

extern "C" lbm_status lbm_add_scale_block(lbm_domain* dom, const double origin[3], double h,
                                          const int32_t dims[3], int32_t* block_id) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (!origin || !dims || !block_id) return dom->fail(LBM_ERR_INVALID_ARG, "null argument");
  if (!(h > 0.0) || !std::isfinite(h)) return dom->fail(LBM_ERR_INVALID_ARG, "h must be positive");
  if (std::fabs(h - 1.0) < 1e-12) return dom->fail(LBM_ERR_INVALID_ARG, "h = 1 is the reference scale");
  if (dom->desc.storage != LBM_FP32)
    return dom->fail(LBM_ERR_UNSUPPORTED, "scale blocks need FP32 storage");
  if (dom->tape)
    return dom->fail(LBM_ERR_STATE, "blocks cannot be added while an adjoint tape is recording");
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 4) return dom->fail(LBM_ERR_INVALID_ARG, "scale blocks need >= 4 nodes per axis");
  if ((double)dims[0] * dims[1] * dims[2] * 27.0 >= 4294967295.0)
    return dom->fail(LBM_ERR_INVALID_ARG, "scale block too large");
  if (dims[2] > 65535) return dom->fail(LBM_ERR_INVALID_ARG, "nz must be <= 65535");
  if ((double)dom->blocks[0].N * 27.0 >= 4294967295.0)
    return dom->fail(LBM_ERR_UNSUPPORTED, "the reference block is too large for coupling tables");
  if (h > 1.0) return add_far_block(dom, origin, h, dims, block_id);
  {
    int last = 0;                    // last refined block (far-field blocks do not count)
    for (size_t i = 1; i < dom->blocks.size(); ++i)
      if (!dom->blocks[i].far) last = (int)i;
    if (last > 0 && h > dom->blocks[last].h + 1e-12)
      return dom->fail(LBM_ERR_INVALID_ARG, "refined blocks must be added coarse to fine");
  }
  Block B;
  B.nx = dims[0]; B.ny = dims[1]; B.nz = dims[2];
  B.N = (size_t)B.nx * B.ny * B.nz;
  for (int a = 0; a < 3; ++a) B.origin[a] = origin[a];
  B.h = h;
  B.nu = dom->desc.nu / h;               // Re invariance: 1/S_f - 1/2 = alpha (1/S_c - 1/2)
  const double ratio = 1.0 / h;
  B.substeps = std::max(1, (int)std::ceil(ratio - 1e-9));
  B.integer_ratio = std::fabs(ratio - std::round(ratio)) < 1e-9;
  B.rp = dom->relax_params(B.nu);
  if (!contains(dom->blocks[0], B))
    return dom->fail(LBM_ERR_INVALID_ARG, "the block must lie inside the reference block");
  if (std::fabs(1.0 - shear_rate(B.nu)) < 1e-12)
    return dom->fail(LBM_ERR_INVALID_ARG, "K_hat is undefined for S = 1 (nu = 1/6 on this block)");
  for (const Block& C : dom->blocks)
    if (std::fabs(1.0 - shear_rate(C.nu)) < 1e-12)
      return dom->fail(LBM_ERR_INVALID_ARG, "K_hat is undefined for S = 1 on a coarser block");

  // prior-mapping source: the finest coarser block that contains the whole block
  int parent = 0;
  for (size_t j = 1; j < dom->blocks.size(); ++j) {
    const Block& C = dom->blocks[j];
    if (C.h > B.h && contains(C, B) && C.h < dom->blocks[parent].h) parent = (int)j;
  }
  B.parent = parent;
  const int id = (int)dom->blocks.size();

  lbm_status st = dom->alloc_block_levels(B, 3);
  if (st != LBM_OK) {
    release_block(dom, B);
    return st;
  }
  // From here on the block is in the domain; any failure takes it out again, with its
  // buffers and tables, so that no later step can launch on a half-built block.
  dom->blocks.push_back(B);
  auto abandon = [dom](lbm_status s) {
    cudaStreamSynchronize(dom->stream);
    release_block(dom, dom->blocks.back());
    dom->blocks.pop_back();
    return s;
  };
  Block& NB = dom->blocks.back();
  st = dom->clear_block(id);
  if (st != LBM_OK) return abandon(st);
  cudaError_t e = launch_set_ghost_layer(NB.flags, NB.nx, NB.ny, NB.nz, dom->stream);
  if (e != cudaSuccess) return abandon(dom->cuda_fail(e, "ghost flags"));

  // prior table: ghost nodes of the new block -> cells of the parent
  {
    std::vector<MapEntry> tab;
    const Block& P = dom->blocks[parent];
    for (int z = 0; z < NB.nz; ++z)
      for (int y = 0; y < NB.ny; ++y)
        for (int x = 0; x < NB.nx; ++x) {
          const bool edge = x == 0 || y == 0 || z == 0 || x == NB.nx - 1 || y == NB.ny - 1 ||
                            z == NB.nz - 1;
          if (!edge) continue;
          const double p[3] = {NB.origin[0] + x * NB.h, NB.origin[1] + y * NB.h,
                               NB.origin[2] + z * NB.h};
          MapEntry m;
          m.dst = (uint32_t)(((size_t)z * NB.ny + y) * NB.nx + x);
          float t[3];
          cell_of(P, p, &m.src, t);
          m.tx = t[0]; m.ty = t[1]; m.tz = t[2];
          tab.push_back(m);
        }
    NB.prior.src = parent;
    NB.prior.dst = id;
    NB.prior.khat = (float)khat(P, NB);
    st = upload_table(dom, tab, &NB.prior);
    if (st != LBM_OK) return abandon(st);
    for (float*& g : NB.gs) {
      g = static_cast<float*>(dom->dev_alloc((size_t)GHOST_PLANES * tab.size() * sizeof(float)));
      if (!g) return abandon(dom->fail(LBM_ERR_OOM, "ghost-layer interpolant buffers"));
    }
  }
  // post tables: nodes of every coarser block inside the new block's interior span
  for (int k = 0; k < id; ++k) {
    const Block& T = dom->blocks[k];
    if (T.far || !(T.h > NB.h)) continue;
    MapTable mt;
    mt.src = id;
    mt.dst = k;
    mt.khat = (float)khat(NB, T);
    st = upload_table(dom, interior_table(NB, T), &mt);
    if (st != LBM_OK) return abandon(st);
    NB.post.push_back(mt);
  }
  dom->pick_tiles(id);
  dom->invalidate_graphs();
  *block_id = id;
  return LBM_OK;
}

extern "C" lbm_status lbm_remove_scale_block(lbm_domain* dom, int32_t block_id) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (block_id < 1 || block_id != (int32_t)dom->blocks.size() - 1)
    return dom->fail(LBM_ERR_INVALID_ARG, "only the most recently added refined block can be removed");
  if (dom->tape)
    return dom->fail(LBM_ERR_STATE, "blocks cannot be removed while an adjoint tape is recording");
  // every launch that may read the block (steps, mappings on the side streams) has been
  // joined into the domain's stream, so waiting for it makes the buffers free to release
  const cudaError_t e = cudaStreamSynchronize(dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "cudaStreamSynchronize");
  const bool far = dom->blocks.back().far;
  const int child = dom->blocks.back().child;
  release_block(dom, dom->blocks.back());
  dom->blocks.pop_back();
  dom->invalidate_graphs();
  if (far) {   // the child's outer layer is again an open face
    Block& C = dom->blocks[child];
    const cudaError_t e2 = launch_outer_ghost(C.flags, C.nx, C.ny, C.nz, 0, dom->stream);
    if (e2 != cudaSuccess) return dom->cuda_fail(e2, "scale-boundary flags");
  }
  return LBM_OK;
}

// Prior-mapping of block b's ghost layer (Sec. 3.2, Algorithm 1).  The ghost layer at
// t_n + theta dt_0 is the K_hat-rescaled trilinear interpolant of the parent blended linearly
// in time between its levels at t_n and t_n + dt_0; the trilinear part is linear, so it is
// gathered once per parent level and reference step, and kept in the block's interpolant
// buffers (0 = t_n, 1 = t_n + dt_0).  ghost_map gathers a level and writes a ghost layer in
// the same launch: first = true the parent's level `src_level` at t_n (ghost layer at
// theta = 0 into `dst_level`), first = false its level at t_n + dt_0, blended with buffer 0
// at `theta` (the ghost layer after the first sub-step).  Every later ghost layer of the step
// only blends the two buffers and rescales (ghost_finish).
static cudaError_t ghost_map(lbm_domain* dom, int b, bool first, int src_level, float theta,
                             int dst_level, cudaStream_t stream) {
  Block& B = dom->blocks[b];
  const Block& P = dom->blocks[B.prior.src];
  MapArgs a{};
  a.rest_if_empty = 1;           // scale boundary
  a.table = B.prior.d;
  a.n = B.prior.n;
  a.f_lo = a.f_hi = P.lv[src_level].f;
  a.c_lo = a.c_hi = P.lv[src_level].c;
  a.theta = first ? 0.0f : theta;
  a.src_flags = P.flags;
  a.snx = P.nx; a.sny = P.ny; a.sN = P.N;
  a.f_dst = B.lv[dst_level].f;
  a.u_dst = B.lv[dst_level].u;
  a.c_dst = B.lv[dst_level].c;
  a.dst_flags = B.flags;
  a.skip_mask = F_SOLID | F_OBST_WALL;   // obstacle voxels keep their own state
  a.dN = B.N;
  a.khat = B.prior.khat;
  a.ghost_store = B.gs[first ? 0 : 1];
  a.ghost_blend = B.gs[0];
  return launch_ghost_map(a, first, stream);
}

static cudaError_t ghost_finish(lbm_domain* dom, int b, float theta, int dst_level,
                                cudaStream_t stream) {
  Block& B = dom->blocks[b];
  const Level& D = B.lv[dst_level];
  return launch_ghost_finish(B.prior.d, B.prior.n, B.gs[0], B.gs[1], theta, B.prior.khat,
                             static_cast<float*>(D.f), D.u, D.c, B.N, stream);
}

static cudaError_t post_map(lbm_domain* dom, int b, const MapTable& t, cudaStream_t stream) {
  const Block& B = dom->blocks[b];
  Block& T = dom->blocks[t.dst];
  MapArgs a{};
  a.rest_if_empty = 0;           // post-mapped nodes keep their own update
  a.table = t.d;
  a.n = t.n;
  a.f_lo = a.f_hi = B.lv[B.cur].f;
  a.c_lo = a.c_hi = B.lv[B.cur].c;
  a.theta = 0.0f;
  a.src_flags = B.flags;
  a.snx = B.nx; a.sny = B.ny; a.sN = B.N;
  a.f_dst = T.lv[T.cur].f;
  a.u_dst = T.lv[T.cur].u;
  a.c_dst = T.lv[T.cur].c;
  a.dst_flags = T.flags;
  a.skip_mask = F_SOLID | F_OBST_WALL | F_GHOST;
  a.dN = T.N;
  a.khat = t.khat;
  return launch_map(a, dom->desc.storage, stream);
}

// Mapping between the current states of two blocks along a far-field table (the destination
// nodes carrying any of `skip` are left alone).
static cudaError_t far_map(lbm_domain* dom, const MapTable& t, uint8_t skip, int rest,
                           cudaStream_t stream) {
  const Block& S = dom->blocks[t.src];
  Block& T = dom->blocks[t.dst];
  MapArgs a{};
  a.rest_if_empty = rest;
  a.table = t.d;
  a.n = t.n;
  a.f_lo = a.f_hi = S.lv[S.cur].f;
  a.c_lo = a.c_hi = S.lv[S.cur].c;
  a.theta = 0.0f;
  a.src_flags = S.flags;
  a.snx = S.nx; a.sny = S.ny; a.snz = S.nz; a.sN = S.N;
  a.f_dst = T.lv[T.cur].f;
  a.u_dst = T.lv[T.cur].u;
  a.c_dst = T.lv[T.cur].c;
  a.dst_flags = T.flags;
  a.skip_mask = skip;
  a.dN = T.N;
  a.khat = t.khat;
  return launch_map(a, dom->desc.storage, stream);
}

// One reference step of Algorithm 1 over all blocks.  Per refined block: the ghost-layer
// mapping for the next sub-step runs on the auxiliary stream while the current sub-step's
// collide-stream runs on the main stream (the two write disjoint nodes); the last sub-step
// stores the temporal alignment directly; post-mappings into different coarser blocks run
// concurrently.  Every fork is joined before the next dependent launch.
lbm_status multiscale_step(lbm_domain* dom) {
  std::vector<int> saved(dom->blocks.size());
  for (size_t b = 0; b < dom->blocks.size(); ++b) saved[b] = dom->blocks[b].cur;
  std::vector<char> pending(dom->blocks.size(), 0);   // target has post-mappings in flight
  cudaStream_t s = dom->stream;
  cudaStream_t aux = nullptr;
  lbm_status st = dom->aux(&aux);
  if (st != LBM_OK) return st;
  cudaError_t e;
  const int nb = (int)dom->blocks.size();
  // early phase, on its own stream, concurrent with s0's step: every refined block's ghost
  // refresh at t_n and first sub-step need only t_n states (its source's saved level and its
  // own), so they run while s0 advances (the later sub-steps need s0's new state)
  cudaStream_t early = dom->post_stream(nb);
  if (!early) return dom->fail(LBM_ERR_CUDA, "early-phase stream");
  e = cudaEventRecord(dom->event(4), s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(early, dom->event(4), 0);
  if (e != cudaSuccess) return dom->cuda_fail(e, "early-phase fork");
  for (int b = 1; b < nb && e == cudaSuccess; ++b) {
    Block& B = dom->blocks[b];
    if (B.far) continue;
    const int L = saved[b], A = (L + 1) % 3;
    e = ghost_map(dom, b, true, saved[B.prior.src], 0.0f, L, early);
    if (e == cudaSuccess) e = cudaEventRecord(dom->event(10 + 2 * nb + b), early);
    if (e == cudaSuccess) e = launch_step(dom->view(b, L, A), dom->desc.storage, B.bx, B.by, early, B.minb);
    if (e == cudaSuccess) e = cudaEventRecord(dom->event(10 + nb + b), early);
  }
  if (e != cudaSuccess) return dom->cuda_fail(e, "early phase");
  {  // reference scale: one step
    Block& B0 = dom->blocks[0];
    const int nxt = B0.cur ^ 1;
    e = launch_step(dom->view(0, B0.cur, nxt), dom->desc.storage, B0.bx, B0.by, s, B0.minb);
    if (e != cudaSuccess) return dom->cuda_fail(e, "collide-stream launch");
    B0.cur = nxt;
  }
  // far field (Sec. 4.2.4-4.2.5): every far block takes one step of its own dt = h dt_0 and
  // is interpolated back to t_n + dt_0 (the fused alignment with weights 0, 1 - 1/h, 1/h);
  // then, inner to outer, its nodes inside its child's interior come from the child, and,
  // outer to inner, the child's outer layer comes from it
  std::vector<int> far;
  for (size_t bi = 1; bi < dom->blocks.size(); ++bi)
    if (dom->blocks[bi].far) far.push_back((int)bi);
  for (int f : far) {
    Block& F = dom->blocks[f];
    const int nxt = F.cur ^ 1;
    BlockView v = dom->view(f, F.cur, nxt);
    v.f_al0 = F.lv[F.cur].f;
    v.c_al0 = F.lv[F.cur].c;
    v.al0 = 0.0f;
    v.al1 = (float)(1.0 - 1.0 / F.h);
    v.al2 = (float)(1.0 / F.h);
    e = launch_step_align(v, F.bx, F.by, s, F.minb);
    if (e != cudaSuccess) return dom->cuda_fail(e, "far-field step");
    F.cur = nxt;
  }
  for (int f : far) {
    const Block& F = dom->blocks[f];
    e = far_map(dom, F.far_in, F_SOLID | F_GHOST, 0, s);
    if (e != cudaSuccess) return dom->cuda_fail(e, "far-field overlap mapping");
  }
  for (size_t k = far.size(); k-- > 0;) {
    const Block& F = dom->blocks[far[k]];
    e = far_map(dom, F.far_out, F_SOLID | F_OBST_WALL | F_INFLOW, 1, s);
    if (e != cudaSuccess) return dom->cuda_fail(e, "far-field boundary mapping");
  }
  for (size_t bi = 1; bi < dom->blocks.size(); ++bi) {
    const int b = (int)bi;
    Block& B = dom->blocks[b];
    if (B.far) continue;
    const int L = saved[b];
    const int A = (L + 1) % 3, Bv = (L + 2) % 3;
    const bool exact = B.integer_ratio && std::fabs(B.substeps * B.h - 1.0) < 1e-9;
    int cur = L;
    if (pending[B.prior.src]) {      // the source block may still receive post-mappings
      e = cudaStreamWaitEvent(s, dom->event(10 + B.prior.src), 0);
      if (e != cudaSuccess) return dom->cuda_fail(e, "post-mapping join");
    }
    // the early phase's interpolant at t_n is needed from the first ghost layer on, its first
    // sub-step only by the second one
    e = cudaStreamWaitEvent(s, dom->event(10 + 2 * nb + b), 0);
    if (e != cudaSuccess) return dom->cuda_fail(e, "early-phase join");
    for (int j = 1; j <= B.substeps; ++j) {
      const int out = (j == 1) ? A : (cur == A ? Bv : A);
      // ghost layer of `out` for the next sub-step (or at t_n + dt_0 after the last): forked,
      // concurrent with this sub-step's collide-stream (disjoint nodes), except after the
      // first sub-step, which ran in the early phase: there the source's new level is
      // gathered (once for every later ghost layer of the step) and blended
      const float theta = j < B.substeps ? (float)(j * B.h) : 1.0f;
      if (j == 1) {
        e = ghost_map(dom, b, false, dom->blocks[B.prior.src].cur, theta, out, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, dom->event(10 + nb + b), 0);
        if (e != cudaSuccess) return dom->cuda_fail(e, "prior-mapping");
        cur = out;
        continue;
      }
      e = cudaEventRecord(dom->event(0), s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, dom->event(0), 0);
      if (e == cudaSuccess) e = ghost_finish(dom, b, theta, out, aux);
      if (e == cudaSuccess) e = cudaEventRecord(dom->event(1), aux);
      if (e != cudaSuccess) return dom->cuda_fail(e, "prior-mapping");
      BlockView v = dom->view(b, cur, out);
      if (j == B.substeps && !exact) {
        const double t1 = (B.substeps - 1) * B.h, t2 = B.substeps * B.h, T = 1.0;
        v.f_al0 = B.lv[L].f;
        v.c_al0 = B.lv[L].c;
        v.al0 = (float)((T - t1) * (T - t2) / ((0.0 - t1) * (0.0 - t2)));
        v.al1 = (float)((T - 0.0) * (T - t2) / ((t1 - 0.0) * (t1 - t2)));
        v.al2 = (float)((T - 0.0) * (T - t1) / ((t2 - 0.0) * (t2 - t1)));
        e = launch_step_align(v, B.bx, B.by, s, B.minb);
      } else {
        e = launch_step(v, dom->desc.storage, B.bx, B.by, s, B.minb);
      }
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, dom->event(1), 0);   // join
      if (e != cudaSuccess) return dom->cuda_fail(e, "collide-stream launch");
      cur = out;
    }
    B.cur = cur;
    // post-mapping: each coarser target block has its own stream, so mappings into different
    // targets run concurrently with each other and with the finer blocks' sub-steps; a later
    // reader of a target (a prior-mapping source, the next step) waits for its mappings
    e = cudaEventRecord(dom->event(2), s);
    for (size_t t = 0; t < B.post.size() && e == cudaSuccess; ++t) {
      const int k = B.post[t].dst;
      cudaStream_t ps = dom->post_stream(k);
      if (!ps) return dom->fail(LBM_ERR_CUDA, "post-mapping stream");
      e = cudaStreamWaitEvent(ps, dom->event(2), 0);
      if (e == cudaSuccess) e = post_map(dom, b, B.post[t], ps);
      if (e == cudaSuccess) e = cudaEventRecord(dom->event(10 + k), ps);
      pending[k] = 1;
    }
    if (e != cudaSuccess) return dom->cuda_fail(e, "post-mapping");
  }
  for (size_t k = 0; k < pending.size(); ++k)      // join every target before the next step
    if (pending[k]) {
      e = cudaStreamWaitEvent(s, dom->event(10 + (int)k), 0);
      if (e != cudaSuccess) return dom->cuda_fail(e, "post-mapping join");
    }
  return LBM_OK;
}

// ------------------------------------------------------------------ phase-by-phase stepping
//
// One reference step of Algorithm 1 as a sequence of calls, so that the blocks of one
// continuous-scale domain can be advanced by different processes (each holds the whole
// domain, computes the blocks it owns and receives, between phases, the node boxes of other
// blocks that its mappings read or that other ranks' mappings wrote).  Every rank issues the
// same phases; a phase that a rank does not compute only advances the block's time levels
// exactly as computing it would, so level indices agree on all ranks.  The kernels, their
// inputs and their order are those of multiscale_step (launched one after another on the
// domain's stream), so the results are bit-identical to lbm_step.

namespace lbm {

// Packs (dir 0) or unpacks (dir 1) the box lo..hi of one level of a block: 27 population
// planes as stored (FP32), then 3 velocity planes and the scalar plane, nb values each.
// Unpacking leaves nodes whose flags carry any bit of `skip` unchanged.
__global__ void k_box(float* f, float* u, float* c, const uint8_t* flags, int nx, int ny,
                      size_t N, int3 lo, int3 dim, size_t nb, float* buf, int dir, int skip) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nb;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = lo.x + (int)(i % dim.x);
    const int y = lo.y + (int)((i / dim.x) % dim.y);
    const int z = lo.z + (int)(i / ((size_t)dim.x * dim.y));
    const size_t idx = ((size_t)z * ny + y) * nx + x;
    if (dir == 0) {
#pragma unroll
      for (int k = 0; k < 27; ++k) buf[(size_t)k * nb + i] = f[(size_t)k * N + idx];
#pragma unroll
      for (int a = 0; a < 3; ++a) buf[(size_t)(27 + a) * nb + i] = u[(size_t)a * N + idx];
      buf[(size_t)30 * nb + i] = c[idx];
    } else {
      if (flags[idx] & skip) continue;
#pragma unroll
      for (int k = 0; k < 27; ++k) f[(size_t)k * N + idx] = buf[(size_t)k * nb + i];
#pragma unroll
      for (int a = 0; a < 3; ++a) u[(size_t)a * N + idx] = buf[(size_t)(27 + a) * nb + i];
      c[idx] = buf[(size_t)30 * nb + i];
    }
  }
}

}  // namespace lbm

namespace {

// Level a refined block ends a reference step in, starting from level L (the rotation of
// multiscale_step: the first sub-step writes L + 1, then the other two levels alternate).
int final_level(const Block& B, int L) {
  const int A = (L + 1) % 3, Bv = (L + 2) % 3;
  int c = L;
  for (int j = 1; j <= B.substeps; ++j) c = (j == 1) ? A : (c == A ? Bv : A);
  return c;
}

// The whole sub-cycle of refined block b in one stream: ghost layer at t_n, then per
// sub-step the collide-stream (the last one with the temporal alignment unless the ratio
// is an integer) followed by the ghost layer of its output level.
cudaError_t block_subcycle(lbm_domain* dom, int b, cudaStream_t s) {
  Block& B = dom->blocks[b];
  const std::vector<int>& saved = dom->phase_saved;
  const int L = saved[b];
  const int A = (L + 1) % 3, Bv = (L + 2) % 3;
  const bool exact = B.integer_ratio && std::fabs(B.substeps * B.h - 1.0) < 1e-9;
  cudaError_t e = ghost_map(dom, b, true, saved[B.prior.src], 0.0f, L, s);
  int cur = L;
  for (int j = 1; j <= B.substeps && e == cudaSuccess; ++j) {
    const int out = (j == 1) ? A : (cur == A ? Bv : A);
    BlockView v = dom->view(b, cur, out);
    if (j == B.substeps && !exact) {
      const double t1 = (B.substeps - 1) * B.h, t2 = B.substeps * B.h, T = 1.0;
      v.f_al0 = B.lv[L].f;
      v.c_al0 = B.lv[L].c;
      v.al0 = (float)((T - t1) * (T - t2) / ((0.0 - t1) * (0.0 - t2)));
      v.al1 = (float)((T - 0.0) * (T - t2) / ((t1 - 0.0) * (t1 - t2)));
      v.al2 = (float)((T - 0.0) * (T - t1) / ((t2 - 0.0) * (t2 - t1)));
      e = launch_step_align(v, B.bx, B.by, s, B.minb);
    } else {
      e = launch_step(v, dom->desc.storage, B.bx, B.by, s, B.minb);
    }
    const float theta = j < B.substeps ? (float)(j * B.h) : 1.0f;
    if (e == cudaSuccess)
      e = j == 1 ? ghost_map(dom, b, false, dom->blocks[B.prior.src].cur, theta, out, s)
                 : ghost_finish(dom, b, theta, out, s);
    cur = out;
  }
  B.cur = cur;
  return e;
}

// Ghost-layer source box of refined block b in its parent P, face f (axis f / 2, low or high
// side f % 2): the parent nodes that are corners of the trilinear cells of that face's nodes.
void prior_face_box(const Block& P, const Block& B, int f, int lo[3], int hi[3]) {
  const int nB[3] = {B.nx, B.ny, B.nz}, nP[3] = {P.nx, P.ny, P.nz};
  for (int a = 0; a < 3; ++a) {
    double p0 = B.origin[a], p1 = B.origin[a] + (nB[a] - 1) * B.h;
    if (a == f / 2) p0 = p1 = (f % 2) ? p1 : p0;
    int i0 = (int)std::floor((p0 - P.origin[a]) / P.h);
    int i1 = (int)std::floor((p1 - P.origin[a]) / P.h);
    i0 = std::max(0, std::min(i0, std::max(nP[a] - 2, 0)));
    i1 = std::max(0, std::min(i1, std::max(nP[a] - 2, 0)));
    lo[a] = i0;
    hi[a] = std::min(i1 + 1, nP[a] - 1);
  }
}

bool valid_box(const Block& B, const int32_t lo[3], const int32_t hi[3]) {
  const int n[3] = {B.nx, B.ny, B.nz};
  for (int a = 0; a < 3; ++a)
    if (lo[a] < 0 || hi[a] >= n[a] || lo[a] > hi[a]) return false;
  return true;
}

size_t box_nodes(const int32_t lo[3], const int32_t hi[3]) {
  return (size_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
}

}  // namespace

extern "C" lbm_status lbm_step_phase(lbm_domain* dom, int32_t phase, int32_t block,
                                     int32_t compute) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  const int nb = (int)dom->blocks.size();
  cudaStream_t s = dom->stream;
  cudaError_t e = cudaSuccess;
  switch (phase) {
    case LBM_PHASE_BEGIN: {
      if (dom->phase_open) return dom->fail(LBM_ERR_STATE, "a phased step is already open");
      if (dom->tape) return dom->fail(LBM_ERR_STATE, "phased steps do not record an adjoint tape");
      for (int b = 1; b < nb; ++b)
        if (dom->blocks[b].far)
          return dom->fail(LBM_ERR_UNSUPPORTED, "phased steps cover refined blocks, not far-field blocks");
      for (int b = 0; b < nb; ++b) {
        lbm_status st = dom->autotune_tiles(b);
        if (st != LBM_OK) return st;
      }
      dom->phase_saved.assign(nb, 0);
      for (int b = 0; b < nb; ++b) dom->phase_saved[b] = dom->blocks[b].cur;
      dom->phase_done.assign(nb, 0);
      dom->phase_ref_done = false;
      dom->phase_open = true;
      return LBM_OK;
    }
    case LBM_PHASE_REFERENCE: {
      if (!dom->phase_open || dom->phase_ref_done)
        return dom->fail(LBM_ERR_STATE, "the reference phase follows LBM_PHASE_BEGIN, once");
      Block& B0 = dom->blocks[0];
      const int nxt = B0.cur ^ 1;
      if (compute) e = launch_step(dom->view(0, B0.cur, nxt), dom->desc.storage, B0.bx, B0.by, s, B0.minb);
      if (e != cudaSuccess) return dom->cuda_fail(e, "collide-stream launch");
      B0.cur = nxt;
      dom->phase_ref_done = true;
      return LBM_OK;
    }
    case LBM_PHASE_BLOCK:
    case LBM_PHASE_POST: {
      if (!dom->phase_open || !dom->phase_ref_done)
        return dom->fail(LBM_ERR_STATE, "block phases follow the reference phase");
      if (block < 1 || block >= nb) return dom->fail(LBM_ERR_INVALID_ARG, "block must be a refined block");
      if (phase == LBM_PHASE_BLOCK) {
        for (int b = 1; b < block; ++b)
          if (dom->phase_done[b] != 2)
            return dom->fail(LBM_ERR_STATE, "blocks are advanced in order, each after the previous one's post-mapping");
        if (dom->phase_done[block] != 0) return dom->fail(LBM_ERR_STATE, "block already advanced");
        Block& B = dom->blocks[block];
        if (compute) {
          e = block_subcycle(dom, block, s);
          if (e != cudaSuccess) return dom->cuda_fail(e, "refined-block sub-cycle");
        } else {
          B.cur = final_level(B, dom->phase_saved[block]);
        }
        dom->phase_done[block] = 1;
      } else {
        if (dom->phase_done[block] != 1) return dom->fail(LBM_ERR_STATE, "post-mapping follows the block's sub-cycle");
        if (compute) {
          const Block& B = dom->blocks[block];
          for (size_t t = 0; t < B.post.size() && e == cudaSuccess; ++t) e = post_map(dom, block, B.post[t], s);
          if (e != cudaSuccess) return dom->cuda_fail(e, "post-mapping");
        }
        dom->phase_done[block] = 2;
      }
      return LBM_OK;
    }
    case LBM_PHASE_END: {
      if (!dom->phase_open || !dom->phase_ref_done)
        return dom->fail(LBM_ERR_STATE, "no phased step to end");
      for (int b = 1; b < nb; ++b)
        if (dom->phase_done[b] != 2) return dom->fail(LBM_ERR_STATE, "every block's phases come before the end");
      dom->phase_open = false;
      ++dom->steps;
      return LBM_OK;
    }
    default:
      return dom->fail(LBM_ERR_INVALID_ARG, "unknown phase");
  }
}

extern "C" lbm_status lbm_mapping_boxes(const lbm_domain* dom_c, int32_t block, int32_t kind,
                                        int32_t other, int32_t* boxes, int32_t* n_boxes) {
  lbm_domain* dom = const_cast<lbm_domain*>(dom_c);
  if (!dom || !boxes || !n_boxes) return LBM_ERR_INVALID_ARG;
  const int nb = (int)dom->blocks.size();
  if (block < 1 || block >= nb || dom->blocks[block].far)
    return dom->fail(LBM_ERR_INVALID_ARG, "block must be a refined block");
  const Block& B = dom->blocks[block];
  *n_boxes = 0;
  if (kind == LBM_BOX_PRIOR_SOURCE) {
    if (other != B.prior.src) return dom->fail(LBM_ERR_INVALID_ARG, "other must be the block's prior-mapping source");
    const Block& P = dom->blocks[other];
    for (int f = 0; f < 6; ++f) {
      int lo[3], hi[3];
      prior_face_box(P, B, f, lo, hi);
      for (int a = 0; a < 3; ++a) { boxes[6 * f + a] = lo[a]; boxes[6 * f + 3 + a] = hi[a]; }
    }
    *n_boxes = 6;
    return LBM_OK;
  }
  if (kind == LBM_BOX_POST_TARGET) {
    if (other < 0 || other >= nb) return dom->fail(LBM_ERR_INVALID_ARG, "other must be a block");
    bool has = false;
    for (const MapTable& t : B.post) has |= t.dst == other && t.n > 0;
    if (!has) return LBM_OK;         // no post-mapping into `other`
    int lo[3], hi[3];
    if (!interior_box(B, dom->blocks[other], lo, hi)) return LBM_OK;
    for (int a = 0; a < 3; ++a) { boxes[a] = lo[a]; boxes[3 + a] = hi[a]; }
    *n_boxes = 1;
    return LBM_OK;
  }
  return dom->fail(LBM_ERR_INVALID_ARG, "unknown box kind");
}

extern "C" size_t lbm_box_bytes(const lbm_domain* dom, int32_t block, const int32_t lo[3],
                                const int32_t hi[3]) {
  if (!dom || !lo || !hi || block < 0 || block >= (int32_t)dom->blocks.size()) return 0;
  if (!valid_box(dom->blocks[block], lo, hi)) return 0;
  return box_nodes(lo, hi) * 31 * sizeof(float);
}

static lbm_status box_transfer(lbm_domain* dom, int32_t block, int32_t level, const int32_t lo[3],
                               const int32_t hi[3], void* buf, int dir, int32_t skip) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (!lo || !hi || !buf) return dom->fail(LBM_ERR_INVALID_ARG, "null box or buffer");
  if (reinterpret_cast<uintptr_t>(buf) % 16 != 0) return dom->fail(LBM_ERR_INVALID_ARG, "buffer must be 16-byte aligned");
  if (block < 0 || block >= (int32_t)dom->blocks.size()) return dom->fail(LBM_ERR_INVALID_ARG, "no such block");
  if (dom->desc.storage != LBM_FP32) return dom->fail(LBM_ERR_UNSUPPORTED, "node boxes need FP32 storage");
  Block& B = dom->blocks[block];
  if (!valid_box(B, lo, hi)) return dom->fail(LBM_ERR_INVALID_ARG, "box outside the block");
  int lv = B.cur;
  if (level == LBM_LEVEL_START) {
    if (!dom->phase_open) return dom->fail(LBM_ERR_STATE, "the start level exists inside a phased step");
    lv = dom->phase_saved[block];
  } else if (level != LBM_LEVEL_CURRENT) {
    return dom->fail(LBM_ERR_INVALID_ARG, "level must be LBM_LEVEL_START or LBM_LEVEL_CURRENT");
  }
  const size_t nb = box_nodes(lo, hi);
  const int3 l3 = make_int3(lo[0], lo[1], lo[2]);
  const int3 d3 = make_int3(hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1);
  const size_t g = (nb + 255) / 256;
  const int grid = (int)(g < 4096 ? g : 4096);
  Level& L = B.lv[lv];
  k_box<<<grid, 256, 0, dom->stream>>>(static_cast<float*>(L.f), L.u, L.c, B.flags, B.nx, B.ny,
                                       B.N, l3, d3, nb, static_cast<float*>(buf), dir, skip);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dom->cuda_fail(e, "node box copy");
  return LBM_OK;
}

extern "C" lbm_status lbm_pack_box(lbm_domain* dom, int32_t block, int32_t level,
                                   const int32_t lo[3], const int32_t hi[3], void* dev_buf) {
  return box_transfer(dom, block, level, lo, hi, dev_buf, 0, 0);
}

extern "C" lbm_status lbm_unpack_box(lbm_domain* dom, int32_t block, int32_t level,
                                     const int32_t lo[3], const int32_t hi[3],
                                     const void* dev_buf, int32_t skip_flags) {
  return box_transfer(dom, block, level, lo, hi, const_cast<void*>(dev_buf), 1,
                      skip_flags & 0xFF);
}
