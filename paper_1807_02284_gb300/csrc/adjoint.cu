// Reverse-mode (adjoint) stepping with checkpointing: gradients of a loss of the final scalar
// (and velocity) field with respect to the initial velocity field.  Not in the paper.
//
// Forward step n -> n+1 at a fluid node x:
//   d_in = pull(D^n);  (rho, u) = moments(d_in);  phi = phi(|grad U^n|(x));
//   D^{n+1}(x) = collide(d_in, u, phi);  U^{n+1}(x) = u;  C^{n+1}(x) = trilinear(C^n, x - u).
// Reverse step, given the adjoints (Lam, Ups, Gam) of (D^{n+1}, U^{n+1}, C^{n+1}):
//   pass A (per fluid node x): recompute the forward at x, then the exact transpose of every
//     stage; the population adjoints go to the pull sources (the pull, with bounce-back, reads
//     every fluid slot exactly once, so these stores never collide), and the adjoint of the
//     adaptive factor becomes 9 per-node terms mu_ab = dL/d(U_a(x+e_b) - U_a(x-e_b));
//   pass B (per node y): Ups^n_a(y) = sum_b mu_ab(y - e_b) - mu_ab(y + e_b) and
//     Gam^n(y) = sum over the nodes x whose departure cell touches y of w_{x->y} Gam^{n+1}(x)
//     (a gather over the 27 neighbours: deterministic, no atomics).
// Initial state: D^0 = f^eq(rho_0, u_0) - w and U^0 = u_0, so
//   dL/du_0 = Ups^0 + (dD^0/du_0)^T Lam^0.
// Inflow nodes: D^{n+1} = f^eq(1, U^n) - w and U^{n+1} = U^n, so their pulled populations get
// a zero adjoint and the adjoint of U^n collects the equilibrium's Jacobian, the copy and the
// scalar's departure-point term; dL/du_0 at an inflow node is then the gradient with respect
// to its (constant) inflow velocity.
// Open faces copy the nearest in-block node, so a slot of a face node can be read by up to 8
// pulls: those slots are zeroed before pass A and accumulated atomically (every other slot
// is read once and stored), pass B's lagged-velocity gather uses the clamped differences
// (a face node's own difference involves itself), and the scalar gather counts a clamped
// repeat of the node once.
// Scope: one block with >= 3 nodes per axis, FP32 storage.
#include <cuda_runtime.h>

#include <vector>

#include "lbm_adjoint.cuh"
#include "lbm_cell.cuh"
#include "runtime.h"

namespace lbm {

struct AdjArgs {
  BlockView fwd;        // D^n, U^n, C^n in (d_out, u_out, c_out unused)
  const float* lam_in;  // Lam^{n+1}: 27 planes (cube order)
  const float* ups_in;  // Ups^{n+1}: 3 planes
  const float* gam_in;  // Gam^{n+1}
  const float* u_next;  // U^{n+1}: 3 planes (scalar gather)
  float* lam_out;       // Lam^n
  float* ups_out;       // Ups^n
  float* gam_out;       // Gam^n
  float* mu;            // 9 planes: adjoint of the velocity differences of the gradient norm
};

// Adjoint of the scalar step with respect to the departure velocity: C^{n+1}(x) is the
// trilinear interpolant of C^n at x - u, so ub -= gam * d(interpolant)/d(fraction) per axis
// (the fraction grows with the displacement -u).  The derivative is 0 where the sample does
// not move with u: a displacement clamped at one node, or a departure point below an open
// face's first node (the forward pins the sample to that node; at the upper face both
// corners already coincide).
__device__ __forceinline__ void scalar_u_vjp(const BlockView& v, int x, int y, int z, float ux,
                                             float uy, float uz, float gam, float (&ub)[3]) {
  if (gam == 0.0f) return;
  const ScalarCell sc = scalar_corners<uint32_t>(v, x, y, z, ux, uy, uz);
  const float tx = sc.tx, ty = sc.ty, tz = sc.tz;
  const float dtx = (1 - ty) * (1 - tz) * (sc.c[1] - sc.c[0]) + ty * (1 - tz) * (sc.c[3] - sc.c[2]) +
                    (1 - ty) * tz * (sc.c[5] - sc.c[4]) + ty * tz * (sc.c[7] - sc.c[6]);
  const float dty = (1 - tx) * (1 - tz) * (sc.c[2] - sc.c[0]) + tx * (1 - tz) * (sc.c[3] - sc.c[1]) +
                    (1 - tx) * tz * (sc.c[6] - sc.c[4]) + tx * tz * (sc.c[7] - sc.c[5]);
  const float dtz = (1 - tx) * (1 - ty) * (sc.c[4] - sc.c[0]) + tx * (1 - ty) * (sc.c[5] - sc.c[1]) +
                    (1 - tx) * ty * (sc.c[6] - sc.c[2]) + tx * ty * (sc.c[7] - sc.c[3]);
  const bool lx = !v.per[0] && x == 0 && ux > 0.0f;
  const bool ly = !v.per[1] && y == 0 && uy > 0.0f;
  const bool lz = !v.per[2] && z == 0 && uz > 0.0f;
  if (fabsf(ux) < 1.0f && !lx) ub[0] -= gam * dtx;
  if (fabsf(uy) < 1.0f && !ly) ub[1] -= gam * dty;
  if (fabsf(uz) < 1.0f && !lz) ub[2] -= gam * dtz;
}

// Which of the candidate source positions (x-1, x, x+1 per axis, after wrapping or clamping)
// lie on an open face, as bits 3a + o + 1 (axis a, offset o).  A slot of a node on an open
// face can be read by more than one pull (the face copies its nearest in-block node), so its
// adjoint is accumulated there; every other slot is read by exactly one pull and stored.
using FaceMask = uint32_t;

template <bool OPEN>
__device__ __forceinline__ FaceMask face_mask(const BlockView& v, int x, int y, int z) {
  if constexpr (!OPEN) return 0u;
  FaceMask f = 0u;
  const int c[3] = {x, y, z}, nn[3] = {v.nx, v.ny, v.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int o = -1; o <= 1; ++o) {
      const int j = nbr(c[a], o, nn[a], v.per[a]);
      if (!v.per[a] && (j == 0 || j == nn[a] - 1)) f |= 1u << (3 * a + o + 1);
    }
  return f;
}

template <bool OPEN, int K = 0>
__device__ __forceinline__ void push_all(const float (&A)[27], float* __restrict__ lam,
                                         uint32_t N, const Nbr<uint32_t>& n, uint32_t idx,
                                         const uint8_t* __restrict__ flags, bool near,
                                         FaceMask fm) {
  if constexpr (K < 27) {
    constexpr int cx = cxk(K), cy = cyk(K), cz = czk(K);
    const uint32_t src = pull_src<K>(n);
    uint32_t slot = (uint32_t)K * N + src;
    const bool bb = K != 13 && near && (__ldg(flags + src) & F_SOLID);
    if (bb) slot = (uint32_t)(26 - K) * N + idx;
    if constexpr (OPEN) {
      constexpr FaceMask own = (1u << 1) | (1u << 4) | (1u << 7);
      constexpr FaceMask src_bits = (1u << (1 - cx)) | (1u << (4 - cy)) | (1u << (7 - cz));
      const bool face = (fm & (bb ? own : src_bits)) != 0u;
      if (face) atomicAdd(lam + slot, A[K]);
      else lam[slot] = A[K];
    } else {
      lam[slot] = A[K];
    }
    push_all<OPEN, K + 1>(A, lam, N, n, idx, flags, near, fm);
  }
}

// Zeroes the adjoint slots of the nodes on open faces before pass A accumulates into them.
__global__ void k_zero_face_slots(float* __restrict__ lam, int nx, int ny, int nz, int px,
                                  int py, int pz) {
  const size_t N = (size_t)nx * ny * nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((size_t)nx * ny));
    const bool face = (!px && (x == 0 || x == nx - 1)) || (!py && (y == 0 || y == ny - 1)) ||
                      (!pz && (z == 0 || z == nz - 1));
    if (!face) continue;
#pragma unroll
    for (int k = 0; k < 27; ++k) lam[(size_t)k * N + idx] = 0.0f;
  }
}

// MINB: CTAs per SM the register allocation is bounded for (3: no spills; 4: some spills,
// more warps in flight); the faster one is chosen at run time.
// OPEN: some face of the block is open (face slots accumulate; see FaceMask).
template <int MINB, bool OPEN>
__global__ void __launch_bounds__(128, MINB) k_adj_a(AdjArgs a) {
  const BlockView& v = a.fwd;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= v.nx) return;
  const uint32_t N = (uint32_t)v.N;
  const Nbr<uint32_t> n = neighbours<uint32_t>(v, x, y, z);
  const uint32_t idx = n.p0 + n.r0 + n.x0;
  const uint8_t fl = v.flags[idx];
  if (fl & F_SOLID) {
#pragma unroll
    for (int i = 0; i < 9; ++i) a.mu[(uint32_t)i * N + idx] = 0.0f;
    return;
  }
  if (fl & F_INFLOW) {
    // D^{n+1} = f^eq(1, U^n) - w, U^{n+1} = U^n, C^{n+1} sampled at x - U^n: the pulled
    // populations are unused (their slots get a zero adjoint) and every adjoint goes to U^n,
    // which pass B completes with the lagged-gradient terms of the neighbours
    const float u[3] = {v.u_in[idx], v.u_in[N + idx], v.u_in[2 * N + idx]};
    float ub[3] = {a.ups_in[idx], a.ups_in[N + idx], a.ups_in[2 * N + idx]};
    if (!(fl & F_SCALAR_SRC)) scalar_u_vjp(v, x, y, z, u[0], u[1], u[2], a.gam_in[idx], ub);
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      const float c[3] = {(float)cxk(k), (float)cyk(k), (float)czk(k)};
      const float cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
      const float l = a.lam_in[(uint32_t)k * N + idx] * wk(k);
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2) ub[a2] = fmaf(l, 3.0f * c[a2] + 9.0f * cu * c[a2] - 3.0f * u[a2], ub[a2]);
    }
    a.ups_out[idx] = ub[0];
    a.ups_out[N + idx] = ub[1];
    a.ups_out[2 * N + idx] = ub[2];
    float Z[27];
#pragma unroll
    for (int k = 0; k < 27; ++k) Z[k] = 0.0f;
    push_all<OPEN>(Z, a.lam_out, N, n, idx, v.flags, (fl & F_NEAR_SOLID) != 0, face_mask<OPEN>(v, x, y, z));
#pragma unroll
    for (int i = 0; i < 9; ++i) a.mu[(uint32_t)i * N + idx] = 0.0f;
    return;
  }
  const float* __restrict__ din = static_cast<const float*>(v.d_in);

  // ---- forward recompute up to the central moments
  float K[27];
  pull_all<float, uint32_t>(K, din, N, n);
  const bool near = (fl & F_NEAR_SOLID) != 0;
  if (near) bounce_back<float, uint32_t>(K, din, N, v.flags, n, idx);
  raw_moments(K);
  const float drho = K[kap(0, 0, 0)];
  const float inv = __frcp_rn(1.0f + drho);
  const float ux = K[kap(1, 0, 0)] * inv, uy = K[kap(0, 1, 0)] * inv, uz = K[kap(0, 0, 1)] * inv;
  float diff[9];
  float g = 0.0f;
  if (v.rp.adaptive) {
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* Uc = v.u_in + (uint32_t)c * N;
      diff[3 * c + 0] = __ldg(Uc + (n.p0 + n.r0 + n.xp)) - __ldg(Uc + (n.p0 + n.r0 + n.xm));
      diff[3 * c + 1] = __ldg(Uc + (n.p0 + n.rp + n.x0)) - __ldg(Uc + (n.p0 + n.rm + n.x0));
      diff[3 * c + 2] = __ldg(Uc + (n.pp + n.r0 + n.x0)) - __ldg(Uc + (n.pm + n.r0 + n.x0));
      s = fmaf(diff[3 * c + 0], diff[3 * c + 0],
               fmaf(diff[3 * c + 1], diff[3 * c + 1], fmaf(diff[3 * c + 2], diff[3 * c + 2], s)));
    }
    g = 0.5f * sqrtf(s);
  }
  const Keep kf = keep_factors(v.rp, g);
  shift_axis<1>(K, ux);
  shift_axis<3>(K, uy);
  shift_axis<9>(K, uz);                  // K = central moments before relaxation

  // ---- adjoint of the stored velocity and of the scalar step
  float ub[3];
  ub[0] = a.ups_in[idx];
  ub[1] = a.ups_in[N + idx];
  ub[2] = a.ups_in[2 * N + idx];
  if (!(fl & F_SCALAR_SRC)) scalar_u_vjp(v, x, y, z, ux, uy, uz, a.gam_in[idx], ub);

  // ---- adjoint of the collision
  float A[27];
#pragma unroll
  for (int k = 0; k < 27; ++k) A[k] = a.lam_in[(uint32_t)k * N + idx];
  float T[27];
  // the inverse sweeps ran z, y, x: undo x first; its input is inv_y(inv_z(relaxed))
#pragma unroll
  for (int k = 0; k < 27; ++k) T[k] = K[k];
  relax_to_equilibrium(T, drho, ux, uy, uz, kf);
  inv_axis<9>(T, uz);
  inv_axis<3>(T, uy);
  inv_axis_vjp<1>(T, A, ux, ub[0]);
#pragma unroll
  for (int k = 0; k < 27; ++k) T[k] = K[k];
  relax_to_equilibrium(T, drho, ux, uy, uz, kf);
  inv_axis<9>(T, uz);
  inv_axis_vjp<3>(T, A, uy, ub[1]);
#pragma unroll
  for (int k = 0; k < 27; ++k) T[k] = K[k];
  relax_to_equilibrium(T, drho, ux, uy, uz, kf);
  inv_axis_vjp<9>(T, A, uz, ub[2]);
  float bar[4] = {0.f, 0.f, 0.f, 0.f};     // d/d(rho - 1), d/du
  float kbar[4] = {0.f, 0.f, 0.f, 0.f};    // d/d(keep factor) of the high-order groups
  relax_vjp(K, A, drho, ux, uy, uz, kf, bar, kbar);
  ub[0] += bar[1];
  ub[1] += bar[2];
  ub[2] += bar[3];
  float drhob = bar[0];
  // the shifts ran x, y, z: undo z first; its input is unshift_z(K)
  unshift_axis<9>(K, uz);
  shift_axis_vjp<9>(K, A, uz, ub[2]);
  unshift_axis<3>(K, uy);
  shift_axis_vjp<3>(K, A, uy, ub[1]);
  unshift_axis<1>(K, ux);
  shift_axis_vjp<1>(K, A, ux, ub[0]);
  // u = j / rho with rho = 1 + r_000, j = (r_100, r_010, r_001)
  drhob -= (ub[0] * ux + ub[1] * uy + ub[2] * uz) * inv;
  A[kap(0, 0, 0)] += drhob;
  A[kap(1, 0, 0)] += ub[0] * inv;
  A[kap(0, 1, 0)] += ub[1] * inv;
  A[kap(0, 0, 1)] += ub[2] * inv;
  raw_axis_vjp<9>(A);
  raw_axis_vjp<3>(A);
  raw_axis_vjp<1>(A);                    // A = adjoint of the pulled populations
  push_all<OPEN>(A, a.lam_out, N, n, idx, v.flags, near, face_mask<OPEN>(v, x, y, z));

  // ---- adjoint of the adaptive factor: K_g = 1 - 1/(phi nu3_g + 1/2)
  float mu_scale = 0.0f;
  if (v.rp.adaptive && g > 0.0f && g * v.rp.inv_gmax < 1.0f) {
    float phib = 0.0f;
#pragma unroll
    for (int gi = 0; gi < 4; ++gi) {
      const float S = 1.0f - kf.g[gi];
      phib = fmaf(kbar[gi], v.rp.nuh3[gi] * S * S, phib);
    }
    const float gb = phib * v.rp.a * v.rp.inv_gmax;   // phi = a g / g_max + b below the clamp
    mu_scale = gb * 0.25f / g;                        // dg/d(diff) = diff / (4 g)
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) a.mu[(uint32_t)i * N + idx] = v.rp.adaptive ? mu_scale * diff[i] : 0.0f;
}

static void launch_pass_a(const AdjArgs& a, int minb, bool open, dim3 grd, dim3 blk, cudaStream_t s) {
  if (open) {
    if (minb == 4) k_adj_a<4, true><<<grd, blk, 0, s>>>(a);
    else k_adj_a<3, true><<<grd, blk, 0, s>>>(a);
  } else {
    if (minb == 4) k_adj_a<4, false><<<grd, blk, 0, s>>>(a);
    else k_adj_a<3, false><<<grd, blk, 0, s>>>(a);
  }
}

__global__ void __launch_bounds__(128) k_adj_b(AdjArgs a) {
  const BlockView& v = a.fwd;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= v.nx) return;
  const uint32_t N = (uint32_t)v.N;
  const Nbr<uint32_t> n = neighbours<uint32_t>(v, x, y, z);
  const uint32_t idx = n.p0 + n.r0 + n.x0;
  // lagged-velocity adjoint (inflow nodes add it to what pass A left there)
  const bool inflow = (v.flags[idx] & (F_INFLOW | F_SOLID)) == F_INFLOW;
  // node q's difference along axis b is U(q+e_b) - U(q-e_b) with the indices wrapped or
  // clamped: this node receives +mu_b(q) from q = this - e_b and -mu_b(q) from q = this + e_b
  // when those nodes exist, and on an open face also its own +mu_b (top: its + neighbour is
  // itself) or -mu_b (bottom: its - neighbour is itself)
  const int cc[3] = {x, y, z}, nn[3] = {v.nx, v.ny, v.nz};
  float wm[3], wp[3], ws[3];            // weights of mu(this - e_b), mu(this + e_b), mu(this)
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const bool per = v.per[b] != 0;
    wm[b] = (per || cc[b] > 0) ? 1.0f : 0.0f;
    wp[b] = (per || cc[b] < nn[b] - 1) ? -1.0f : 0.0f;
    ws[b] = per ? 0.0f : (cc[b] == nn[b] - 1 ? 1.0f : 0.0f) - (cc[b] == 0 ? 1.0f : 0.0f);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* m0 = a.mu + (uint32_t)(3 * c + 0) * N;
    const float* m1 = a.mu + (uint32_t)(3 * c + 1) * N;
    const float* m2 = a.mu + (uint32_t)(3 * c + 2) * N;
    float s = wm[0] * __ldg(m0 + (n.p0 + n.r0 + n.xm)) + wp[0] * __ldg(m0 + (n.p0 + n.r0 + n.xp)) +
              wm[1] * __ldg(m1 + (n.p0 + n.rm + n.x0)) + wp[1] * __ldg(m1 + (n.p0 + n.rp + n.x0)) +
              wm[2] * __ldg(m2 + (n.pm + n.r0 + n.x0)) + wp[2] * __ldg(m2 + (n.pp + n.r0 + n.x0));
    s = fmaf(ws[0], __ldg(m0 + idx), fmaf(ws[1], __ldg(m1 + idx), fmaf(ws[2], __ldg(m2 + idx), s)));
    a.ups_out[(uint32_t)c * N + idx] = inflow ? a.ups_out[(uint32_t)c * N + idx] + s : s;
  }
  // scalar adjoint: gather from the neighbours whose departure cell contains this node
  const uint32_t xs[3] = {n.xm, n.x0, n.xp};
  const uint32_t rs[3] = {n.rm, n.r0, n.rp};
  const uint32_t ps[3] = {n.pm, n.p0, n.pp};
  const int cx[3] = {(int)n.xm, x, (int)n.xp};
  const int cy[3] = {(int)(n.rm / (uint32_t)v.nx), y, (int)(n.rp / (uint32_t)v.nx)};
  const int cz[3] = {(int)(n.pm / ((uint32_t)v.nx * v.ny)), z, (int)(n.pp / ((uint32_t)v.nx * v.ny))};
  float gam = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        // a clamped neighbour index repeats the node itself: count every node once
        if ((dx == 0 && xs[0] == xs[1]) || (dx == 2 && xs[2] == xs[1]) ||
            (dy == 0 && rs[0] == rs[1]) || (dy == 2 && rs[2] == rs[1]) ||
            (dz == 0 && ps[0] == ps[1]) || (dz == 2 && ps[2] == ps[1]))
          continue;
        const uint32_t j = ps[dz] + rs[dy] + xs[dx];
        if (__ldg(v.flags + j) & (F_SOLID | F_SCALAR_SRC)) continue;
        const float G = __ldg(a.gam_in + j);
        if (G == 0.0f) continue;
        const Axis1 ax = sl_axis(cx[dx], __ldg(a.u_next + j), v.nx, v.per[0]);
        const Axis1 ay = sl_axis(cy[dy], __ldg(a.u_next + N + j), v.ny, v.per[1]);
        const Axis1 az = sl_axis(cz[dz], __ldg(a.u_next + 2 * N + j), v.nz, v.per[2]);
        const float wx = (ax.i0 == x ? 1.0f - ax.t : 0.0f) + (ax.i1 == x ? ax.t : 0.0f);
        const float wy = (ay.i0 == y ? 1.0f - ay.t : 0.0f) + (ay.i1 == y ? ay.t : 0.0f);
        const float wz = (az.i0 == z ? 1.0f - az.t : 0.0f) + (az.i1 == z ? az.t : 0.0f);
        gam = fmaf(wx * wy * wz, G, gam);
      }
  a.gam_out[idx] = gam;
}

// dL/du_0 = Ups^0 + (dD^0/du_0)^T Lam^0 with D^0_k = w_k (drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)).
__global__ void k_adj_init(const float* __restrict__ d0, const float* __restrict__ u0,
                           const uint8_t* __restrict__ flags, const float* __restrict__ lam,
                           const float* __restrict__ ups, float* __restrict__ out, uint32_t N) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    if (flags[idx] & F_SOLID) {
      out[idx] = out[N + idx] = out[2 * N + idx] = 0.0f;
      continue;
    }
    float drho = 0.0f;
#pragma unroll
    for (int k = 0; k < 27; ++k) drho += d0[(uint32_t)k * N + idx];
    const float rho = 1.0f + drho;
    const float u[3] = {u0[idx], u0[N + idx], u0[2 * N + idx]};
    float gsum[3] = {ups[idx], ups[N + idx], ups[2 * N + idx]};
#pragma unroll
    for (int k = 0; k < 27; ++k) {
      const float c[3] = {(float)cxk(k), (float)cyk(k), (float)czk(k)};
      const float cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
      const float l = lam[(uint32_t)k * N + idx] * wk(k) * rho;
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2) gsum[a2] = fmaf(l, 3.0f * c[a2] + 9.0f * cu * c[a2] - 3.0f * u[a2], gsum[a2]);
    }
    out[idx] = gsum[0];
    out[N + idx] = gsum[1];
    out[2 * N + idx] = gsum[2];
  }
}

// The inflow velocity of a node is its stored velocity, carried unchanged from step to step
// and set with u_0, so the gradient with respect to it is dL/du_0 at inflow nodes.
__global__ void k_inflow_grad(const float* __restrict__ du0, const uint8_t* __restrict__ flags,
                              float* __restrict__ out, uint32_t N) {
  for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const bool in = (flags[idx] & (F_INFLOW | F_SOLID)) == F_INFLOW;
    out[idx] = in ? du0[idx] : 0.0f;
    out[N + idx] = in ? du0[N + idx] : 0.0f;
    out[2 * N + idx] = in ? du0[2 * N + idx] : 0.0f;
  }
}

struct TapeState {
  int every = 0;
  int pass_a_minb = 0;        // chosen launch bound of pass A (0: not yet timed)
  std::vector<Level> ckpt;    // states at steps 0, every, 2 every, ...
  std::vector<Level> seg;     // recompute levels 1..every of one segment
  float* lam[2] = {nullptr, nullptr};
  float* ups[2] = {nullptr, nullptr};
  float* gam[2] = {nullptr, nullptr};
  float* mu = nullptr;
};

}  // namespace lbm

using namespace lbm;

static void free_level(lbm_domain* dom, Level& L) {
  dom->dev_free(L.f);
  dom->dev_free(L.u);
  dom->dev_free(L.c);
  L = Level();
}

void release_tape(lbm_domain* dom) {
  TapeState* t = dom->tape;
  if (!t) return;
  for (Level& L : t->ckpt) free_level(dom, L);
  for (Level& L : t->seg) free_level(dom, L);
  for (int i = 0; i < 2; ++i) {
    dom->dev_free(t->lam[i]);
    dom->dev_free(t->ups[i]);
    dom->dev_free(t->gam[i]);
  }
  dom->dev_free(t->mu);
  delete t;
  dom->tape = nullptr;
}

static bool alloc_level(lbm_domain* dom, size_t N, Level& L) {
  L.f = dom->dev_alloc(N * 27 * sizeof(float));
  L.u = static_cast<float*>(dom->dev_alloc(N * 3 * sizeof(float)));
  L.c = static_cast<float*>(dom->dev_alloc(N * sizeof(float)));
  return L.f && L.u && L.c;
}

static BlockView view_of(lbm_domain* dom, const Level& from, const Level& to) {
  BlockView v = dom->view(0, 0, 0);
  v.d_in = from.f;
  v.u_in = from.u;
  v.c_in = from.c;
  v.d_out = to.f;
  v.u_out = to.u;
  v.c_out = to.c;
  return v;
}

// Records a checkpoint of the current state every `every` steps since the last init.
lbm_status tape_before_step(lbm_domain* dom) {
  TapeState* t = dom->tape;
  if (!t) return LBM_OK;
  if (dom->steps % t->every != 0) return LBM_OK;
  const size_t i = (size_t)(dom->steps / t->every);
  Block& B = dom->blocks[0];
  while (t->ckpt.size() <= i) {
    Level L;
    if (!alloc_level(dom, B.N, L)) {
      free_level(dom, L);
      return dom->fail(LBM_ERR_OOM, "checkpoint allocation failed");
    }
    t->ckpt.push_back(L);
  }
  const Level& S = B.lv[B.cur];
  Level& D = t->ckpt[i];
  cudaError_t e = cudaMemcpyAsync(D.f, S.f, B.N * 27 * sizeof(float), cudaMemcpyDeviceToDevice, dom->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D.u, S.u, B.N * 3 * sizeof(float), cudaMemcpyDeviceToDevice, dom->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D.c, S.c, B.N * sizeof(float), cudaMemcpyDeviceToDevice, dom->stream);
  if (e != cudaSuccess) return dom->cuda_fail(e, "checkpoint copy");
  return LBM_OK;
}

static lbm_status adjoint_supported(lbm_domain* dom) {
  if (dom->blocks.size() != 1) return dom->fail(LBM_ERR_UNSUPPORTED, "the adjoint covers single-block domains");
  if (dom->desc.storage != LBM_FP32) return dom->fail(LBM_ERR_UNSUPPORTED, "the adjoint needs FP32 storage");
  if (dom->desc.grad_mode != LBM_GRAD_LAGGED)
    return dom->fail(LBM_ERR_UNSUPPORTED, "the adjoint covers the lagged-gradient relaxation");
  const Block& B = dom->blocks[0];
  if (B.nx < 3 || B.ny < 3 || B.nz < 3) return dom->fail(LBM_ERR_UNSUPPORTED, "the adjoint needs >= 3 nodes per axis");
  if (27ull * B.N >= 0xFFFFFFFFull) return dom->fail(LBM_ERR_UNSUPPORTED, "block too large for the adjoint");
  return LBM_OK;
}

extern "C" lbm_status lbm_set_tape(lbm_domain* dom, int32_t every) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  if (every < 0) return dom->fail(LBM_ERR_INVALID_ARG, "checkpoint_every must be >= 0");
  release_tape(dom);
  if (every == 0) return LBM_OK;
  if (dom->steps != 0)
    return dom->fail(LBM_ERR_STATE, "the tape must be enabled right after lbm_init_macro");
  lbm_status st = adjoint_supported(dom);
  if (st != LBM_OK) return st;
  dom->tape = new TapeState();
  dom->tape->every = every;
  dom->invalidate_graphs();
  return LBM_OK;
}

extern "C" lbm_status lbm_adjoint_step(lbm_domain* dom, int32_t n_steps, const float* dL_dc,
                                       const float* dL_du, float* dL_du0, float* dL_dinflow) {
  if (!dom) return LBM_ERR_INVALID_ARG;
  cudaSetDevice(dom->desc.device);
  TapeState* t = dom->tape;
  if (!t) return dom->fail(LBM_ERR_STATE, "no tape: call lbm_set_tape after lbm_init_macro");
  if (n_steps < 0 || n_steps != dom->steps)
    return dom->fail(LBM_ERR_INVALID_ARG, "n_steps must equal the steps recorded since lbm_init_macro");
  if (!dL_dc || !dL_du0) return dom->fail(LBM_ERR_INVALID_ARG, "dL_dscalar_final and dL_du0 are required");
  Block& B = dom->blocks[0];
  const size_t N = B.N;
  cudaStream_t s = dom->stream;
  // buffers
  for (int i = 0; i < 2; ++i) {
    if (!t->lam[i]) t->lam[i] = static_cast<float*>(dom->dev_alloc(N * 27 * sizeof(float)));
    if (!t->ups[i]) t->ups[i] = static_cast<float*>(dom->dev_alloc(N * 3 * sizeof(float)));
    if (!t->gam[i]) t->gam[i] = static_cast<float*>(dom->dev_alloc(N * sizeof(float)));
    if (!t->lam[i] || !t->ups[i] || !t->gam[i]) return dom->fail(LBM_ERR_OOM, "adjoint buffers");
  }
  if (!t->mu) t->mu = static_cast<float*>(dom->dev_alloc(N * 9 * sizeof(float)));
  if (!t->mu) return dom->fail(LBM_ERR_OOM, "adjoint buffers");
  const int seg_len = std::min(t->every, std::max(1, n_steps));
  while ((int)t->seg.size() < seg_len) {
    Level L;
    if (!alloc_level(dom, N, L)) {
      free_level(dom, L);
      return dom->fail(LBM_ERR_OOM, "recompute levels");
    }
    t->seg.push_back(L);
  }
  if (t->ckpt.empty()) {  // no step was taken: the checkpoint of step 0 is the current state
    lbm_status st = tape_before_step(dom);
    if (st != LBM_OK) return st;
  }
  int c = 0;
  cudaError_t e = cudaMemsetAsync(t->lam[0], 0, N * 27 * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->lam[1], 0, N * 27 * sizeof(float), s);
  if (e == cudaSuccess) {
    if (dL_du) e = cudaMemcpyAsync(t->ups[0], dL_du, N * 3 * sizeof(float), cudaMemcpyDeviceToDevice, s);
    else e = cudaMemsetAsync(t->ups[0], 0, N * 3 * sizeof(float), s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(t->gam[0], dL_dc, N * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return dom->cuda_fail(e, "adjoint initialisation");

  const int n_seg = (n_steps + t->every - 1) / t->every;
  const bool open_faces = !dom->desc.periodic[0] || !dom->desc.periodic[1] || !dom->desc.periodic[2];
  const int zgrid = (int)std::min<size_t>((N + 255) / 256, 16384);
  const dim3 blk(128, 1, 1);
  const dim3 grd((B.nx + 127) / 128, B.ny, B.nz);
  for (int sg = n_seg - 1; sg >= 0; --sg) {
    const int s0 = sg * t->every;
    const int len = std::min(t->every, n_steps - s0);
    // recompute the segment's states 1..len from its checkpoint
    auto level = [&](int i) -> const Level& { return i == 0 ? t->ckpt[sg] : t->seg[i - 1]; };
    for (int i = 0; i < len; ++i) {
      e = launch_step(view_of(dom, level(i), level(i + 1)), ST_FP32, B.bx, B.by, s, B.minb);
      if (e != cudaSuccess) return dom->cuda_fail(e, "adjoint recompute");
    }
    for (int i = len - 1; i >= 0; --i) {
      AdjArgs a;
      a.fwd = view_of(dom, level(i), level(i));
      a.lam_in = t->lam[c];
      a.ups_in = t->ups[c];
      a.gam_in = t->gam[c];
      a.u_next = level(i + 1).u;
      a.lam_out = t->lam[c ^ 1];
      a.ups_out = t->ups[c ^ 1];
      a.gam_out = t->gam[c ^ 1];
      a.mu = t->mu;
      if (t->pass_a_minb == 0) {
        // time both register bounds on this step's inputs (pass A only writes lam_out, mu and
        // the inflow nodes' ups_out, which the launches below rewrite), keep the faster
        cudaEvent_t e0, e1, e2;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventCreate(&e2);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2; ++r) launch_pass_a(a, 3, open_faces, grd, blk, s);
        cudaEventRecord(e1, s);
        for (int r = 0; r < 2; ++r) launch_pass_a(a, 4, open_faces, grd, blk, s);
        cudaEventRecord(e2, s);
        e = cudaEventSynchronize(e2);
        float m3 = 0.f, m4 = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&m3, e0, e1);
        if (e == cudaSuccess) cudaEventElapsedTime(&m4, e1, e2);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        if (e != cudaSuccess) return dom->cuda_fail(e, "adjoint tuning");
        t->pass_a_minb = m4 < m3 ? 4 : 3;
      }
      if (open_faces)   // open-face slots accumulate; the tuning launches above also wrote them
        k_zero_face_slots<<<zgrid, 256, 0, s>>>(a.lam_out, B.nx, B.ny, B.nz, dom->desc.periodic[0],
                                                dom->desc.periodic[1], dom->desc.periodic[2]);
      launch_pass_a(a, t->pass_a_minb, open_faces, grd, blk, s);
      k_adj_b<<<grd, blk, 0, s>>>(a);
      e = cudaGetLastError();
      if (e != cudaSuccess) return dom->cuda_fail(e, "adjoint step");
      c ^= 1;
    }
  }
  const int g = (int)std::min<size_t>((N + 255) / 256, 16384);
  k_adj_init<<<g, 256, 0, s>>>(static_cast<const float*>(t->ckpt[0].f), t->ckpt[0].u, B.flags,
                               t->lam[c], t->ups[c], dL_du0, (uint32_t)N);
  if (dL_dinflow) k_inflow_grad<<<g, 256, 0, s>>>(dL_du0, B.flags, dL_dinflow, (uint32_t)N);
  e = cudaGetLastError();
  if (e != cudaSuccess) return dom->cuda_fail(e, "initial-state adjoint");
  dom->post_error_probe();
  return LBM_OK;
}
