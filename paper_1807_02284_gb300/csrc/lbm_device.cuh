// Device-side building blocks of the D3Q27 central-moment (CMR) collide-and-stream update.
//
// Populations live in "cube order": k = (cx+1) + 3 (cy+1) + 9 (cz+1), so the opposite of k
// is 26 - k and the three velocities of a line along one axis are three consecutive (or
// 3-/9-strided) slots.  Storage holds the shifted population d_k = f_k - w_k (f_k minus the
// rest-state weight), which keeps the stored magnitudes small; the FP16 mode stores the same
// quantity in half precision.
//
// The collision (Sec. 3.1, Eq. 2: Omega = -T S (m - m^eq)) is evaluated in the factorised
// form  f~ = f^eq + P(u)^{-1} (I - S) P(u) (f - f^eq),  where P(u) maps populations to the
// raw central moments kappa_abc = sum_i f_i (c_ix-u_x)^a (c_iy-u_y)^b (c_iz-u_z)^c by three
// per-axis sweeps over 3-point lines.  The paper's moments m_j are fixed linear combinations
// of the kappa_abc (the Appendix basis), and S is constant inside each combination group, so
// relaxing kappa with the per-group rates is the paper's m-space relaxation; the only mixing
// group is the second-order diagonal (m_7 = k200-k020, m_8 = k200-k002 relax with the shear
// rate, the trace m_9 with the high-order rate of group 9..16).  f^eq is the second-order
// polynomial equilibrium, which equals T m^eq(rho,u) for the Appendix m^eq.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

// Cell flags (bits 0..3 are user-visible, bit 4 is derived by the library).
enum : uint8_t {
  F_SOLID = 1, F_INFLOW = 2, F_SCALAR_SRC = 4, F_GHOST = 8, F_NEAR_SOLID = 16
};

__host__ __device__ constexpr int cxk(int k) { return k % 3 - 1; }
__host__ __device__ constexpr int cyk(int k) { return (k / 3) % 3 - 1; }
__host__ __device__ constexpr int czk(int k) { return k / 9 - 1; }
__host__ __device__ constexpr int normk(int k) {
  return (cxk(k) != 0) + (cyk(k) != 0) + (czk(k) != 0);
}
// D3Q27 lattice weights by |c|^2 (rest 8/27, face 2/27, edge 1/54, corner 1/216).
__host__ __device__ constexpr float wk(int k) {
  return normk(k) == 0 ? 8.0f / 27.0f
       : normk(k) == 1 ? 2.0f / 27.0f
       : normk(k) == 2 ? 1.0f / 54.0f
                       : 1.0f / 216.0f;
}
__host__ __device__ constexpr double wkd(int k) {
  return normk(k) == 0 ? 8.0 / 27.0
       : normk(k) == 1 ? 2.0 / 27.0
       : normk(k) == 2 ? 1.0 / 54.0
                       : 1.0 / 216.0;
}

// Storage element conversions.
__device__ __forceinline__ float load_pop(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load_pop(const __half* p) {
  return __half2float(__ldg(reinterpret_cast<const __half*>(p)));
}
__device__ __forceinline__ void store_pop(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void store_pop(__half* p, float v) { *p = __float2half_rn(v); }

// Relaxation "keep" factors 1 - S for the moment groups of the Appendix.
struct Keep {
  float nu;      // moments 4..8 (shear / deviatoric stress), S = 1/(3 nu + 1/2)
  float g[4];    // high-order groups 9..16, 17..22, 23..25, 26
};

struct RelaxParams {
  float s_nu;        // S for moments 4..8
  float nuh3[4];     // 3 * nu'_g for the four high-order groups
  float a, b;        // adaptive model parameters (Sec. 4.1)
  float inv_gmax;    // 1 / g_max
  int adaptive;
};

// Sec. 4.1: S_i = 1/(3 phi nu'_i + 1/2) for i >= 9 with phi = a min(|grad u|/g_max, 1) + b.
__device__ __forceinline__ Keep keep_factors(const RelaxParams& rp, float grad_norm) {
  Keep kf;
  kf.nu = 1.0f - rp.s_nu;
  float phi = 1.0f;
  if (rp.adaptive) phi = rp.a * fminf(grad_norm * rp.inv_gmax, 1.0f) + rp.b;
#pragma unroll
  for (int g = 0; g < 4; ++g) kf.g[g] = 1.0f - 1.0f / (phi * rp.nuh3[g] + 0.5f);
  return kf;
}

// Shifted equilibrium d^eq_k = f^eq_k - w_k = w_k (drho + rho (3 cu + 9/2 cu^2 - 3/2 u.u)).
template <int K>
__device__ __forceinline__ float deq_k(float drho, float rho, float ux, float uy, float uz,
                                       float usq15) {
  const float cu = float(cxk(K)) * ux + float(cyk(K)) * uy + float(czk(K)) * uz;
  return wk(K) * (drho + rho * (cu * (3.0f + 4.5f * cu) - usq15));
}

template <int K0 = 0>
__device__ __forceinline__ void sub_deq(float (&d)[27], float drho, float rho, float ux, float uy,
                                        float uz, float usq15) {
  if constexpr (K0 < 27) {
    d[K0] -= deq_k<K0>(drho, rho, ux, uy, uz, usq15);
    sub_deq<K0 + 1>(d, drho, rho, ux, uy, uz, usq15);
  }
}
template <int K0 = 0>
__device__ __forceinline__ void add_deq(float (&d)[27], float drho, float rho, float ux, float uy,
                                        float uz, float usq15) {
  if constexpr (K0 < 27) {
    d[K0] += deq_k<K0>(drho, rho, ux, uy, uz, usq15);
    add_deq<K0 + 1>(d, drho, rho, ux, uy, uz, usq15);
  }
}

// Forward 3-point central-moment transform of one line (slots s0,s1,s2 = velocity -1,0,+1)
// into orders 0,1,2 about velocity u.
__device__ __forceinline__ void fwd_line(float& s0, float& s1, float& s2, float u) {
  const float k0 = s0 + s1 + s2;
  const float s = s2 - s0;
  const float t = s2 + s0;
  const float k1 = s - u * k0;
  const float k2 = t - u * (s + k1);
  s0 = k0; s1 = k1; s2 = k2;
}
// Exact inverse of fwd_line.
__device__ __forceinline__ void inv_line(float& s0, float& s1, float& s2, float u) {
  const float k0 = s0, k1 = s1, k2 = s2;
  const float r1 = k1 + u * k0;
  const float r2 = k2 + u * (k1 + r1);
  s0 = 0.5f * (r2 - r1);
  s1 = k0 - r2;
  s2 = 0.5f * (r2 + r1);
}

// stride 1: x lines, stride 3: y lines, stride 9: z lines
template <int STRIDE>
__device__ __forceinline__ void fwd_axis(float (&v)[27], float u) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int base = (STRIDE == 1) ? 3 * l : (STRIDE == 3) ? (l % 3) + 9 * (l / 3) : l;
    fwd_line(v[base], v[base + STRIDE], v[base + 2 * STRIDE], u);
  }
}
template <int STRIDE>
__device__ __forceinline__ void inv_axis(float (&v)[27], float u) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int base = (STRIDE == 1) ? 3 * l : (STRIDE == 3) ? (l % 3) + 9 * (l / 3) : l;
    inv_line(v[base], v[base + STRIDE], v[base + 2 * STRIDE], u);
  }
}

// kappa index of orders (a, b, c)
__host__ __device__ constexpr int kap(int a, int b, int c) { return a + 3 * b + 9 * c; }

// Relaxation of non-equilibrium central moments in place (orders are slot indices).
__device__ __forceinline__ void relax(float (&v)[27], const Keep& kf) {
  // second order, off-diagonal (m_4, m_5, m_6)
  v[kap(1, 1, 0)] *= kf.nu;
  v[kap(1, 0, 1)] *= kf.nu;
  v[kap(0, 1, 1)] *= kf.nu;
  // second order, diagonal: deviators m_7, m_8 at the shear rate, trace m_9 at group 9..16
  {
    const float A = v[kap(2, 0, 0)], B = v[kap(0, 2, 0)], Cc = v[kap(0, 0, 2)];
    const float d1 = kf.nu * (A - B);
    const float d2 = kf.nu * (A - Cc);
    const float tr = kf.g[0] * (A + B + Cc);
    const float third = 1.0f / 3.0f;
    v[kap(2, 0, 0)] = third * (tr + d1 + d2);
    v[kap(0, 2, 0)] = third * (tr - 2.0f * d1 + d2);
    v[kap(0, 0, 2)] = third * (tr + d1 - 2.0f * d2);
  }
  // third order (m_10 .. m_16)
  v[kap(1, 2, 0)] *= kf.g[0];
  v[kap(1, 0, 2)] *= kf.g[0];
  v[kap(2, 1, 0)] *= kf.g[0];
  v[kap(0, 1, 2)] *= kf.g[0];
  v[kap(2, 0, 1)] *= kf.g[0];
  v[kap(0, 2, 1)] *= kf.g[0];
  v[kap(1, 1, 1)] *= kf.g[0];
  // fourth order (m_17 .. m_22)
  v[kap(2, 2, 0)] *= kf.g[1];
  v[kap(2, 0, 2)] *= kf.g[1];
  v[kap(0, 2, 2)] *= kf.g[1];
  v[kap(2, 1, 1)] *= kf.g[1];
  v[kap(1, 2, 1)] *= kf.g[1];
  v[kap(1, 1, 2)] *= kf.g[1];
  // fifth order (m_23 .. m_25)
  v[kap(1, 2, 2)] *= kf.g[2];
  v[kap(2, 1, 2)] *= kf.g[2];
  v[kap(2, 2, 1)] *= kf.g[2];
  // sixth order (m_26)
  v[kap(2, 2, 2)] *= kf.g[3];
  // orders 0 and 1 (S_0..3 = 0) are left as they are
}

// Macroscopic moments of shifted populations: drho = rho - 1, j = sum c d.
__device__ __forceinline__ void macros(const float (&d)[27], float& drho, float& jx, float& jy,
                                       float& jz) {
  float s = 0.f, x = 0.f, y = 0.f, z = 0.f;
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    s += d[k];
    if (cxk(k) > 0) x += d[k]; else if (cxk(k) < 0) x -= d[k];
    if (cyk(k) > 0) y += d[k]; else if (cyk(k) < 0) y -= d[k];
    if (czk(k) > 0) z += d[k]; else if (czk(k) < 0) z -= d[k];
  }
  drho = s; jx = x; jy = y; jz = z;
}

// Full CMR collision of shifted populations, in place: d -> d~.
__device__ __forceinline__ void collide(float (&d)[27], float drho, float ux, float uy, float uz,
                                        const Keep& kf) {
  const float rho = 1.0f + drho;
  const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
  sub_deq(d, drho, rho, ux, uy, uz, usq15);      // f - f^eq
  fwd_axis<1>(d, ux);
  fwd_axis<3>(d, uy);
  fwd_axis<9>(d, uz);                            // kappa^neq
  relax(d, kf);                                  // (I - S) kappa^neq
  inv_axis<9>(d, uz);
  inv_axis<3>(d, uy);
  inv_axis<1>(d, ux);                            // back to populations
  add_deq(d, drho, rho, ux, uy, uz, usq15);      // + f^eq
}

// Equilibrium (shifted) for given rho, u.
__device__ __forceinline__ void equilibrium(float (&d)[27], float rho, float ux, float uy,
                                            float uz) {
#pragma unroll
  for (int k = 0; k < 27; ++k) d[k] = 0.0f;
  add_deq(d, rho - 1.0f, rho, ux, uy, uz, 1.5f * (ux * ux + uy * uy + uz * uz));
}

// Index of node k+o along an axis of n nodes: periodic wrap or clamp (open face).
__device__ __forceinline__ int nbr(int k, int o, int n, int periodic) {
  int j = k + o;
  if (j < 0) j = periodic ? j + n : 0;
  else if (j >= n) j = periodic ? j - n : n - 1;
  return j;
}

// Departure-point sampling of the scalar: trilinear interpolation of c at x - u, with the
// displacement limited to one node per step; periodic axes wrap, open axes clamp.
struct Axis1 { int i0, i1; float t; };
__device__ __forceinline__ Axis1 sl_axis(int x, float u, int n, int periodic) {
  float dsp = -u;
  if (!(dsp == dsp)) dsp = 0.0f;                 // NaN guard: keeps indices in range
  dsp = fminf(fmaxf(dsp, -1.0f), 1.0f);
  const float fl = floorf(dsp);
  Axis1 r;
  r.t = dsp - fl;
  int i0 = x + int(fl);
  if (periodic) {
    if (i0 < 0) i0 += n;
    if (i0 >= n) i0 -= n;
    int i1 = i0 + 1;
    if (i1 >= n) i1 -= n;
    r.i0 = i0; r.i1 = i1;
  } else {
    if (i0 < 0) { i0 = 0; r.t = 0.0f; }
    if (i0 > n - 1) { i0 = n - 1; r.t = 0.0f; }
    int i1 = i0 + 1;
    if (i1 > n - 1) { i1 = n - 1; }
    r.i0 = i0; r.i1 = i1;
  }
  return r;
}

}  // namespace lbm
