// Device-side building blocks of the D3Q27 central-moment (CMR) collide-and-stream update.
//
// Populations live in "cube order": k = (cx+1) + 3 (cy+1) + 9 (cz+1), so the opposite of k
// is 26 - k and the three velocities of a line along one axis are three consecutive (or
// 3-/9-strided) slots.  Storage holds the shifted population d_k = f_k - w_k (f_k minus the
// rest-state weight), which keeps the stored magnitudes small; the FP16 mode stores the same
// quantity in half precision.
//
// Collision (Sec. 3.1, Eq. 2: Omega = -T S (m - m^eq)).  The paper's moments m_j are fixed
// linear combinations of the raw central moments
//     kappa_abc = sum_i f_i (c_ix - u_x)^a (c_iy - u_y)^b (c_iz - u_z)^c ,
// and S is constant inside each combination group, so relaxing every kappa_abc towards its
// equilibrium with its group's rate is the paper's m-space relaxation.  The only group that
// mixes is the second-order diagonal: the deviators m_7 = k200 - k020, m_8 = k200 - k002
// relax with the shear rate and the trace m_9 with the rate of group 9..16.
//
// Evaluation per node:
//   1. raw moments r_abc = sum_i d_i c_ix^a c_iy^b c_iz^c by three 3-point sweeps; they give
//      rho - 1 = r_000 and the momentum j = (r_100, r_010, r_001) for free;
//   2. a binomial shift turns raw moments of d into central moments about u;
//   3. relaxation towards Delta_abc = kappa^eq_abc - kappa_abc(w): the equilibrium central
//      moments of the Appendix (m^eq recombined per kappa) minus the central moments of the
//      rest weights (a product of the 1-D moments 1, -u, 1/3 + u^2).  All Delta are small
//      numbers, so FP32 keeps the non-equilibrium part accurate;
//   4. inverse sweeps (exact inverse of 1 + 2) give the post-collision shifted populations.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

// Cell flags (bits 0..3 are user-visible, bits 4..6 are derived by the library).  With
// obstacle walls on, an obstacle's surface voxels carry F_OBST_WALL instead of F_SOLID (they
// are active wall nodes at rest) and only its inner voxels keep F_SOLID.
enum : uint8_t {
  F_SOLID = 1, F_INFLOW = 2, F_SCALAR_SRC = 4, F_GHOST = 8, F_NEAR_SOLID = 16, F_WALL = 32,
  F_OBST_WALL = 64
};

// Bit of BlockView::walls (above the six face bits) for obstacle surfaces as walls.
constexpr int WALLS_OBSTACLES = 64;

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

// Paper velocity index q (Appendix list, index 13 read as (1,0,-1)) -> cube slot k.
__host__ __device__ constexpr int paper_to_cube(int q) {
  constexpr int t[27] = {13, 14, 12, 16, 10, 22, 4, 17, 15, 11, 9, 23, 21, 5,
                         3,  25, 19, 7,  1,  26, 24, 20, 18, 8, 6, 2,  0};
  return t[q];
}

// Storage element conversions.
// FP32 populations: read-only loads with a 256-byte L2 prefetch hint (the planes are read
// as streams; measured +0.7 % on the 256^3 collide-stream over plain __ldg)
__device__ __forceinline__ float load_pop(const float* p) {
  float v;
  asm volatile("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float load_pop(const __half* p) {
  return __half2float(__ldg(reinterpret_cast<const __half*>(p)));
}
// FP32 populations: plain stores (measured 0.4 % faster than streaming stores on the 256^3
// collide-stream; evict-first loads were 5 % slower)
__device__ __forceinline__ void store_pop(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_pop(__half* p, float v) {
  __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v)));
}
// Two consecutive populations of one plane (p aligned to two elements).
__device__ __forceinline__ float2 load_pop2(const float* p) {
  float2 v;
  asm volatile("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 load_pop2(const __half* p) {
  return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
}
__device__ __forceinline__ void store_pop2(float* p, float2 v) {
  *reinterpret_cast<float2*>(p) = v;
}
__device__ __forceinline__ void store_pop2(__half* p, float2 v) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&h));
}

// Lane arithmetic of the collision.  V is float (one node per thread) or float2 (two
// nodes of a row per thread, the sm_100 paired FP32 instructions); every operation is an
// explicitly rounded intrinsic (no contraction left to the compiler) and the float2 forms
// are the float forms per component, so both widths give bit-identical nodes.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a + (-1) b: the product is exact, so the one rounding is that of the difference
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return __fmul2_rn(a, make_float2(-1.0f, -1.0f)); }
template <typename V> __device__ __forceinline__ V vsplat(float c);
template <> __device__ __forceinline__ float vsplat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 vsplat<float2>(float c) { return make_float2(c, c); }

// Relaxation "keep" factors 1 - S for the moment groups of the Appendix.
template <typename V>
struct KeepT {
  V nu;      // moments 4..8 (shear / deviatoric stress), S = 1/(3 nu + 1/2)
  V g[4];    // high-order groups 9..16, 17..22, 23..25, 26
};
using Keep = KeepT<float>;

// The keep factors of two nodes as one pair.
__device__ __forceinline__ KeepT<float2> pair_keep(const Keep& a, const Keep& b) {
  KeepT<float2> k;
  k.nu = make_float2(a.nu, b.nu);
#pragma unroll
  for (int g = 0; g < 4; ++g) k.g[g] = make_float2(a.g[g], b.g[g]);
  return k;
}

struct RelaxParams {
  float s_nu;        // S for moments 4..8
  float nuh3[4];     // 3 * nu'_g for the four high-order groups
  float a, b;        // adaptive model parameters (Sec. 4.1)
  float inv_gmax;    // 1 / g_max
  int adaptive;
  int local;         // 1: |grad u| from the node's non-equilibrium moments, 0: lagged field
};

// Hardware reciprocal (PTX rcp.approx.ftz.f32, at most 1 ulp from the exact value): the
// arguments here are densities and relaxation denominators near 1, far from denormals.
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Sec. 4.1: S_i = 1/(3 phi nu'_i + 1/2) for i >= 9 with phi = a min(|grad u|/g_max, 1) + b.
__device__ __forceinline__ Keep keep_factors(const RelaxParams& rp, float grad_norm) {
  Keep kf;
  kf.nu = __fsub_rn(1.0f, rp.s_nu);
  float phi = 1.0f;
  if (rp.adaptive) phi = __fmaf_rn(rp.a, fminf(__fmul_rn(grad_norm, rp.inv_gmax), 1.0f), rp.b);
#pragma unroll
  for (int g = 0; g < 4; ++g) kf.g[g] = __fsub_rn(1.0f, fast_rcp(__fmaf_rn(phi, rp.nuh3[g], 0.5f)));
  return kf;
}

// Shifted equilibrium d^eq_k = f^eq_k - w_k = w_k (drho + rho (3 cu + 9/2 cu^2 - 3/2 u.u))
// (used for initialisation and Dirichlet inflow nodes).
template <int K>
__device__ __forceinline__ float deq_k(float drho, float rho, float ux, float uy, float uz,
                                       float usq15) {
  const float cu = float(cxk(K)) * ux + float(cyk(K)) * uy + float(czk(K)) * uz;
  return wk(K) * (drho + rho * (cu * (3.0f + 4.5f * cu) - usq15));
}
template <int K0 = 0>
__device__ __forceinline__ void add_deq(float (&d)[27], float drho, float rho, float ux, float uy,
                                        float uz, float usq15) {
  if constexpr (K0 < 27) {
    d[K0] += deq_k<K0>(drho, rho, ux, uy, uz, usq15);
    add_deq<K0 + 1>(d, drho, rho, ux, uy, uz, usq15);
  }
}

// line base of line l (0..8) for sweeps along stride 1 (x), 3 (y) or 9 (z)
template <int STRIDE>
__host__ __device__ constexpr int line_base(int l) {
  return (STRIDE == 1) ? 3 * l : (STRIDE == 3) ? (l % 3) + 9 * (l / 3) : l;
}

// Raw 3-point moments of one line (slots = velocity -1, 0, +1) -> orders 0, 1, 2:
// (a + c) + m, c - a, a + c (three operations per line).
template <int STRIDE, typename V>
__device__ __forceinline__ void raw_axis(V (&v)[27]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const V a = v[b], m = v[b + STRIDE], c = v[b + 2 * STRIDE];
    const V ac = vadd(a, c);
    v[b] = vadd(ac, m);
    v[b + STRIDE] = vsub(c, a);
    v[b + 2 * STRIDE] = ac;
  }
}
// Binomial shift of raw moments (orders 0,1,2) to central moments about u.
template <int STRIDE, typename V>
__device__ __forceinline__ void shift_axis(V (&v)[27], V u) {
  const V nu = vneg(u);
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const V r0 = v[b], r1 = v[b + STRIDE], r2 = v[b + 2 * STRIDE];
    const V k1 = vfma(nu, r0, r1);
    v[b + STRIDE] = k1;
    v[b + 2 * STRIDE] = vfma(nu, vadd(r1, k1), r2);
  }
}
// Central moments about u (orders 0,1,2) back to the three populations of the line: raw
// moments r1 = u k0 + k1, r2 = u (k1 + r1) + k2, then with h = r1/2: f(-1) = r2/2 - h,
// f(0) = k0 - r2, f(+1) = r2/2 + h (seven operations per line, the negation folded into
// the one-node form's fma; h off the r2 chain, which measured faster on the latency-bound
// small blocks of the multi-scale step than halving r2: 413 -> 407 us per reference step).
template <int STRIDE, typename V>
__device__ __forceinline__ void inv_axis(V (&v)[27], V u) {
  const V half = vsplat<V>(0.5f);
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const V k0 = v[b], k1 = v[b + STRIDE], k2 = v[b + 2 * STRIDE];
    const V r1 = vfma(u, k0, k1);
    const V r2 = vfma(u, vadd(k1, r1), k2);
    const V h1 = vmul(half, r1);
    v[b] = vfma(half, r2, vneg(h1));
    v[b + STRIDE] = vsub(k0, r2);
    v[b + 2 * STRIDE] = vfma(half, r2, h1);
  }
}

// kappa index of orders (a, b, c)
__host__ __device__ constexpr int kap(int a, int b, int c) { return a + 3 * b + 9 * c; }

// Relaxation of one central moment towards its offset dl with keep factor k.
template <typename V>
__device__ __forceinline__ void relax1(V& m, V dl, V k) { m = vfma(k, vsub(m, dl), dl); }

// Relaxation of the central moments of d towards Delta (see header), in place.
// v holds central moments of the shifted populations about u; keep factors kf; K = 1 - S.
template <typename V>
__device__ __forceinline__ void relax_to_equilibrium(V (&v)[27], V drho, V X, V Y, V Z,
                                                     const KeepT<V>& kf) {
  const V third = vsplat<V>(1.0f / 3.0f), ninth = vsplat<V>(1.0f / 9.0f);
  const V mthird = vsplat<V>(-1.0f / 3.0f);
  const V X2 = vmul(X, X), Y2 = vmul(Y, Y), Z2 = vmul(Z, Z);
  const V nX = vneg(X), nY = vneg(Y), ndrho = vneg(drho);
  // second order, off-diagonal (m_4, m_5, m_6): kappa^eq = 0, kappa(w) = u_a u_b
  relax1(v[kap(1, 1, 0)], vmul(nX, Y), kf.nu);
  relax1(v[kap(1, 0, 1)], vmul(nX, Z), kf.nu);
  relax1(v[kap(0, 1, 1)], vmul(nY, Z), kf.nu);
  // second order, diagonal: kappa^eq = rho/3, kappa(w) = 1/3 + u_a^2
  const V dr3 = vmul(drho, third);
  {
    const V ex = vsub(dr3, X2), ey = vsub(dr3, Y2), ez = vsub(dr3, Z2);
    const V A = vsub(v[kap(2, 0, 0)], ex), B = vsub(v[kap(0, 2, 0)], ey);
    const V Cc = vsub(v[kap(0, 0, 2)], ez);
    const V d1 = vmul(kf.nu, vsub(A, B));
    const V d2 = vmul(kf.nu, vsub(A, Cc));
    const V tr = vmul(kf.g[0], vadd(vadd(A, B), Cc));
    const V m2 = vsplat<V>(-2.0f);
    v[kap(2, 0, 0)] = vfma(third, vadd(vadd(tr, d1), d2), ex);
    v[kap(0, 2, 0)] = vfma(third, vadd(vfma(m2, d1, tr), d2), ey);
    v[kap(0, 0, 2)] = vfma(third, vfma(m2, d2, vadd(tr, d1)), ez);
  }
  // third order (m_10 .. m_16)
  relax1(v[kap(1, 2, 0)], vmul(X, vfma(ndrho, Y2, third)), kf.g[0]);
  relax1(v[kap(1, 0, 2)], vmul(X, vfma(ndrho, Z2, third)), kf.g[0]);
  relax1(v[kap(2, 1, 0)], vmul(Y, vfma(ndrho, X2, third)), kf.g[0]);
  relax1(v[kap(0, 1, 2)], vmul(Y, vfma(ndrho, Z2, third)), kf.g[0]);
  relax1(v[kap(2, 0, 1)], vmul(Z, vfma(ndrho, X2, third)), kf.g[0]);
  relax1(v[kap(0, 2, 1)], vmul(Z, vfma(ndrho, Y2, third)), kf.g[0]);
  relax1(v[kap(1, 1, 1)], vmul(vmul(vmul(ndrho, X), Y), Z), kf.g[0]);
  const V X2Y2 = vmul(X2, Y2), X2Z2 = vmul(X2, Z2), Y2Z2 = vmul(Y2, Z2);
  // fourth order (m_17 .. m_22)
  {
    const V r3m1 = vfma(vsplat<V>(3.0f), drho, vsplat<V>(2.0f));  // 3 rho - 1
    const V dr9 = vmul(drho, ninth);
    relax1(v[kap(2, 2, 0)], vfma(r3m1, X2Y2, vfma(vadd(X2, Y2), mthird, dr9)), kf.g[1]);
    relax1(v[kap(2, 0, 2)], vfma(r3m1, X2Z2, vfma(vadd(X2, Z2), mthird, dr9)), kf.g[1]);
    relax1(v[kap(0, 2, 2)], vfma(r3m1, Y2Z2, vfma(vadd(Y2, Z2), mthird, dr9)), kf.g[1]);
    relax1(v[kap(2, 1, 1)], vmul(vmul(Y, Z), vfma(r3m1, X2, mthird)), kf.g[1]);
    relax1(v[kap(1, 2, 1)], vmul(vmul(X, Z), vfma(r3m1, Y2, mthird)), kf.g[1]);
    relax1(v[kap(1, 1, 2)], vmul(vmul(X, Y), vfma(r3m1, Z2, mthird)), kf.g[1]);
  }
  // fifth order (m_23 .. m_25)
  {
    const V o6 = vfma(vsplat<V>(-6.0f), drho, vsplat<V>(-5.0f));  // 1 - 6 rho
    const V ndr3 = vneg(dr3);
    relax1(v[kap(1, 2, 2)], vmul(X, vfma(o6, Y2Z2, vfma(ndr3, vadd(Y2, Z2), ninth))), kf.g[2]);
    relax1(v[kap(2, 1, 2)], vmul(Y, vfma(o6, X2Z2, vfma(ndr3, vadd(X2, Z2), ninth))), kf.g[2]);
    relax1(v[kap(2, 2, 1)], vmul(Z, vfma(o6, X2Y2, vfma(ndr3, vadd(X2, Y2), ninth))), kf.g[2]);
  }
  // sixth order (m_26)
  {
    const V rho = vadd(vsplat<V>(1.0f), drho);
    const V p2 = vadd(vadd(X2Y2, X2Z2), Y2Z2);
    const V s2 = vadd(vadd(X2, Y2), Z2);
    const V lo = vfma(drho, vsplat<V>(1.0f / 27.0f), vmul(s2, vsplat<V>(-1.0f / 9.0f)));
    const V d222 = vfma(vfma(vsplat<V>(10.0f), rho, vsplat<V>(-1.0f)), vmul(X2Y2, Z2),
                        vfma(vsub(rho, third), p2, lo));
    relax1(v[kap(2, 2, 2)], d222, kf.g[3]);
  }
  // orders 0 and 1 (S_0..3 = 0) are left as they are
}

// Raw moment sweeps: afterwards v[kap(0,0,0)] = rho - 1 and v[kap(1,0,0)] = j_x etc.
template <typename V>
__device__ __forceinline__ void raw_moments(V (&v)[27]) {
  raw_axis<1>(v);
  raw_axis<3>(v);
  raw_axis<9>(v);
}

// Raw moments -> central moments about u (in place).
template <typename V>
__device__ __forceinline__ void central_from_raw(V (&v)[27], V ux, V uy, V uz) {
  shift_axis<1>(v, ux);
  shift_axis<3>(v, uy);
  shift_axis<9>(v, uz);
}

// Relaxation of central moments and the inverse sweeps back to populations (in place).
template <typename V>
__device__ __forceinline__ void collide_from_central(V (&v)[27], V drho, V ux, V uy, V uz,
                                                     const KeepT<V>& kf) {
  relax_to_equilibrium(v, drho, ux, uy, uz, kf);
  inv_axis<9>(v, uz);
  inv_axis<3>(v, uy);
  inv_axis<1>(v, ux);
}

// Collision of shifted populations given their raw moments (from raw_moments) and u:
// raw -> central, relax towards equilibrium, back to populations (in place).
template <typename V>
__device__ __forceinline__ void collide_from_raw(V (&v)[27], V drho, V ux, V uy, V uz,
                                                 const KeepT<V>& kf) {
  central_from_raw(v, ux, uy, uz);
  collide_from_central(v, drho, ux, uy, uz, kf);
}

// |grad u| from a node's central moments (of the shifted populations, before relaxation):
// the non-equilibrium second moments Pi = kappa - Delta give the strain rate through
// Pi^(1) = -2 c_s^2 rho S_hat / S (Sec. 4.2.1, c_s^2 = 1/3); returns sqrt(2 S_hat : S_hat).
template <typename V>
__device__ __forceinline__ V local_strain_sq(const V (&v)[27], V drho, V X, V Y, V Z) {
  const V dr3 = vmul(drho, vsplat<V>(1.0f / 3.0f));
  const V pxx = vsub(v[kap(2, 0, 0)], vsub(dr3, vmul(X, X)));
  const V pyy = vsub(v[kap(0, 2, 0)], vsub(dr3, vmul(Y, Y)));
  const V pzz = vsub(v[kap(0, 0, 2)], vsub(dr3, vmul(Z, Z)));
  const V pxy = vfma(X, Y, v[kap(1, 1, 0)]);
  const V pxz = vfma(X, Z, v[kap(1, 0, 1)]);
  const V pyz = vfma(Y, Z, v[kap(0, 1, 1)]);
  const V dg = vfma(pxx, pxx, vfma(pyy, pyy, vmul(pzz, pzz)));
  const V od = vfma(pxy, pxy, vfma(pxz, pxz, vmul(pyz, pyz)));
  return vfma(vsplat<V>(2.0f), od, dg);
}
__device__ __forceinline__ float strain_from_sq(float ss, float drho, float s_nu) {
  const float scale = __fdiv_rn(__fmul_rn(1.5f, s_nu), __fadd_rn(1.0f, drho));
  return __fmul_rn(scale, sqrtf(__fmul_rn(2.0f, ss)));
}
__device__ __forceinline__ float local_strain(const float (&v)[27], float drho, float X, float Y,
                                              float Z, float s_nu) {
  return strain_from_sq(local_strain_sq(v, drho, X, Y, Z), drho, s_nu);
}

// Equilibrium (shifted) for given rho, u.
__device__ __forceinline__ void equilibrium(float (&d)[27], float rho, float ux, float uy,
                                            float uz) {
#pragma unroll
  for (int k = 0; k < 27; ++k) d[k] = 0.0f;
  add_deq(d, rho - 1.0f, rho, ux, uy, uz, 1.5f * (ux * ux + uy * uy + uz * uz));
}

// Sums of shifted populations: drho = rho - 1, j = sum c d (for kernels that do not sweep).
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
