// Reverse-mode (vector-Jacobian) building blocks of the collide-stream update.
//
// Every forward stage of lbm_device.cuh has its exact transpose here.  Stage inputs that the
// reverse needs are reconstructed from the central moments with the exact inverse sweeps
// (unshift_axis, inv_axis), so a node's reverse keeps three 27-arrays live instead of seven.
// The equilibrium offsets Delta(rho - 1, u) of the relaxation are differentiated with a small
// forward-mode dual number (value plus the partials with respect to rho - 1 and u that are not
// zero by construction).
#pragma once
#include "lbm_device.cuh"

namespace lbm {

// Value and the partials with respect to (rho - 1, u_x, u_y, u_z) whose bits are set in M
// (bit 0: rho - 1, bits 1-3: u_x, u_y, u_z).  Partials that are zero by construction are
// neither stored nor computed: IEEE arithmetic does not let the compiler drop 0 * x, so a
// dense dual number would multiply every zero partial out.
template <unsigned M>
struct Dual {
  float v;
  float d[4];
};
template <unsigned M>
__device__ __forceinline__ constexpr bool dual_has(int i) { return ((M >> i) & 1u) != 0u; }

template <unsigned A, unsigned B>
__device__ __forceinline__ Dual<A | B> operator+(const Dual<A>& a, const Dual<B>& b) {
  Dual<A | B> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    r.d[i] = dual_has<A>(i) && dual_has<B>(i) ? a.d[i] + b.d[i]
             : dual_has<A>(i)                 ? a.d[i]
             : dual_has<B>(i)                 ? b.d[i]
                                              : 0.0f;
  return r;
}
template <unsigned A, unsigned B>
__device__ __forceinline__ Dual<A | B> operator-(const Dual<A>& a, const Dual<B>& b) {
  Dual<A | B> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    r.d[i] = dual_has<A>(i) && dual_has<B>(i) ? a.d[i] - b.d[i]
             : dual_has<A>(i)                 ? a.d[i]
             : dual_has<B>(i)                 ? -b.d[i]
                                              : 0.0f;
  return r;
}
template <unsigned A, unsigned B>
__device__ __forceinline__ Dual<A | B> operator*(const Dual<A>& a, const Dual<B>& b) {
  Dual<A | B> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    r.d[i] = dual_has<A>(i) && dual_has<B>(i) ? a.d[i] * b.v + a.v * b.d[i]
             : dual_has<A>(i)                 ? a.d[i] * b.v
             : dual_has<B>(i)                 ? a.v * b.d[i]
                                              : 0.0f;
  return r;
}
template <unsigned A>
__device__ __forceinline__ Dual<A> operator-(const Dual<A>& a) {
  Dual<A> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = dual_has<A>(i) ? -a.d[i] : 0.0f;
  return r;
}
template <unsigned A>
__device__ __forceinline__ Dual<A> operator*(const Dual<A>& a, float s) {
  Dual<A> r;
  r.v = a.v * s;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = dual_has<A>(i) ? a.d[i] * s : 0.0f;
  return r;
}
template <unsigned A>
__device__ __forceinline__ Dual<A> operator+(const Dual<A>& a, float s) {
  Dual<A> r = a;
  r.v = a.v + s;
  return r;
}
template <unsigned A>
__device__ __forceinline__ Dual<A> operator-(float s, const Dual<A>& a) {
  Dual<A> r;
  r.v = s - a.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = dual_has<A>(i) ? -a.d[i] : 0.0f;
  return r;
}
__device__ __forceinline__ Dual<0u> dual_const(float c) { return Dual<0u>{c, {0.f, 0.f, 0.f, 0.f}}; }

// bar[i] += db * d(dl)/d(variable i) for the partials dl carries
template <unsigned M>
__device__ __forceinline__ void dual_grad(float db, const Dual<M>& dl, float (&bar)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (dual_has<M>(i)) bar[i] = fmaf(db, dl.d[i], bar[i]);
}

// Central moments about u back to raw moments (inverse of shift_axis).
template <int STRIDE>
__device__ __forceinline__ void unshift_axis(float (&v)[27], float u) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const float k0 = v[b], k1 = v[b + STRIDE], k2 = v[b + 2 * STRIDE];
    const float r1 = fmaf(u, k0, k1);
    v[b + STRIDE] = r1;
    v[b + 2 * STRIDE] = fmaf(u, k1 + r1, k2);
  }
}

// Transpose of inv_axis: T holds the sweep's inputs (central moments), A the adjoint of its
// outputs on entry and of its inputs on return; ubar accumulates d/du.
template <int STRIDE>
__device__ __forceinline__ void inv_axis_vjp(const float (&T)[27], float (&A)[27], float u,
                                             float& ubar) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const float k0 = T[b], k1 = T[b + STRIDE];
    const float r1 = fmaf(u, k0, k1);
    const float s0 = A[b], s1 = A[b + STRIDE], s2 = A[b + 2 * STRIDE];
    const float r2b = 0.5f * s0 - s1 + 0.5f * s2;
    float r1b = 0.5f * (s2 - s0);
    float k0b = s1;
    float k1b = u * r2b;
    r1b = fmaf(u, r2b, r1b);
    ubar = fmaf(k1 + r1, r2b, ubar);
    k1b += r1b;
    k0b = fmaf(u, r1b, k0b);
    ubar = fmaf(k0, r1b, ubar);
    A[b] = k0b;
    A[b + STRIDE] = k1b;
    A[b + 2 * STRIDE] = r2b;
  }
}

// Transpose of shift_axis: T holds the shift's inputs (raw-ordered moments).
template <int STRIDE>
__device__ __forceinline__ void shift_axis_vjp(const float (&T)[27], float (&A)[27], float u,
                                               float& ubar) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const float r0 = T[b], r1 = T[b + STRIDE];
    const float k1 = fmaf(-u, r0, r1);
    const float k0b = A[b], k1b0 = A[b + STRIDE], k2b = A[b + 2 * STRIDE];
    const float r2b = k2b;
    float r1b = -u * k2b;
    const float k1b = fmaf(-u, k2b, k1b0);
    ubar = fmaf(-(r1 + k1), k2b, ubar);
    r1b += k1b;
    const float r0b = fmaf(-u, k1b, k0b);
    ubar = fmaf(-r0, k1b, ubar);
    A[b] = r0b;
    A[b + STRIDE] = r1b;
    A[b + 2 * STRIDE] = r2b;
  }
}

// Transpose of raw_axis (a linear map with constant coefficients).
template <int STRIDE>
__device__ __forceinline__ void raw_axis_vjp(float (&A)[27]) {
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int b = line_base<STRIDE>(l);
    const float r0 = A[b], r1 = A[b + STRIDE], r2 = A[b + 2 * STRIDE];
    A[b] = r0 - r1 + r2;
    A[b + STRIDE] = r0;
    A[b + 2 * STRIDE] = r0 + r1 + r2;
  }
}

// Transpose of relax_to_equilibrium.  K: the node's keep factors; v: the central moments
// before relaxation; A: adjoint of the relaxed moments on entry, of v on return.  Adds the
// adjoints of (rho - 1, u) to bar[0..3] and of the high-order keep factors to kbar[0..3].
__device__ __forceinline__ void relax_vjp(const float (&v)[27], float (&A)[27], float drho,
                                          float X, float Y, float Z, const Keep& kf,
                                          float (&bar)[4], float (&kbar)[4]) {
  // Each moment's Delta (with its four partials) is formed and consumed at once, so only a
  // few dual numbers are live at any time.
  const float third = 1.0f / 3.0f, ninth = 1.0f / 9.0f;
  const Dual<1u> dr{drho, {1.f, 0.f, 0.f, 0.f}};
  const Dual<2u> x{X, {0.f, 1.f, 0.f, 0.f}};
  const Dual<4u> y{Y, {0.f, 0.f, 1.f, 0.f}};
  const Dual<8u> z{Z, {0.f, 0.f, 0.f, 1.f}};
  // out_i = Delta_i + K (v_i - Delta_i): dv_i = K o, dDelta_i = (1 - K) o, dK = o (v_i - Delta_i)
  auto one = [&](int i, const auto& dl, float K, int grp) {
    const float o = A[i];
    A[i] = K * o;
    if (grp >= 0) kbar[grp] = fmaf(o, v[i] - dl.v, kbar[grp]);
    dual_grad((1.0f - K) * o, dl, bar);
  };
  one(kap(1, 1, 0), -(x * y), kf.nu, -1);
  one(kap(1, 0, 1), -(x * z), kf.nu, -1);
  one(kap(0, 1, 1), -(y * z), kf.nu, -1);
  const auto x2 = x * x;
  const auto y2 = y * y;
  const auto z2 = z * z;
  {  // second-order diagonal: deviators at the shear rate, trace at group 9..16
    const auto dr3 = dr * third;
    const auto ex = dr3 - x2;
    const auto ey = dr3 - y2;
    const auto ez = dr3 - z2;
    const float Aa = v[kap(2, 0, 0)] - ex.v, Bb = v[kap(0, 2, 0)] - ey.v, Cc = v[kap(0, 0, 2)] - ez.v;
    const float o2 = A[kap(2, 0, 0)], o3 = A[kap(0, 2, 0)], o4 = A[kap(0, 0, 2)];
    const float trb = (o2 + o3 + o4) * third;
    const float d1b = (o2 - 2.0f * o3 + o4) * third;
    const float d2b = (o2 + o3 - 2.0f * o4) * third;
    const float Ab = kf.nu * (d1b + d2b) + kf.g[0] * trb;
    const float Bb_ = -kf.nu * d1b + kf.g[0] * trb;
    const float Cb = -kf.nu * d2b + kf.g[0] * trb;
    kbar[0] = fmaf(trb, Aa + Bb + Cc, kbar[0]);
    A[kap(2, 0, 0)] = Ab;
    A[kap(0, 2, 0)] = Bb_;
    A[kap(0, 0, 2)] = Cb;
    dual_grad(o2 - Ab, ex, bar);
    dual_grad(o3 - Bb_, ey, bar);
    dual_grad(o4 - Cb, ez, bar);
  }
  one(kap(1, 2, 0), x * (third - dr * y2), kf.g[0], 0);
  one(kap(1, 0, 2), x * (third - dr * z2), kf.g[0], 0);
  one(kap(2, 1, 0), y * (third - dr * x2), kf.g[0], 0);
  one(kap(0, 1, 2), y * (third - dr * z2), kf.g[0], 0);
  one(kap(2, 0, 1), z * (third - dr * x2), kf.g[0], 0);
  one(kap(0, 2, 1), z * (third - dr * y2), kf.g[0], 0);
  one(kap(1, 1, 1), -(dr * x * y * z), kf.g[0], 0);
  {
    const auto r3m1 = dr * 3.0f + 2.0f;   // 3 rho - 1
    const auto dr9 = dr * ninth;
    one(kap(2, 2, 0), r3m1 * x2 * y2 + dr9 - (x2 + y2) * third, kf.g[1], 1);
    one(kap(2, 0, 2), r3m1 * x2 * z2 + dr9 - (x2 + z2) * third, kf.g[1], 1);
    one(kap(0, 2, 2), r3m1 * y2 * z2 + dr9 - (y2 + z2) * third, kf.g[1], 1);
    one(kap(2, 1, 1), y * z * (r3m1 * x2 - dual_const(third)), kf.g[1], 1);
    one(kap(1, 2, 1), x * z * (r3m1 * y2 - dual_const(third)), kf.g[1], 1);
    one(kap(1, 1, 2), x * y * (r3m1 * z2 - dual_const(third)), kf.g[1], 1);
  }
  {
    const auto o6 = dr * (-6.0f) + (-5.0f);   // 1 - 6 rho
    const auto dr3 = dr * third;
    one(kap(1, 2, 2), x * (o6 * y2 * z2 + (ninth - dr3 * (y2 + z2))), kf.g[2], 2);
    one(kap(2, 1, 2), y * (o6 * x2 * z2 + (ninth - dr3 * (x2 + z2))), kf.g[2], 2);
    one(kap(2, 2, 1), z * (o6 * x2 * y2 + (ninth - dr3 * (x2 + y2))), kf.g[2], 2);
  }
  {
    const auto rho = dr + 1.0f;
    const auto p2 = x2 * y2 + x2 * z2 + y2 * z2;
    const auto d222 = (rho * 10.0f + (-1.0f)) * x2 * y2 * z2 + (rho + (-third)) * p2 +
                    dr * (1.0f / 27.0f) - (x2 + y2 + z2) * ninth;
    one(kap(2, 2, 2), d222, kf.g[3], 3);
  }
}

}  // namespace lbm
