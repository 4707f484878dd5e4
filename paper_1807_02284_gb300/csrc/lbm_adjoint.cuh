// Reverse-mode (vector-Jacobian) building blocks of the collide-stream update.
//
// Every forward stage of lbm_device.cuh has its exact transpose here.  Stage inputs that the
// reverse needs are reconstructed from the central moments with the exact inverse sweeps
// (unshift_axis, inv_axis), so a node's reverse keeps three 27-arrays live instead of seven.
// The equilibrium offsets Delta(rho - 1, u) of the relaxation are differentiated with a small
// forward-mode dual number (value plus four partials).
#pragma once
#include "lbm_device.cuh"

namespace lbm {

// Value and partials with respect to (rho - 1, u_x, u_y, u_z).
struct D4 {
  float v, d0, d1, d2, d3;
};
__device__ __forceinline__ D4 d4c(float c) { return D4{c, 0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ D4 operator+(D4 a, D4 b) { return D4{a.v + b.v, a.d0 + b.d0, a.d1 + b.d1, a.d2 + b.d2, a.d3 + b.d3}; }
__device__ __forceinline__ D4 operator-(D4 a, D4 b) { return D4{a.v - b.v, a.d0 - b.d0, a.d1 - b.d1, a.d2 - b.d2, a.d3 - b.d3}; }
__device__ __forceinline__ D4 operator-(D4 a) { return D4{-a.v, -a.d0, -a.d1, -a.d2, -a.d3}; }
__device__ __forceinline__ D4 operator*(D4 a, D4 b) {
  return D4{a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2,
            a.d3 * b.v + a.v * b.d3};
}
__device__ __forceinline__ D4 operator*(D4 a, float s) { return D4{a.v * s, a.d0 * s, a.d1 * s, a.d2 * s, a.d3 * s}; }
__device__ __forceinline__ D4 operator+(D4 a, float s) { return D4{a.v + s, a.d0, a.d1, a.d2, a.d3}; }
__device__ __forceinline__ D4 operator-(float s, D4 a) { return D4{s - a.v, -a.d0, -a.d1, -a.d2, -a.d3}; }

// Delta_abc = kappa^eq_abc - kappa_abc(w) of the relaxed moments (the diagonal second-order
// slots hold rho/3 - 1/3 - u_a^2); the same algebra as relax_to_equilibrium.
__device__ __forceinline__ void delta_moments(D4 drho, D4 X, D4 Y, D4 Z, D4 (&D)[27]) {
  const float third = 1.0f / 3.0f, ninth = 1.0f / 9.0f;
  const D4 X2 = X * X, Y2 = Y * Y, Z2 = Z * Z;
  D[kap(1, 1, 0)] = -(X * Y);
  D[kap(1, 0, 1)] = -(X * Z);
  D[kap(0, 1, 1)] = -(Y * Z);
  const D4 dr3 = drho * third;
  D[kap(2, 0, 0)] = dr3 - X2;
  D[kap(0, 2, 0)] = dr3 - Y2;
  D[kap(0, 0, 2)] = dr3 - Z2;
  D[kap(1, 2, 0)] = X * (third - drho * Y2);
  D[kap(1, 0, 2)] = X * (third - drho * Z2);
  D[kap(2, 1, 0)] = Y * (third - drho * X2);
  D[kap(0, 1, 2)] = Y * (third - drho * Z2);
  D[kap(2, 0, 1)] = Z * (third - drho * X2);
  D[kap(0, 2, 1)] = Z * (third - drho * Y2);
  D[kap(1, 1, 1)] = -(drho * X * Y * Z);
  const D4 r3m1 = drho * 3.0f + 2.0f;
  const D4 dr9 = drho * ninth;
  D[kap(2, 2, 0)] = r3m1 * X2 * Y2 + dr9 - (X2 + Y2) * third;
  D[kap(2, 0, 2)] = r3m1 * X2 * Z2 + dr9 - (X2 + Z2) * third;
  D[kap(0, 2, 2)] = r3m1 * Y2 * Z2 + dr9 - (Y2 + Z2) * third;
  D[kap(2, 1, 1)] = Y * Z * (r3m1 * X2 - d4c(third));
  D[kap(1, 2, 1)] = X * Z * (r3m1 * Y2 - d4c(third));
  D[kap(1, 1, 2)] = X * Y * (r3m1 * Z2 - d4c(third));
  const D4 o6 = drho * (-6.0f) + (-5.0f);
  D[kap(1, 2, 2)] = X * (o6 * Y2 * Z2 + (ninth - dr3 * (Y2 + Z2)));
  D[kap(2, 1, 2)] = Y * (o6 * X2 * Z2 + (ninth - dr3 * (X2 + Z2)));
  D[kap(2, 2, 1)] = Z * (o6 * X2 * Y2 + (ninth - dr3 * (X2 + Y2)));
  const D4 rho = drho + 1.0f;
  const D4 p2 = X2 * Y2 + X2 * Z2 + Y2 * Z2;
  D[kap(2, 2, 2)] = (rho * 10.0f + (-1.0f)) * X2 * Y2 * Z2 + (rho + (-third)) * p2 +
                    drho * (1.0f / 27.0f) - (X2 + Y2 + Z2) * ninth;
  D[kap(0, 0, 0)] = d4c(0.f);
  D[kap(1, 0, 0)] = d4c(0.f);
  D[kap(0, 1, 0)] = d4c(0.f);
  D[kap(0, 0, 1)] = d4c(0.f);
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
  D4 D[27];
  delta_moments(D4{drho, 1.f, 0.f, 0.f, 0.f}, D4{X, 0.f, 1.f, 0.f, 0.f},
                D4{Y, 0.f, 0.f, 1.f, 0.f}, D4{Z, 0.f, 0.f, 0.f, 1.f}, D);
  float db[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) db[i] = 0.0f;
  // group of each relaxed moment: -1 shear (keep nu), 0..3 high-order groups
  auto relax_one = [&](int i, float K, int grp) {
    const float o = A[i];
    A[i] = K * o;
    db[i] = (1.0f - K) * o;
    if (grp >= 0) kbar[grp] = fmaf(o, v[i] - D[i].v, kbar[grp]);
  };
  relax_one(kap(1, 1, 0), kf.nu, -1);
  relax_one(kap(1, 0, 1), kf.nu, -1);
  relax_one(kap(0, 1, 1), kf.nu, -1);
  {
    const float ex = D[kap(2, 0, 0)].v, ey = D[kap(0, 2, 0)].v, ez = D[kap(0, 0, 2)].v;
    const float Aa = v[kap(2, 0, 0)] - ex, Bb = v[kap(0, 2, 0)] - ey, Cc = v[kap(0, 0, 2)] - ez;
    const float o2 = A[kap(2, 0, 0)], o3 = A[kap(0, 2, 0)], o4 = A[kap(0, 0, 2)];
    const float third = 1.0f / 3.0f;
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
    db[kap(2, 0, 0)] = o2 - Ab;
    db[kap(0, 2, 0)] = o3 - Bb_;
    db[kap(0, 0, 2)] = o4 - Cb;
  }
  relax_one(kap(1, 2, 0), kf.g[0], 0);
  relax_one(kap(1, 0, 2), kf.g[0], 0);
  relax_one(kap(2, 1, 0), kf.g[0], 0);
  relax_one(kap(0, 1, 2), kf.g[0], 0);
  relax_one(kap(2, 0, 1), kf.g[0], 0);
  relax_one(kap(0, 2, 1), kf.g[0], 0);
  relax_one(kap(1, 1, 1), kf.g[0], 0);
  relax_one(kap(2, 2, 0), kf.g[1], 1);
  relax_one(kap(2, 0, 2), kf.g[1], 1);
  relax_one(kap(0, 2, 2), kf.g[1], 1);
  relax_one(kap(2, 1, 1), kf.g[1], 1);
  relax_one(kap(1, 2, 1), kf.g[1], 1);
  relax_one(kap(1, 1, 2), kf.g[1], 1);
  relax_one(kap(1, 2, 2), kf.g[2], 2);
  relax_one(kap(2, 1, 2), kf.g[2], 2);
  relax_one(kap(2, 2, 1), kf.g[2], 2);
  relax_one(kap(2, 2, 2), kf.g[3], 3);
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    bar[0] = fmaf(db[i], D[i].d0, bar[0]);
    bar[1] = fmaf(db[i], D[i].d1, bar[1]);
    bar[2] = fmaf(db[i], D[i].d2, bar[2]);
    bar[3] = fmaf(db[i], D[i].d3, bar[3]);
  }
}

}  // namespace lbm
