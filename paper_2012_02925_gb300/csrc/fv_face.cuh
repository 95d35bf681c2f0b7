// Per-cell primitive recovery and per-face MUSCL reconstruction, slope
// limiter and Roe flux, written once for every arithmetic type T.
//
//  * Section 2 (vector Q, inviscid normal flux F_{i,n}, Roe's flux-difference
//    splitting, MUSCL on primitive variables);
//  * Eq. (flux) of Section 7.2 (V4): the kappa-scheme with limiter values
//    Psi^{+/-}; each limiter value multiplies the difference that is the
//    denominator of its ratio, so a limited term is Psi(a/b) b.
#pragma once
#include <type_traits>
#include "fv_arith.cuh"
#include "fv_internal.h"

template <class T>
struct FaceC {
  T gm1;          // gamma - 1
  T g_gm1;        // gamma / (gamma - 1)
  T half, one;
  T e4km, e4kp;   // eps/4 (1 - kappa), eps/4 (1 + kappa)
  T harten;       // entropy-fix width / c~
  T va_d2;        // van Albada delta^2
  T g, ig, i2g, gm1x2, igm1, i2g2m1, quarter, two;   // gamma, 1/gamma, 1/(2 gamma), 2(gamma-1),
                                                     // 1/(gamma-1), 1/(2(gamma^2-1)), 1/4, 2
  int flux;       // 0 Roe, 1 van Leer flux-vector splitting, 2 Steger-Warming
  int limiter, fix_all, has_fix;
  int upwind_only;  // kappa == -1: the (1+kappa) terms of Eq. (flux) vanish
  int unit_slope;   // eps (1 - kappa) / 2 == 1: the upwind slope enters with weight one
  // the scheme switches as the face code reads them
  __device__ __forceinline__ int k_flux() const { return flux; }
  __device__ __forceinline__ int k_lim() const { return limiter; }
  __device__ __forceinline__ int k_upw() const { return upwind_only; }
  __device__ __forceinline__ int k_unit() const { return unit_slope; }
  __device__ __forceinline__ int k_fix() const { return has_fix; }
  __device__ __forceinline__ int k_fixall() const { return fix_all; }
  static __device__ __forceinline__ FaceC from(const FaceC& b) { return b; }
};

// The default scheme fixed at compile time - Roe flux, van Leer limiter,
// eps = 1, kappa = -1, Harten fix on the acoustic waves only - so that the face code
// carries no run-time switches (their branches split the face into basic
// blocks the scheduler cannot interleave).  Same data as FaceC.
template <class T>
struct FaceCFast : FaceC<T> {
  __device__ __forceinline__ int k_flux() const { return 0; }
  __device__ __forceinline__ int k_lim() const { return 1; }
  __device__ __forceinline__ int k_upw() const { return 1; }
  __device__ __forceinline__ int k_unit() const { return 1; }
  __device__ __forceinline__ int k_fix() const { return 1; }
  __device__ __forceinline__ int k_fixall() const { return 0; }
  static __device__ __forceinline__ FaceCFast from(const FaceC<T>& b) {
    FaceCFast f;
    static_cast<FaceC<T>&>(f) = b;
    return f;
  }
};

template <class T>
__device__ __forceinline__ FaceC<T> make_face_consts(const FvFaceParams& p) {
  using S = Sc<T>;
  FaceC<T> c;
  c.gm1 = S::c(p.gamma - 1.0);
  c.g_gm1 = S::c(p.gamma / (p.gamma - 1.0));
  c.half = S::c(0.5);
  c.one = S::c(1.0);
  c.e4km = S::c(p.eps * 0.25 * (1.0 - p.kappa));
  c.e4kp = S::c(p.eps * 0.25 * (1.0 + p.kappa));
  c.harten = S::c(p.harten);
  c.va_d2 = S::c(p.va_delta2);
  c.g = S::c(p.gamma);
  c.ig = S::c(1.0 / p.gamma);
  c.i2g = S::c(0.5 / p.gamma);
  c.gm1x2 = S::c(2.0 * (p.gamma - 1.0));
  c.igm1 = S::c(1.0 / (p.gamma - 1.0));
  c.i2g2m1 = S::c(0.5 / (p.gamma * p.gamma - 1.0));
  c.quarter = S::c(0.25);
  c.two = S::c(2.0);
  c.flux = p.flux;
  c.limiter = p.limiter;
  c.fix_all = p.fix_all;
  c.has_fix = p.harten > 0.0;
  c.upwind_only = (p.kappa == -1.0);
  c.unit_slope = (p.eps * 0.5 * (1.0 - p.kappa) == 1.0);
  return c;
}

// Q = (rho, rho u, rho v, rho w, rho e_t) -> V = (rho, u, v, w, p), the
// kinetic energy rho |u|^2 / 2 as (rho u) . u / 2
template <class T, class CC>
__device__ __forceinline__ void prim_from_cons(const CC& C, const T q[5], T V[5]) {
  T rinv = Sc<T>::rcp(q[0]);
  T u = q[1] * rinv, v = q[2] * rinv, w = q[3] * rinv;
  V[0] = q[0];
  V[1] = u;
  V[2] = v;
  V[3] = w;
  V[4] = C.gm1 * (q[4] - Sc<T>::halve(Sc<T>::dot3(q[1], u, q[2], v, q[3], w)));
}

// Half the van Leer limited slope, Psi(a/b) b / 2 with Psi(r) = (r + |r|)/(1 + |r|).
// Psi(a/b) b = (a|b| + |a| b)/(|a| + |b|), which is 2ab/(a + b) when a and b
// have the same sign and 0 otherwise.  Both differences below 1e-30
// (rounding noise of a quantity that is zero, e.g. a transverse velocity):
// zero slope, as the oracle's guarded ratio gives to within 2e-30; it also
// keeps the binary32 reciprocal of a subnormal sum from overflowing.
template <class T>
__device__ __forceinline__ T vanleer_half(T a, T b) {
  using S = Sc<T>;
  const T p = a * b, s = a + b;
  const T h = S::div(p, s);
  return S::sel(S::pos(p) && S::above(S::abs(s), 1e-30f), h, S::c(0.0));
}

// Psi(a/b) * b
template <class T, class CC>
__device__ __forceinline__ T limited(const CC& C, T a, T b) {
  using S = Sc<T>;
  if (C.k_lim() == 0) return b;
  if (C.k_lim() == 1) {
    const T h = vanleer_half(a, b);
    return h + h;
  }
  // van Albada in smooth product form: b (a^2 + a b)/(a^2 + b^2 + delta^2)
  const T a2 = a * a;
  const T num = b * (a2 + a * b);
  return num * S::rcp(a2 + b * b + C.va_d2);
}

// Eq. (flux) for one component from V_{i-1}, V_i, V_{i+1}, V_{i+2}
template <class T, class CC>
__device__ __forceinline__ void muscl(const CC& C, T vm1, T v0, T vp1, T vp2, T& L, T& R) {
  T dm = v0 - vm1, d0 = vp1 - v0, dp = vp2 - vp1;
  if (C.k_upw() && C.k_unit() && C.k_lim() == 1) {
    // eps (1 - kappa)/4 * Psi(a/b) b = Psi(a/b) b / 2
    L = v0 + vanleer_half(d0, dm);
    R = vp1 - vanleer_half(d0, dp);
  } else if (C.k_upw()) {
    L = v0 + C.e4km * limited(C, d0, dm);
    R = vp1 - C.e4km * limited(C, d0, dp);
  } else {
    L = v0 + (C.e4km * limited(C, d0, dm) + C.e4kp * limited(C, dm, d0));
    R = vp1 - (C.e4kp * limited(C, dp, d0) + C.e4km * limited(C, d0, dp));
  }
}

// Harten: |l| <- (l^2 + d^2) / (2 d) when |l| < d (a branch: the fix is
// rare, near sonic points; a select costing both sides always was slower)
// (lam = |eigenvalue| and delta > 0 are non-negative)
template <class T, class CC>
__device__ __forceinline__ T entropy_fixed(const CC& C, T lam, T delta) {
  if (Sc<T>::lt_nonneg(lam, delta)) return (lam * lam + delta * delta) * Sc<T>::halve(Sc<T>::rcp(delta));
  return lam;
}

// Roe flux times face area for reconstructed primitive states VL, VR and the
// unit normal (nx, ny, nz) with area A.
template <class T, class CC>
__device__ __forceinline__ void roe_flux(const CC& C, const T VL[5], const T VR[5], T nx, T ny,
                                         T nz, T A, T out[5]) {
  using S = Sc<T>;
  const T rL = VL[0], uL = VL[1], vL = VL[2], wL = VL[3], pL = VL[4];
  const T rR = VR[0], uR = VR[1], vR = VR[2], wR = VR[3], pR = VR[4];
  const T VnL = S::dot3(nx, uL, ny, vL, nz, wL);
  const T VnR = S::dot3(nx, uR, ny, vR, nz, wR);
  const T riL = S::rcp(rL), riR = S::rcp(rR);
  const T hL = C.g_gm1 * pL * riL + S::halve(S::dot3(uL, uL, vL, vL, wL, wL));
  const T hR = C.g_gm1 * pR * riR + S::halve(S::dot3(uR, uR, vR, vR, wR, wR));

  // Roe averages: R = sqrt(rho_R/rho_L), rho~ = rho_L R, and
  // phi~ = (phi_L + R phi_R)/(1 + R) = phi_L + beta (phi_R - phi_L) with
  // beta = R/(1 + R): one multiply-add per velocity from the jumps below
  const T dr = rR - rL, du = uR - uL, dv = vR - vL, dw = wR - wL, dp = pR - pL;
  const T Rt = S::sqrt(rR * riL);
  const T rt = rL * Rt;
  const T beta = Rt * S::rcp(C.one + Rt);
  const T ut = uL + beta * du;
  const T vt = vL + beta * dv;
  const T wt = wL + beta * dw;
  const T ht = hL + beta * (hR - hL);
  const T q2h = S::halve(S::dot3(ut, ut, vt, vt, wt, wt));
  const T c2 = C.gm1 * (ht - q2h);
  const T ct = S::sqrt(c2);
  const T ic2 = S::rcp(c2);
  // the averaged normal velocity by the same weights: n . u~ = VnL + beta dVn
  const T dVn = VnR - VnL;
  const T Vnt = VnL + beta * dVn;

  T l1 = S::abs(Vnt - ct), l2 = S::abs(Vnt), l5 = S::abs(Vnt + ct);
  if (C.k_fix()) {
    const T delta = C.harten * ct;
    l1 = entropy_fixed(C, l1, delta);
    l5 = entropy_fixed(C, l5, delta);
    if (C.k_fixall()) l2 = entropy_fixed(C, l2, delta);
  }
  // the factor |S|/2 of the face flux is folded into the wave strengths and
  // the mass fluxes (F^ |S| is then a sum of products with no final
  // scaling: five binary64 instructions fewer per face)
  const T hA = S::halve(A);
  const T rcd = rt * ct * dVn;
  const T hic2A = S::halve(ic2) * hA;
  const T l2A = l2 * hA;
  const T a1 = l1 * (dp - rcd) * hic2A;
  const T a5 = l5 * (dp + rcd) * hic2A;
  const T a2 = l2A * (dr - dp * ic2);
  const T a3 = l2A * rt;
  const T a15 = a1 + a5, d51 = (a5 - a1) * ct;

  // dissipation (|dF1| + |dF234| + |dF5|) |S|/2 (the velocity components
  // take a15 + a2 = D0 times the averaged velocity)
  T D0 = a15 + a2;
  T D1 = S::dot3(D0, ut, d51, nx, a3, du - nx * dVn);
  T D2 = S::dot3(D0, vt, d51, ny, a3, dv - ny * dVn);
  T D3 = S::dot3(D0, wt, d51, nz, a3, dw - nz * dVn);
  T D4 = S::dot4(a15, ht, d51, Vnt, a2, q2h, a3, S::dot4(ut, du, vt, dv, wt, dw, -Vnt, dVn));

  const T mLA = (rL * hA) * VnL, mRA = (rR * hA) * VnR;
  const T pLRA = (pL + pR) * hA;
  out[0] = (mLA + mRA) - D0;
  out[1] = S::dot3m(mLA, uL, mRA, uR, nx, pLRA, D1);
  out[2] = S::dot3m(mLA, vL, mRA, vR, ny, pLRA, D2);
  out[3] = S::dot3m(mLA, wL, mRA, wR, nz, pLRA, D3);
  out[4] = S::dot2m(mLA, hL, mRA, hR, D4);
}

// ---------------------------------------------------------------------------
// Flux-vector splittings (Section 2 lists them beside Roe): F^ = F+(V_L) +
// F-(V_R), times the face area.
// ---------------------------------------------------------------------------

// van Leer: split by the normal Mach number; sgn = +1 (F+) or -1 (F-)
template <class T, class CC>
__device__ __forceinline__ void vanleer_part(const CC& C, const T V[5], T nx, T ny, T nz, int sgn,
                                             T F[5]) {
  using S = Sc<T>;
  const T r = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
  const T c = S::sqrt(C.g * p * S::rcp(r));
  const T Vn = nx * u + ny * v + nz * w;
  const T M = Vn * S::rcp(c);
  const bool sup = S::ge(M, 1.0f), sub = S::le(M, -1.0f);
  if (sup || sub) {
    if (sup == (sgn > 0)) {
      const T ht = C.g_gm1 * p * S::rcp(r) + C.half * (u * u + v * v + w * w);
      const T m = r * Vn;
      F[0] = m; F[1] = m * u + nx * p; F[2] = m * v + ny * p; F[3] = m * w + nz * p; F[4] = m * ht;
    } else {
#pragma unroll
      for (int n = 0; n < 5; ++n) F[n] = S::c(0.0);
    }
    return;
  }
  const T one = sgn > 0 ? C.one : S::c(-1.0);
  const T mp = M + one;
  const T fm = one * r * c * mp * mp * C.quarter;
  const T c2 = C.two * c;
  const T a = (one * c2 - Vn) * C.ig;
  const T e = C.gm1 * Vn + one * c2;
  F[0] = fm;
  F[1] = fm * (u + nx * a);
  F[2] = fm * (v + ny * a);
  F[3] = fm * (w + nz * a);
  F[4] = fm * (e * e * C.i2g2m1 + C.half * (u * u + v * v + w * w - Vn * Vn));
}

// Steger-Warming: eigenvalue splitting l+- = (l +- |l|)/2
template <class T, class CC>
__device__ __forceinline__ void steger_warming_part(const CC& C, const T V[5], T nx, T ny, T nz, int sgn,
                                                    T F[5]) {
  using S = Sc<T>;
  const T r = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
  const T c = S::sqrt(C.g * p * S::rcp(r));
  const T Vn = nx * u + ny * v + nz * w;
  const T one = sgn > 0 ? C.one : S::c(-1.0);
  const T l1 = C.half * ((Vn - c) + one * S::abs(Vn - c));
  const T l2 = C.half * (Vn + one * S::abs(Vn));
  const T l5 = C.half * ((Vn + c) + one * S::abs(Vn + c));
  const T q2 = u * u + v * v + w * w;
  const T H = c * c * C.igm1 + C.half * q2;
  const T k = r * C.i2g;
  const T a2 = C.gm1x2 * l2;
  const T l15 = l1 + l5, d51 = (l5 - l1) * c;
  F[0] = k * (a2 + l15);
  F[1] = k * (a2 * u + l15 * u + d51 * nx);
  F[2] = k * (a2 * v + l15 * v + d51 * ny);
  F[3] = k * (a2 * w + l15 * w + d51 * nz);
  F[4] = k * (a2 * (C.half * q2) + l15 * H + d51 * Vn);
}

template <class T, class CC>
__device__ __forceinline__ void face_riemann(const CC& C, const T VL[5], const T VR[5], T nx, T ny, T nz, T A,
                                             T out[5]) {
  if (C.k_flux() == 0) { roe_flux(C, VL, VR, nx, ny, nz, A, out); return; }
  T Fp[5], Fm[5];
  if (C.k_flux() == 1) {
    vanleer_part(C, VL, nx, ny, nz, +1, Fp);
    vanleer_part(C, VR, nx, ny, nz, -1, Fm);
  } else {
    steger_warming_part(C, VL, nx, ny, nz, +1, Fp);
    steger_warming_part(C, VR, nx, ny, nz, -1, Fm);
  }
#pragma unroll
  for (int n = 0; n < 5; ++n) out[n] = (Fp[n] + Fm[n]) * A;
}

// ---------------------------------------------------------------------------
// Overwritten boundary-face fluxes (Section 7.2, V7), times the face area.
// ---------------------------------------------------------------------------

// slip wall: pressure only, p_w = (3 p_1 - p_2)/2 from the two nearest cells
template <class T, class CC>
__device__ __forceinline__ void wall_face_flux(const CC& C, T p1, T p2, T nx, T ny, T nz, T A, T out[5]) {
  using S = Sc<T>;
  const T pwA = (S::c(1.5) * p1 - S::c(0.5) * p2) * A;
  out[0] = S::c(0.0);
  out[1] = pwA * nx;
  out[2] = pwA * ny;
  out[3] = pwA * nz;
  out[4] = S::c(0.0);
}

// farfield: the physical normal flux F(V_b).n of the boundary state (the ghost)
template <class T, class CC>
__device__ __forceinline__ void normal_face_flux(const CC& C, const T V[5], T nx, T ny, T nz, T A, T out[5]) {
  using S = Sc<T>;
  const T r = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
  const T Vn = nx * u + ny * v + nz * w;
  const T ht = C.g_gm1 * p * S::rcp(r) + C.half * (u * u + v * v + w * w);
  const T m = r * Vn;
  out[0] = m * A;
  out[1] = (m * u + nx * p) * A;
  out[2] = (m * v + ny * p) * A;
  out[3] = (m * w + nz * p) * A;
  out[4] = (m * ht) * A;
}

// Full face: reconstruct the 5 primitive components along the stencil
// c0..c3 (pointers to component 0 of each cell, components `cs` apart) and
// evaluate the Roe flux times area.
template <class T, class CC>
__device__ __forceinline__ void face_flux(const CC& C, const T* c0, const T* c1, const T* c2,
                                          const T* c3, int cs, T nx, T ny, T nz, T A, T out[5]) {
  T VL[5], VR[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) muscl(C, c0[n * cs], c1[n * cs], c2[n * cs], c3[n * cs], VL[n], VR[n]);
  face_riemann(C, VL, VR, nx, ny, nz, A, out);
}

// Full face from stencil values held in registers: v[c][n] is component n of
// stencil cell c (c = 0..3 along the face normal).
template <class T, class CC>
__device__ __forceinline__ void face_flux_vals(const CC& C, const T (&v)[4][5], T nx, T ny, T nz, T A,
                                               T out[5]) {
  T VL[5], VR[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) muscl(C, v[0][n], v[1][n], v[2][n], v[3][n], VL[n], VR[n]);
  face_riemann(C, VL, VR, nx, ny, nz, A, out);
}
