// Laminar viscous flux of one face inside the fused stage kernel (Section 2):
// F_v.S = (0, tau.S, Theta.S), tau = mu (grad u + grad u^T - 2/3 div u I),
// Theta = tau.u_f + k grad T, k = mu c_p / Pr, T = p / (rho R), mu constant
// or by Sutherland's law at the face temperature.  The face gradient is
// Green's theorem over the auxiliary volume between the two cell centres
// (Section 2: "a Green's theorem approach" with a wider stencil):
//   grad phi = [(phi_R - phi_L) A_a + D_b A_b + D_c A_c] / Omega_f,
//   D_b = ((phi_L,b+ - phi_L,b-) + (phi_R,b+ - phi_R,b-)) / 4,
// with A_d the mean of the two cells' averaged face vectors of family d and
// Omega_f their mean volume (no c term in 2D).  The stencil's velocities and
// T (as its deviation from a reference of the tile) come from the kernel's
// shared-memory plane ring; the cell geometry records (Omega, Sbar_xi,
// Sbar_eta, Sbar_zeta) from global memory.
#pragma once
#include "fv_arith.cuh"
#include "fv_internal.h"

// storage type of each arithmetic form and a 12-entry geometry record reader
template <class T> struct VGeo;
template <> struct VGeo<double> {
  using type = double;
  static __device__ __forceinline__ void ld10(const double* p, long long c, double o[10]) {
    const double2* q = reinterpret_cast<const double2*>(p + 12 * c);
#pragma unroll
    for (int x = 0; x < 5; ++x) {
      const double2 a = __ldg(q + x);
      o[2 * x] = a.x;
      o[2 * x + 1] = a.y;
    }
  }
};
template <> struct VGeo<df64> {
  using type = float2;
  static __device__ __forceinline__ void ld10(const float2* p, long long c, df64 o[10]) {
    const float4* q = reinterpret_cast<const float4*>(p + 12 * c);
#pragma unroll
    for (int x = 0; x < 5; ++x) {
      const float4 a = __ldg(q + x);
      o[2 * x] = mk(a.x, a.y);
      o[2 * x + 1] = mk(a.z, a.w);
    }
  }
};
template <> struct VGeo<float> {
  using type = float;
  static __device__ __forceinline__ void ld10(const float* p, long long c, float o[10]) {
    const float4* q = reinterpret_cast<const float4*>(p + 12 * c);
    const float4 a = __ldg(q), b = __ldg(q + 1), d = __ldg(q + 2);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    o[8] = d.x; o[9] = d.y;
  }
};

// the viscous constants in the arithmetic of the form
template <class T>
struct ViscC {
  T iR, mu, kfac, itref, tref_s, s_suth;
  int sutherland;
};
template <class T>
__device__ __forceinline__ ViscC<T> make_visc_consts(const FvViscParams& p) {
  using S = Sc<T>;
  ViscC<T> v;
  v.iR = S::c(1.0 / p.r_gas);
  v.mu = S::c(p.mu);
  v.kfac = S::c(p.kfac);
  v.itref = S::c(1.0 / p.t_ref);
  v.tref_s = S::c(p.t_ref + p.s_suth);
  v.s_suth = S::c(p.s_suth);
  v.sutherland = p.sutherland;
  return v;
}

// fv = F_v.S (momentum x, y, z, energy) of the face between L and R along
// axis a; cell pointers address component 0 of the ring cells (rho, u, v, w,
// p, T - tref), components cs apart; gl, gr: geometry records of L and R;
// b_ax, c_ax: the tangential axes; tref: the tile's reference T.
template <class T>
__device__ __forceinline__ void viscous_face_flux(const ViscC<T>& K, const T* L, const T* R, const T* Lbm,
                                                  const T* Lbp, const T* Rbm, const T* Rbp, const T* Lcm,
                                                  const T* Lcp, const T* Rcm, const T* Rcp, int cs, bool three,
                                                  const T gl[10], const T gr[10], int a_ax, int b_ax, int c_ax,
                                                  T Sx, T Sy, T Sz, T tref, T fv[4]) {
  using S = Sc<T>;
  // (u, v, w) are ring variables 1..3, T - tref is variable 5
  auto phi = [&](const T* c, int m) { return c[(m < 3 ? 1 + m : 5) * cs]; };
  const T iOm = S::rcp(S::halve(gl[0] + gr[0]));
  T Aa[3], Ab[3], Ac[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    Aa[x] = S::halve(a_ax == 0 ? gl[1 + x] + gr[1 + x] : (a_ax == 1 ? gl[4 + x] + gr[4 + x] : gl[7 + x] + gr[7 + x]));
    Ab[x] = S::halve(b_ax == 0 ? gl[1 + x] + gr[1 + x] : gl[4 + x] + gr[4 + x]);
    Ac[x] = S::halve(c_ax == 1 ? gl[4 + x] + gr[4 + x] : gl[7 + x] + gr[7 + x]);
  }
  const T quarter = S::c(0.25);
  T grad[4][3];
  T tL = S::c(0.0), tR = S::c(0.0);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const T pL = phi(L, m), pR = phi(R, m);
    if (m == 3) { tL = pL; tR = pR; }
    const T da = pR - pL;
    const T db = quarter * ((phi(Lbp, m) - phi(Lbm, m)) + (phi(Rbp, m) - phi(Rbm, m)));
    T dc = S::c(0.0);
    if (three) dc = quarter * ((phi(Lcp, m) - phi(Lcm, m)) + (phi(Rcp, m) - phi(Rcm, m)));
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      T g = da * Aa[x] + db * Ab[x];
      if (three) g = g + dc * Ac[x];
      grad[m][x] = g * iOm;
    }
  }
  T uf[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) uf[x] = S::halve(L[(1 + x) * cs] + R[(1 + x) * cs]);
  const T Tf = S::halve(tL + tR) + tref;
  T mu = K.mu;
  if (K.sutherland) {
    const T tr = Tf * K.itref;
    mu = mu * tr * S::sqrt(tr) * K.tref_s * S::rcp(Tf + K.s_suth);
  }
  const T div = grad[0][0] + grad[1][1] + grad[2][2];
  const T Sv[3] = {Sx, Sy, Sz};
  T energy = S::c(0.0);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    T f = S::c(0.0);
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      T t = grad[x][y] + grad[y][x];
      if (x == y) t = t - S::c(2.0 / 3.0) * div;
      f = f + mu * t * Sv[y];
    }
    fv[x] = f;
    energy = energy + f * uf[x];
  }
  fv[3] = energy + mu * K.kfac * (grad[3][0] * Sx + grad[3][1] * Sy + grad[3][2] * Sz);
}
