// Reverse-mode (vector-Jacobian) form of one face of the residual.
//
// The forward face is the one of fv_face.cuh: primitive recovery of the four
// stencil cells (Section 2), MUSCL reconstruction with limiter, Eq. (flux) of
// Section 7.2, and Roe's flux times the face area (Section 2).  Given the
// cotangent Fbar of the face flux, face_vjp returns the cotangents of the 20
// conserved inputs (4 cells x 5 variables).  Every intermediate of the forward
// pass is recomputed and then swept backwards, statement by statement.
//
// Written once for an arithmetic type T (fv_arith.cuh): binary64, or
// double-float on the FP32 pipe (~48-bit significand; GB300's FP64 unit runs
// at 1/64 of the binary32 rate, and the sweep costs ~3 forward faces).
//
// The paper has no adjoint; this is the discrete adjoint of its residual.
#pragma once
#include "fv_arith.cuh"

// method parameters (binary64, from the handle)
struct AdjParams {
  double gm1, g_gm1;       // gamma - 1, gamma / (gamma - 1)
  double e4km, e4kp;       // eps/4 (1 - kappa), eps/4 (1 + kappa)
  double harten, va_d2;
  int limiter, fix_all;
};

// the same in the arithmetic type, with the constants the sweep uses
template <class T>
struct AdjC {
  T gm1, g_gm1, e4km, e4kp, harten, va_d2, half, one, two;
  int limiter, fix_all;
  bool fix;
};

template <class T>
__device__ __forceinline__ AdjC<T> adj_consts(const AdjParams& P) {
  using S = Sc<T>;
  AdjC<T> c;
  c.gm1 = S::c(P.gm1);
  c.g_gm1 = S::c(P.g_gm1);
  c.e4km = S::c(P.e4km);
  c.e4kp = S::c(P.e4kp);
  c.harten = S::c(P.harten);
  c.va_d2 = S::c(P.va_d2);
  c.half = S::c(0.5);
  c.one = S::c(1.0);
  c.two = S::c(2.0);
  c.limiter = P.limiter;
  c.fix_all = P.fix_all;
  c.fix = P.harten > 0.0;
  return c;
}

// limited difference phi(a, b) = Psi(a/b) b and its partial derivatives
template <class T>
__device__ __forceinline__ T lim_phi(const AdjC<T>& P, T a, T b, T& da, T& db) {
  using S = Sc<T>;
  if (P.limiter == 0) { da = S::c(0.0); db = P.one; return b; }
  if (P.limiter == 1) {
    // van Leer: 2ab/(a+b) when ab > 0, else 0
    if (S::pos(a * b)) {
      const T s = a + b, is2 = S::rcp(s * s);
      da = S::twice(b * b * is2);
      db = S::twice(a * a * is2);
      return S::twice(a * b) * S::rcp(s);
    }
    da = S::c(0.0); db = S::c(0.0);
    return S::c(0.0);
  }
  // van Albada product form: N / D, N = a^2 b + a b^2, D = a^2 + b^2 + delta^2
  const T N = a * a * b + a * b * b, D = a * a + b * b + P.va_d2, iD = S::rcp(D);
  da = ((S::twice(a * b) + b * b) - S::twice(N * a * iD)) * iD;
  db = ((a * a + S::twice(a * b)) - S::twice(N * b * iD)) * iD;
  return N * iD;
}

template <class T>
struct PrimFwd {
  T r, u, v, w, p, ri, k;
};

template <class T>
__device__ __forceinline__ PrimFwd<T> prim_fwd(const AdjC<T>& P, const T q[5]) {
  using S = Sc<T>;
  PrimFwd<T> s;
  s.r = q[0];
  s.ri = S::rcp(q[0]);
  s.u = q[1] * s.ri;
  s.v = q[2] * s.ri;
  s.w = q[3] * s.ri;
  s.k = s.u * s.u + s.v * s.v + s.w * s.w;
  s.p = P.gm1 * (q[4] - S::halve(q[0] * s.k));
  return s;
}

// qbar += (dV/dq)^T Vbar for V = (rho, u, v, w, p), from the primitives
// alone (rho u = r u etc.), so the conserved inputs need not stay live
template <class T>
__device__ __forceinline__ void prim_bwd(const AdjC<T>& P, const PrimFwd<T>& s, const T Vb[5], T qb[5]) {
  using S = Sc<T>;
  const T pb = Vb[4];
  qb[4] = qb[4] + P.gm1 * pb;
  const T gpb = P.gm1 * s.r * pb;
  const T ub = Vb[1] - gpb * s.u;
  const T vb = Vb[2] - gpb * s.v;
  const T wb = Vb[3] - gpb * s.w;
  qb[1] = qb[1] + ub * s.ri;
  qb[2] = qb[2] + vb * s.ri;
  qb[3] = qb[3] + wb * s.ri;
  // d(1/rho)/d rho = -1/rho^2 against rib = ub rho u + vb rho v + wb rho w
  const T rib = s.r * (ub * s.u + vb * s.v + wb * s.w);
  qb[0] = qb[0] + ((Vb[0] - S::halve(P.gm1 * s.k * pb)) - rib * s.ri * s.ri);
}

template <class T>
__device__ __forceinline__ T fix_fwd(const AdjC<T>& P, T l, T d, bool on, T& dl, T& dd) {
  using S = Sc<T>;
  if (on && S::lt_nonneg(l, d)) {
    const T id = S::rcp(d);
    dl = l * id;
    dd = P.half - S::halve(dl * dl);
    return S::halve((l * l + d * d) * id);
  }
  dl = P.one; dd = S::c(0.0);
  return l;
}

// sign of x as +-1 (x = 0 counts as positive)
template <class T>
__device__ __forceinline__ T sgn(T x) {
  return Sc<T>::sel(Sc<T>::neg(x), Sc<T>::c(-1.0), Sc<T>::c(1.0));
}

// Shared-memory parking of values that are dead between the MUSCL forward
// and the MUSCL reverse (SN > 0: value v of this thread at p[v * SN]); the
// compiler barriers keep the stores before and the loads after the Roe part,
// so those values hold no registers across it.
template <class T>
struct Park {
  static __device__ __forceinline__ void put(T* p, T v) { *p = v; }
  static __device__ __forceinline__ T get(const T* p) { return *p; }
};
template <>
struct Park<df64> {
  static __device__ __forceinline__ void put(df64* p, df64 v) { *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo); }
  static __device__ __forceinline__ df64 get(const df64* p) {
    const float2 f = *reinterpret_cast<const float2*>(p);
    return mk(f.x, f.y);
  }
};
// values parked per thread: r, u, v, w, 1/r, |u|^2 of the four cells, the
// four MUSCL Jacobian coefficients of the five variables and the two MUSCL
// states of the five variables
constexpr int ADJ_PARK = 4 * 6 + 4 * 5 + 2 * 5;

// Face VJP: q[c][n] conserved state of stencil cell c (c = 0..3 along the face
// normal, the face between cells 1 and 2), unit normal n, area A, cotangent Fb
// of the 5 face fluxes (F^ |S|).  Accumulates qb[c][n].  Returns F in F (may be
// used to check the forward).  SN > 0: park (shared memory at park, stride SN).
template <class T, int SN = 0, bool LOCK = false>
__device__ __forceinline__ void face_vjp(const AdjC<T>& P, const T q[4][5], T nx, T ny, T nz, T A, const T Fb[5],
                                         T qb[4][5], T F[5], T* park = nullptr) {
  using S = Sc<T>;
  // ---------------- forward ----------------
  PrimFwd<T> s[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) s[c] = prim_fwd(P, q[c]);
  if constexpr (LOCK) __syncthreads();
  // MUSCL states and their derivatives with respect to the three neighbour
  // differences: VL = V1 + e4km phi(d0, dm) + e4kp phi(dm, d0),
  // VR = V2 - e4kp phi(dp, d0) - e4km phi(d0, dp);
  // jL0 = dVL/dd0, jLm = dVL/ddm, jR0 = dVR/dd0 (sign included), jRp = dVR/ddp
  T VL[5], VR[5], jL0[5], jLm[5], jR0[5], jRp[5];
  auto muscl_n = [&](int n, T& L, T& R, T& j0, T& j1, T& j2, T& j3) {
    const T v0 = n == 0 ? s[0].r : (n == 1 ? s[0].u : (n == 2 ? s[0].v : (n == 3 ? s[0].w : s[0].p)));
    const T v1 = n == 0 ? s[1].r : (n == 1 ? s[1].u : (n == 2 ? s[1].v : (n == 3 ? s[1].w : s[1].p)));
    const T v2 = n == 0 ? s[2].r : (n == 1 ? s[2].u : (n == 2 ? s[2].v : (n == 3 ? s[2].w : s[2].p)));
    const T v3 = n == 0 ? s[3].r : (n == 1 ? s[3].u : (n == 2 ? s[3].v : (n == 3 ? s[3].w : s[3].p)));
    const T dm = v1 - v0, d0 = v2 - v1, dp = v3 - v2;
    T a1, b1, a2, b2, a3, b3, a4, b4;
    const T f1 = lim_phi(P, d0, dm, a1, b1);
    const T f2 = lim_phi(P, dm, d0, a2, b2);
    const T f3 = lim_phi(P, dp, d0, a3, b3);
    const T f4 = lim_phi(P, d0, dp, a4, b4);
    L = v1 + (P.e4km * f1 + P.e4kp * f2);
    R = v2 - (P.e4kp * f3 + P.e4km * f4);
    j0 = P.e4km * a1 + P.e4kp * b2;
    j1 = P.e4km * b1 + P.e4kp * a2;
    j2 = -(P.e4kp * b3 + P.e4km * a4);
    j3 = -(P.e4kp * a3 + P.e4km * b4);
  };
  if constexpr (SN > 0) {
    // one copy of the variable's code, run five times (the unrolled
    // straight-line sweep waits on instruction fetch); its results go to
    // the parked shared memory, the states come back to registers
#pragma unroll 1
    for (int n = 0; n < 5; ++n) {
      T L, R, j0, j1, j2, j3;
      muscl_n(n, L, R, j0, j1, j2, j3);
      Park<T>::put(park + (24 + n) * SN, j0);
      Park<T>::put(park + (29 + n) * SN, j1);
      Park<T>::put(park + (34 + n) * SN, j2);
      Park<T>::put(park + (39 + n) * SN, j3);
      Park<T>::put(park + (44 + n) * SN, L);
      Park<T>::put(park + (49 + n) * SN, R);
    }
#pragma unroll
    for (int n = 0; n < 5; ++n) {
      VL[n] = Park<T>::get(park + (44 + n) * SN);
      VR[n] = Park<T>::get(park + (49 + n) * SN);
    }
  } else {
#pragma unroll
    for (int n = 0; n < 5; ++n) muscl_n(n, VL[n], VR[n], jL0[n], jLm[n], jR0[n], jRp[n]);
  }
  if constexpr (SN > 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Park<T>::put(park + (6 * c + 0) * SN, s[c].r);
      Park<T>::put(park + (6 * c + 1) * SN, s[c].u);
      Park<T>::put(park + (6 * c + 2) * SN, s[c].v);
      Park<T>::put(park + (6 * c + 3) * SN, s[c].w);
      Park<T>::put(park + (6 * c + 4) * SN, s[c].ri);
      Park<T>::put(park + (6 * c + 5) * SN, s[c].k);
    }
    asm volatile("" ::: "memory");
  }
  if constexpr (LOCK) __syncthreads();
  const T rL = VL[0], uL = VL[1], vL = VL[2], wL = VL[3], pL = VL[4];
  const T rR = VR[0], uR = VR[1], vR = VR[2], wR = VR[3], pR = VR[4];
  const T VnL = nx * uL + ny * vL + nz * wL, VnR = nx * uR + ny * vR + nz * wR;
  const T riL = S::rcp(rL), riR = S::rcp(rR);
  const T hL = P.g_gm1 * pL * riL + S::halve(uL * uL + vL * vL + wL * wL);
  const T hR = P.g_gm1 * pR * riR + S::halve(uR * uR + vR * vR + wR * wR);
  const T mL = rL * VnL, mR = rR * VnR;
  const T z = rR * riL;
  const T Rt = S::sqrt(z);
  const T rt = rL * Rt;
  const T w1 = S::rcp(P.one + Rt);
  const T ut = (uL + Rt * uR) * w1, vt = (vL + Rt * vR) * w1, wt = (wL + Rt * wR) * w1;
  const T ht = (hL + Rt * hR) * w1;
  const T q2h = S::halve(ut * ut + vt * vt + wt * wt);
  const T c2 = P.gm1 * (ht - q2h);
  const T ct = S::sqrt(c2);
  const T ic2 = S::rcp(c2);
  const T Vnt = nx * ut + ny * vt + nz * wt;
  const T dr = rR - rL, du = uR - uL, dv = vR - vL, dw = wR - wL, dP = pR - pL, dVn = VnR - VnL;
  const T x1 = Vnt - ct, x2 = Vnt, x5 = Vnt + ct;
  const T la1 = S::abs(x1), la2 = S::abs(x2), la5 = S::abs(x5);
  const bool fix = P.fix;
  const T delta = P.harten * ct;
  T d1l, d1d, d2l, d2d, d5l, d5d;
  const T l1 = fix_fwd(P, la1, delta, fix, d1l, d1d);
  const T l2 = fix_fwd(P, la2, delta, fix && P.fix_all, d2l, d2d);
  const T l5 = fix_fwd(P, la5, delta, fix, d5l, d5d);
  const T rcd = rt * ct * dVn;
  const T hic2 = S::halve(ic2);
  const T a1 = l1 * (dP - rcd) * hic2;
  const T a5 = l5 * (dP + rcd) * hic2;
  const T a2 = l2 * (dr - dP * ic2);
  const T a3 = l2 * rt;
  const T a15 = a1 + a5, d51 = (a5 - a1) * ct;
  const T D0 = a15 + a2;
  const T D1 = a15 * ut + d51 * nx + a2 * ut + a3 * (du - nx * dVn);
  const T D2 = a15 * vt + d51 * ny + a2 * vt + a3 * (dv - ny * dVn);
  const T D3 = a15 * wt + d51 * nz + a2 * wt + a3 * (dw - nz * dVn);
  const T E4 = ut * du + vt * dv + wt * dw - Vnt * dVn;
  const T D4 = a15 * ht + d51 * Vnt + a2 * q2h + a3 * E4;
  const T hA = S::halve(A);
  F[0] = (mL + mR - D0) * hA;
  F[1] = (mL * uL + mR * uR + nx * (pL + pR) - D1) * hA;
  F[2] = (mL * vL + mR * vR + ny * (pL + pR) - D2) * hA;
  F[3] = (mL * wL + mR * wR + nz * (pL + pR) - D3) * hA;
  F[4] = (mL * hL + mR * hR - D4) * hA;
  if constexpr (LOCK) __syncthreads();

  // ---------------- reverse ----------------
  const T G0 = Fb[0] * hA, G1 = Fb[1] * hA, G2 = Fb[2] * hA, G3 = Fb[3] * hA, G4 = Fb[4] * hA;
  T rLb = S::c(0.0), uLb = S::c(0.0), vLb = S::c(0.0), wLb = S::c(0.0), pLb = S::c(0.0), rRb = S::c(0.0), uRb = S::c(0.0), vRb = S::c(0.0), wRb = S::c(0.0), pRb = S::c(0.0);
  T hLb = S::c(0.0), hRb = S::c(0.0), VnLb = S::c(0.0), VnRb = S::c(0.0);
  // central part
  T mLb = G0 + G1 * uL + G2 * vL + G3 * wL + G4 * hL;
  T mRb = G0 + G1 * uR + G2 * vR + G3 * wR + G4 * hR;
  uLb += G1 * mL; vLb += G2 * mL; wLb += G3 * mL; hLb += G4 * mL;
  uRb += G1 * mR; vRb += G2 * mR; wRb += G3 * mR; hRb += G4 * mR;
  const T pnb = nx * G1 + ny * G2 + nz * G3;
  pLb += pnb; pRb += pnb;
  // dissipation, Dn enters with -1
  const T D0b = -G0, D1b = -G1, D2b = -G2, D3b = -G3, D4b = -G4;
  const T a15b = D0b + D1b * ut + D2b * vt + D3b * wt + D4b * ht;
  const T d51b = D1b * nx + D2b * ny + D3b * nz + D4b * Vnt;
  const T a2b = D0b + D1b * ut + D2b * vt + D3b * wt + D4b * q2h;
  const T a3b = D1b * (du - nx * dVn) + D2b * (dv - ny * dVn) + D3b * (dw - nz * dVn) + D4b * E4;
  T utb = D1b * (a15 + a2) + D4b * a3 * du;
  T vtb = D2b * (a15 + a2) + D4b * a3 * dv;
  T wtb = D3b * (a15 + a2) + D4b * a3 * dw;
  T htb = D4b * a15;
  T Vntb = D4b * (d51 - a3 * dVn);
  T q2hb = D4b * a2;
  T dub = D1b * a3 + D4b * a3 * ut;
  T dvb = D2b * a3 + D4b * a3 * vt;
  T dwb = D3b * a3 + D4b * a3 * wt;
  T dVnb = -a3 * (D1b * nx + D2b * ny + D3b * nz + D4b * Vnt);
  T ctb = d51b * (a5 - a1);
  const T a1b = a15b - d51b * ct;
  const T a5b = a15b + d51b * ct;
  T l1b = S::c(0.0), l2b = S::c(0.0), l5b = S::c(0.0), rtb = S::c(0.0), drb = S::c(0.0), dPb = S::c(0.0), ic2b = S::c(0.0), hic2b = S::c(0.0), rcdb = S::c(0.0);
  l2b += a3b * rt; rtb += a3b * l2;
  l2b += a2b * (dr - dP * ic2); drb += a2b * l2; dPb += -a2b * l2 * ic2; ic2b += -a2b * l2 * dP;
  l5b += a5b * (dP + rcd) * hic2; dPb += a5b * l5 * hic2; rcdb += a5b * l5 * hic2; hic2b += a5b * l5 * (dP + rcd);
  l1b += a1b * (dP - rcd) * hic2; dPb += a1b * l1 * hic2; rcdb += -a1b * l1 * hic2; hic2b += a1b * l1 * (dP - rcd);
  ic2b += S::halve(hic2b);
  rtb += rcdb * ct * dVn; ctb += rcdb * rt * dVn; dVnb += rcdb * rt * ct;
  if constexpr (LOCK) __syncthreads();
  // eigenvalue magnitudes with the entropy fix (delta = harten * ct)
  T deltab = l1b * d1d + l2b * d2d + l5b * d5d;
  const T la1b = l1b * d1l, la2b = l2b * d2l, la5b = l5b * d5l;
  ctb += deltab * P.harten;
  const T x1b = la1b * sgn(x1);
  const T x2b = la2b * sgn(x2);
  const T x5b = la5b * sgn(x5);
  Vntb += x1b + x2b + x5b;
  ctb += -x1b + x5b;
  // jumps
  rRb += drb; rLb -= drb;
  uRb += dub; uLb -= dub;
  vRb += dvb; vLb -= dvb;
  wRb += dwb; wLb -= dwb;
  pRb += dPb; pLb -= dPb;
  VnRb += dVnb; VnLb -= dVnb;
  // Roe-averaged normal velocity and sound speed
  utb += nx * Vntb; vtb += ny * Vntb; wtb += nz * Vntb;
  T c2b = -ic2b * ic2 * ic2 + S::halve(ctb * S::rcp(ct));
  htb += P.gm1 * c2b;
  q2hb += -P.gm1 * c2b;
  utb += q2hb * ut; vtb += q2hb * vt; wtb += q2hb * wt;
  T Rtb = S::c(0.0), w1b = S::c(0.0);
  uLb += utb * w1; uRb += utb * Rt * w1; Rtb += utb * uR * w1; w1b += utb * (uL + Rt * uR);
  vLb += vtb * w1; vRb += vtb * Rt * w1; Rtb += vtb * vR * w1; w1b += vtb * (vL + Rt * vR);
  wLb += wtb * w1; wRb += wtb * Rt * w1; Rtb += wtb * wR * w1; w1b += wtb * (wL + Rt * wR);
  hLb += htb * w1; hRb += htb * Rt * w1; Rtb += htb * hR * w1; w1b += htb * (hL + Rt * hR);
  Rtb += -w1b * w1 * w1;
  rLb += rtb * Rt; Rtb += rtb * rL;
  const T zb = S::halve(Rtb * S::rcp(Rt));
  T riLb = zb * rR, riRb = S::c(0.0);
  rRb += zb * riL;
  // mass fluxes and enthalpies
  rLb += mLb * VnL; VnLb += mLb * rL;
  rRb += mRb * VnR; VnRb += mRb * rR;
  pLb += hLb * P.g_gm1 * riL; riLb += hLb * P.g_gm1 * pL;
  uLb += hLb * uL; vLb += hLb * vL; wLb += hLb * wL;
  pRb += hRb * P.g_gm1 * riR; riRb += hRb * P.g_gm1 * pR;
  uRb += hRb * uR; vRb += hRb * vR; wRb += hRb * wR;
  rLb += -riLb * riL * riL;
  rRb += -riRb * riR * riR;
  uLb += nx * VnLb; vLb += ny * VnLb; wLb += nz * VnLb;
  uRb += nx * VnRb; vRb += ny * VnRb; wRb += nz * VnRb;
  // MUSCL reverse
  if constexpr (LOCK) __syncthreads();
  if constexpr (SN > 0) {
    asm volatile("" ::: "memory");
#pragma unroll
    for (int n = 0; n < 5; ++n) {
      jL0[n] = Park<T>::get(park + (24 + n) * SN);
      jLm[n] = Park<T>::get(park + (29 + n) * SN);
      jR0[n] = Park<T>::get(park + (34 + n) * SN);
      jRp[n] = Park<T>::get(park + (39 + n) * SN);
    }
  }
  const T VLb[5] = {rLb, uLb, vLb, wLb, pLb};
  const T VRb[5] = {rRb, uRb, vRb, wRb, pRb};
  T Vb[4][5];
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    const T Lb = VLb[n], Rb = VRb[n];
    const T d0b = Lb * jL0[n] + Rb * jR0[n];
    const T dmb = Lb * jLm[n];
    const T dpb = Rb * jRp[n];
    Vb[0][n] = -dmb;
    Vb[1][n] = Lb + dmb - d0b;
    Vb[2][n] = Rb + d0b - dpb;
    Vb[3][n] = dpb;
  }
  if constexpr (SN > 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      s[c].r = Park<T>::get(park + (6 * c + 0) * SN);
      s[c].u = Park<T>::get(park + (6 * c + 1) * SN);
      s[c].v = Park<T>::get(park + (6 * c + 2) * SN);
      s[c].w = Park<T>::get(park + (6 * c + 3) * SN);
      s[c].ri = Park<T>::get(park + (6 * c + 4) * SN);
      s[c].k = Park<T>::get(park + (6 * c + 5) * SN);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) prim_bwd(P, s[c], Vb[c], qb[c]);
}
