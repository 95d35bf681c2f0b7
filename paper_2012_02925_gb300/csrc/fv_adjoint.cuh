// Reverse-mode (vector-Jacobian) form of one face of the residual, in binary64.
//
// The forward face is the one of fv_face.cuh: primitive recovery of the four
// stencil cells (Section 2), MUSCL reconstruction with limiter, Eq. (flux) of
// Section 7.2, and Roe's flux times the face area (Section 2).  Given the
// cotangent Fbar of the face flux, face_vjp returns the cotangents of the 20
// conserved inputs (4 cells x 5 variables).  Every intermediate of the forward
// pass is recomputed and then swept backwards, statement by statement.
//
// The paper has no adjoint; this is the discrete adjoint of its residual.
#pragma once
#include <cmath>

#ifdef __CUDACC__
#define FVA_HD __host__ __device__ __forceinline__
#else
#define FVA_HD inline
#endif

struct AdjParams {
  double gm1, g_gm1;       // gamma - 1, gamma / (gamma - 1)
  double e4km, e4kp;       // eps/4 (1 - kappa), eps/4 (1 + kappa)
  double harten, va_d2;
  int limiter, fix_all;
};

// limited difference phi(a, b) = Psi(a/b) b and its partial derivatives
FVA_HD double lim_phi(const AdjParams& P, double a, double b, double& da, double& db) {
  if (P.limiter == 0) { da = 0.0; db = 1.0; return b; }
  if (P.limiter == 1) {
    // van Leer: 2ab/(a+b) when ab > 0, else 0
    if (a * b > 0.0) {
      const double s = a + b, is2 = 1.0 / (s * s);
      da = 2.0 * b * b * is2;
      db = 2.0 * a * a * is2;
      return 2.0 * a * b / s;
    }
    da = 0.0; db = 0.0;
    return 0.0;
  }
  // van Albada product form: N / D, N = a^2 b + a b^2, D = a^2 + b^2 + delta^2
  const double N = a * a * b + a * b * b, D = a * a + b * b + P.va_d2, iD = 1.0 / D;
  da = ((2.0 * a * b + b * b) - N * 2.0 * a * iD) * iD;
  db = ((a * a + 2.0 * a * b) - N * 2.0 * b * iD) * iD;
  return N * iD;
}

struct PrimFwd {
  double r, u, v, w, p, ri, k;
};

FVA_HD PrimFwd prim_fwd(const AdjParams& P, const double q[5]) {
  PrimFwd s;
  s.r = q[0];
  s.ri = 1.0 / q[0];
  s.u = q[1] * s.ri;
  s.v = q[2] * s.ri;
  s.w = q[3] * s.ri;
  s.k = s.u * s.u + s.v * s.v + s.w * s.w;
  s.p = P.gm1 * (q[4] - 0.5 * q[0] * s.k);
  return s;
}

// qbar += (dV/dq)^T Vbar for V = (rho, u, v, w, p)
FVA_HD void prim_bwd(const AdjParams& P, const double q[5], const PrimFwd& s, const double Vb[5], double qb[5]) {
  const double pb = Vb[4];
  qb[4] += P.gm1 * pb;
  const double ub = Vb[1] - P.gm1 * s.r * s.u * pb;
  const double vb = Vb[2] - P.gm1 * s.r * s.v * pb;
  const double wb = Vb[3] - P.gm1 * s.r * s.w * pb;
  double rb = Vb[0] - P.gm1 * 0.5 * s.k * pb;
  qb[1] += ub * s.ri;
  qb[2] += vb * s.ri;
  qb[3] += wb * s.ri;
  const double rib = ub * q[1] + vb * q[2] + wb * q[3];
  rb += -rib * s.ri * s.ri;
  qb[0] += rb;
}

FVA_HD double fix_fwd(double l, double d, bool on, double& dl, double& dd) {
  if (on && l < d) {
    dl = l / d;
    dd = 0.5 - l * l / (2.0 * d * d);
    return (l * l + d * d) / (2.0 * d);
  }
  dl = 1.0; dd = 0.0;
  return l;
}

// Face VJP: q[c][n] conserved state of stencil cell c (c = 0..3 along the face
// normal, the face between cells 1 and 2), unit normal n, area A, cotangent Fb
// of the 5 face fluxes (F^ |S|).  Accumulates qb[c][n].  Returns F in F (may be
// used to check the forward).
FVA_HD void face_vjp(const AdjParams& P, const double q[4][5], double nx, double ny, double nz, double A,
                     const double Fb[5], double qb[4][5], double F[5]) {
  // ---------------- forward ----------------
  PrimFwd s[4];
  for (int c = 0; c < 4; ++c) s[c] = prim_fwd(P, q[c]);
  double V[4][5];
  for (int c = 0; c < 4; ++c) { V[c][0] = s[c].r; V[c][1] = s[c].u; V[c][2] = s[c].v; V[c][3] = s[c].w; V[c][4] = s[c].p; }
  double VL[5], VR[5];
  double pa[5][4], pb[5][4];  // limiter partials: [n][phi index] (a and b)
  double dm[5], d0[5], dp[5];
  for (int n = 0; n < 5; ++n) {
    dm[n] = V[1][n] - V[0][n];
    d0[n] = V[2][n] - V[1][n];
    dp[n] = V[3][n] - V[2][n];
    const double f1 = lim_phi(P, d0[n], dm[n], pa[n][0], pb[n][0]);
    const double f2 = lim_phi(P, dm[n], d0[n], pa[n][1], pb[n][1]);
    const double f3 = lim_phi(P, dp[n], d0[n], pa[n][2], pb[n][2]);
    const double f4 = lim_phi(P, d0[n], dp[n], pa[n][3], pb[n][3]);
    VL[n] = V[1][n] + (P.e4km * f1 + P.e4kp * f2);
    VR[n] = V[2][n] - (P.e4kp * f3 + P.e4km * f4);
  }
  const double rL = VL[0], uL = VL[1], vL = VL[2], wL = VL[3], pL = VL[4];
  const double rR = VR[0], uR = VR[1], vR = VR[2], wR = VR[3], pR = VR[4];
  const double VnL = nx * uL + ny * vL + nz * wL, VnR = nx * uR + ny * vR + nz * wR;
  const double riL = 1.0 / rL, riR = 1.0 / rR;
  const double hL = P.g_gm1 * pL * riL + 0.5 * (uL * uL + vL * vL + wL * wL);
  const double hR = P.g_gm1 * pR * riR + 0.5 * (uR * uR + vR * vR + wR * wR);
  const double mL = rL * VnL, mR = rR * VnR;
  const double z = rR * riL;
  const double Rt = sqrt(z);
  const double rt = rL * Rt;
  const double w1 = 1.0 / (1.0 + Rt);
  const double ut = (uL + Rt * uR) * w1, vt = (vL + Rt * vR) * w1, wt = (wL + Rt * wR) * w1;
  const double ht = (hL + Rt * hR) * w1;
  const double q2h = 0.5 * (ut * ut + vt * vt + wt * wt);
  const double c2 = P.gm1 * (ht - q2h);
  const double ct = sqrt(c2);
  const double ic2 = 1.0 / c2;
  const double Vnt = nx * ut + ny * vt + nz * wt;
  const double dr = rR - rL, du = uR - uL, dv = vR - vL, dw = wR - wL, dP = pR - pL, dVn = VnR - VnL;
  const double x1 = Vnt - ct, x2 = Vnt, x5 = Vnt + ct;
  const double la1 = fabs(x1), la2 = fabs(x2), la5 = fabs(x5);
  const bool fix = P.harten > 0.0;
  const double delta = P.harten * ct;
  double d1l, d1d, d2l, d2d, d5l, d5d;
  const double l1 = fix_fwd(la1, delta, fix, d1l, d1d);
  const double l2 = fix_fwd(la2, delta, fix && P.fix_all, d2l, d2d);
  const double l5 = fix_fwd(la5, delta, fix, d5l, d5d);
  const double rcd = rt * ct * dVn;
  const double hic2 = 0.5 * ic2;
  const double a1 = l1 * (dP - rcd) * hic2;
  const double a5 = l5 * (dP + rcd) * hic2;
  const double a2 = l2 * (dr - dP * ic2);
  const double a3 = l2 * rt;
  const double a15 = a1 + a5, d51 = (a5 - a1) * ct;
  const double D0 = a15 + a2;
  const double D1 = a15 * ut + d51 * nx + a2 * ut + a3 * (du - nx * dVn);
  const double D2 = a15 * vt + d51 * ny + a2 * vt + a3 * (dv - ny * dVn);
  const double D3 = a15 * wt + d51 * nz + a2 * wt + a3 * (dw - nz * dVn);
  const double E4 = ut * du + vt * dv + wt * dw - Vnt * dVn;
  const double D4 = a15 * ht + d51 * Vnt + a2 * q2h + a3 * E4;
  const double hA = 0.5 * A;
  F[0] = (mL + mR - D0) * hA;
  F[1] = (mL * uL + mR * uR + nx * (pL + pR) - D1) * hA;
  F[2] = (mL * vL + mR * vR + ny * (pL + pR) - D2) * hA;
  F[3] = (mL * wL + mR * wR + nz * (pL + pR) - D3) * hA;
  F[4] = (mL * hL + mR * hR - D4) * hA;

  // ---------------- reverse ----------------
  const double G0 = Fb[0] * hA, G1 = Fb[1] * hA, G2 = Fb[2] * hA, G3 = Fb[3] * hA, G4 = Fb[4] * hA;
  double rLb = 0, uLb = 0, vLb = 0, wLb = 0, pLb = 0, rRb = 0, uRb = 0, vRb = 0, wRb = 0, pRb = 0;
  double hLb = 0, hRb = 0, VnLb = 0, VnRb = 0;
  // central part
  double mLb = G0 + G1 * uL + G2 * vL + G3 * wL + G4 * hL;
  double mRb = G0 + G1 * uR + G2 * vR + G3 * wR + G4 * hR;
  uLb += G1 * mL; vLb += G2 * mL; wLb += G3 * mL; hLb += G4 * mL;
  uRb += G1 * mR; vRb += G2 * mR; wRb += G3 * mR; hRb += G4 * mR;
  const double pnb = nx * G1 + ny * G2 + nz * G3;
  pLb += pnb; pRb += pnb;
  // dissipation, Dn enters with -1
  const double D0b = -G0, D1b = -G1, D2b = -G2, D3b = -G3, D4b = -G4;
  const double a15b = D0b + D1b * ut + D2b * vt + D3b * wt + D4b * ht;
  const double d51b = D1b * nx + D2b * ny + D3b * nz + D4b * Vnt;
  const double a2b = D0b + D1b * ut + D2b * vt + D3b * wt + D4b * q2h;
  const double a3b = D1b * (du - nx * dVn) + D2b * (dv - ny * dVn) + D3b * (dw - nz * dVn) + D4b * E4;
  double utb = D1b * (a15 + a2) + D4b * a3 * du;
  double vtb = D2b * (a15 + a2) + D4b * a3 * dv;
  double wtb = D3b * (a15 + a2) + D4b * a3 * dw;
  double htb = D4b * a15;
  double Vntb = D4b * (d51 - a3 * dVn);
  double q2hb = D4b * a2;
  double dub = D1b * a3 + D4b * a3 * ut;
  double dvb = D2b * a3 + D4b * a3 * vt;
  double dwb = D3b * a3 + D4b * a3 * wt;
  double dVnb = -a3 * (D1b * nx + D2b * ny + D3b * nz + D4b * Vnt);
  double ctb = d51b * (a5 - a1);
  const double a1b = a15b - d51b * ct;
  const double a5b = a15b + d51b * ct;
  double l1b = 0, l2b = 0, l5b = 0, rtb = 0, drb = 0, dPb = 0, ic2b = 0, hic2b = 0, rcdb = 0;
  l2b += a3b * rt; rtb += a3b * l2;
  l2b += a2b * (dr - dP * ic2); drb += a2b * l2; dPb += -a2b * l2 * ic2; ic2b += -a2b * l2 * dP;
  l5b += a5b * (dP + rcd) * hic2; dPb += a5b * l5 * hic2; rcdb += a5b * l5 * hic2; hic2b += a5b * l5 * (dP + rcd);
  l1b += a1b * (dP - rcd) * hic2; dPb += a1b * l1 * hic2; rcdb += -a1b * l1 * hic2; hic2b += a1b * l1 * (dP - rcd);
  ic2b += 0.5 * hic2b;
  rtb += rcdb * ct * dVn; ctb += rcdb * rt * dVn; dVnb += rcdb * rt * ct;
  // eigenvalue magnitudes with the entropy fix (delta = harten * ct)
  double deltab = l1b * d1d + l2b * d2d + l5b * d5d;
  const double la1b = l1b * d1l, la2b = l2b * d2l, la5b = l5b * d5l;
  ctb += deltab * P.harten;
  const double x1b = la1b * (x1 < 0 ? -1.0 : 1.0);
  const double x2b = la2b * (x2 < 0 ? -1.0 : 1.0);
  const double x5b = la5b * (x5 < 0 ? -1.0 : 1.0);
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
  double c2b = -ic2b * ic2 * ic2 + ctb / (2.0 * ct);
  htb += P.gm1 * c2b;
  q2hb += -P.gm1 * c2b;
  utb += q2hb * ut; vtb += q2hb * vt; wtb += q2hb * wt;
  double Rtb = 0, w1b = 0;
  uLb += utb * w1; uRb += utb * Rt * w1; Rtb += utb * uR * w1; w1b += utb * (uL + Rt * uR);
  vLb += vtb * w1; vRb += vtb * Rt * w1; Rtb += vtb * vR * w1; w1b += vtb * (vL + Rt * vR);
  wLb += wtb * w1; wRb += wtb * Rt * w1; Rtb += wtb * wR * w1; w1b += wtb * (wL + Rt * wR);
  hLb += htb * w1; hRb += htb * Rt * w1; Rtb += htb * hR * w1; w1b += htb * (hL + Rt * hR);
  Rtb += -w1b * w1 * w1;
  rLb += rtb * Rt; Rtb += rtb * rL;
  const double zb = Rtb / (2.0 * Rt);
  double riLb = zb * rR, riRb = 0;
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
  const double VLb[5] = {rLb, uLb, vLb, wLb, pLb};
  const double VRb[5] = {rRb, uRb, vRb, wRb, pRb};
  double Vb[4][5];
  for (int n = 0; n < 5; ++n) {
    double d0b = 0, dmb = 0, dpb = 0;
    const double Lb = VLb[n], Rb = VRb[n];
    // VL = V1 + e4km phi(d0, dm) + e4kp phi(dm, d0)
    d0b += Lb * P.e4km * pa[n][0]; dmb += Lb * P.e4km * pb[n][0];
    dmb += Lb * P.e4kp * pa[n][1]; d0b += Lb * P.e4kp * pb[n][1];
    // VR = V2 - e4kp phi(dp, d0) - e4km phi(d0, dp)
    dpb += -Rb * P.e4kp * pa[n][2]; d0b += -Rb * P.e4kp * pb[n][2];
    d0b += -Rb * P.e4km * pa[n][3]; dpb += -Rb * P.e4km * pb[n][3];
    Vb[0][n] = -dmb;
    Vb[1][n] = Lb + dmb - d0b;
    Vb[2][n] = Rb + d0b - dpb;
    Vb[3][n] = dpb;
  }
  for (int c = 0; c < 4; ++c) prim_bwd(P, q[c], s[c], Vb[c], qb[c]);
}
