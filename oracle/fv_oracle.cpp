// CPU oracle for the explicit finite-volume Euler residual and Runge-Kutta
// stage of a multi-block structured-grid solver (Xue, Jackson, Roy,
// arXiv 2012.02925).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// restatement of the method that the CUDA library is checked against.  Only
// the tests, the package's smoke check and the benchmark's CPU-baseline leg
// may load it.  It shares no code with the CUDA path.
//
// Every routine is a direct loop over cells or faces in the order the method
// states it; it is templated on the scalar type so that the same arithmetic
// runs in double, in forward-mode dual numbers (for Jacobian-vector products)
// and in an operation-counting type.  Build with -ffp-contract=off so that no
// multiply-add is fused.
//
// Citations (paper sections and equations):
//   * governing weak form, conserved Q and inviscid normal flux: Section 2,
//     Eq. (governing) and the Q / F_{i,n} definitions;
//   * primitive-variable MUSCL reconstruction: Section 2 and Section 7.2 (V4),
//     Eq. (flux), with limiter values Psi^{+/-};
//   * Roe's approximate Riemann flux: Section 2 (flux-difference splitting);
//   * ghost cells for connected boundaries: Section 2 and Section 4;
//   * explicit M-step Runge-Kutta time marching: Section 2;
//   * physical boundaries enforced through ghost cells (slip wall, supersonic
//     inflow, extrapolated outflow, farfield): Section 2 and Section 7.2
//     (V2/V3); wall and farfield face fluxes overwritten after the boundary
//     enforcement: Section 7.2 (V7).
// Points the paper leaves open are fixed as follows:
//   limiter: van Leer Psi(r) = (r+|r|)/(1+|r|) with r = a/b, b guarded to
//     copysign(max(|b|,1e-30), b) (sign(0)=+1); van Albada in the smooth
//     product form Psi(a/b) b = b (a^2 + a b) / (a^2 + b^2 + delta^2);
//     "none" means Psi = 1;
//   entropy fix: Harten's |l| <- (l^2 + d^2)/(2d) when |l| < d, d = harten*c~,
//     on the acoustic eigenvalues (and on V_n as well when fix_all);
//   metrics: face vector S = 1/2 (x_c - x_a) x (x_d - x_b) for the face's
//     nodes a,b,c,d in order; volume = 1/3 sum_faces xbar_f . S_f (outward);
//   residual summation order: xi pair, eta pair, zeta pair, then the source;
//   RK: Q^(m) = Q^(0) - alpha_m dt / Omega R(Q^(m-1));
//   boundaries: ghosts at depth d mirror interior depth d across a slip wall
//     (normal momentum reflected with the boundary face's unit normal); an
//     extrapolated outflow copies the first interior cell into both layers; a
//     supersonic inflow holds the prescribed state; a farfield holds the
//     characteristic state built from the first interior cell and the free
//     stream with the 1D Riemann invariants V_n +- 2c/(gamma-1) along the
//     outward normal (entropy and tangential velocity from the upwind side;
//     all from the interior/free stream when |V_n|/c >= 1 inside);
//   overwritten fluxes: a slip-wall face carries only pressure, p_w S with
//     p_w = (3 p_1 - p_2)/2 from the two nearest interior cells; a farfield
//     face carries the physical flux F(V_b).S of the ghost state.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// scalar types
// ---------------------------------------------------------------------------

struct Dual {           // value + one tangent direction
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual sqrt_(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual abs_(Dual a) { return a.v < 0 ? -a : a; }
inline double val(Dual a) { return a.v; }

inline double sqrt_(double a) { return std::sqrt(a); }
inline double abs_(double a) { return std::fabs(a); }
inline double val(double a) { return a; }

// Operation-counting scalar: every arithmetic operation bumps a counter.
struct OpCount { long add, mul, div, sqrt, abs_, cmp; };
OpCount g_ops;
struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops.add; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops.mul; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops.div; return Cnt(a.v / b.v); }
inline Cnt sqrt_(Cnt a) { ++g_ops.sqrt; return Cnt(std::sqrt(a.v)); }
inline Cnt abs_(Cnt a) { ++g_ops.abs_; return Cnt(std::fabs(a.v)); }
inline double val(Cnt a) { ++g_ops.cmp; return a.v; }

struct Params {
  double gamma, eps, kappa;
  int limiter;        // 0 none (Psi = 1), 1 van Leer, 2 van Albada
  double harten;      // entropy-fix width as a fraction of c~ (0 = off)
  int fix_all;        // also fix |V_n|
  double va_delta2;   // van Albada smoothing delta^2
  int dim;            // 2 or 3
  int flux;           // 0 Roe, 1 van Leer flux-vector splitting, 2 Steger-Warming
  int visc;           // 1: laminar viscous flux (Section 2)
  double mu;          // viscosity (constant), or mu(t_ref) under Sutherland's law
  double prandtl, r_gas;
  int sutherland;
  double t_ref, s_suth;
};

Params unpack(const double* p) {
  Params q;
  q.gamma = p[0]; q.eps = p[1]; q.kappa = p[2]; q.limiter = (int)p[3];
  q.harten = p[4]; q.fix_all = (int)p[5]; q.va_delta2 = p[6]; q.dim = (int)p[7];
  q.flux = (int)p[8];
  q.visc = (int)p[9]; q.mu = p[10]; q.prandtl = p[11]; q.r_gas = p[12];
  q.sutherland = (int)p[13]; q.t_ref = p[14]; q.s_suth = p[15];
  return q;
}

constexpr int G = 2;  // ghost layers

// ---------------------------------------------------------------------------
// Section 2: primitive variables from the conserved vector
// Q = (rho, rho u, rho v, rho w, rho e_t), p = (gamma-1)(rho e_t - rho|u|^2/2)
// ---------------------------------------------------------------------------
template <class T>
void cons_to_prim(const T q[5], double gamma, T V[5]) {
  T rho = q[0];
  T u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
  V[0] = rho; V[1] = u; V[2] = v; V[3] = w;
  V[4] = T(gamma - 1.0) * (q[4] - T(0.5) * rho * (u * u + v * v + w * w));
}

// ---------------------------------------------------------------------------
// Limited difference Psi(a/b) * b.  In Eq. (flux) every limiter value
// multiplies the difference that forms the denominator of its ratio, so each
// of the four limited terms is Psi(a/b) b for a pair of neighbouring
// differences (a, b).
// ---------------------------------------------------------------------------
template <class T>
T limited(const Params& P, T a, T b) {
  if (P.limiter == 0) return b;
  if (P.limiter == 1) {
    T den = b;
    double bv = val(b);
    if (std::fabs(bv) < 1e-30) den = T(bv < 0 ? -1e-30 : 1e-30);
    T r = a / den;
    T ar = abs_(r);
    T psi = (r + ar) / (T(1.0) + ar);
    return psi * b;
  }
  return b * (a * a + a * b) / (a * a + b * b + T(P.va_delta2));
}

// ---------------------------------------------------------------------------
// Eq. (flux): MUSCL extrapolation of one primitive component to face i+1/2
// from V_{i-1}, V_i, V_{i+1}, V_{i+2}.
//   Psi^+_{i-1/2} = Psi(D_{i+1/2}/D_{i-1/2}),  Psi^-_{i+1/2} = Psi(D_{i-1/2}/D_{i+1/2}),
//   Psi^+_{i+1/2} = Psi(D_{i+3/2}/D_{i+1/2}),  Psi^-_{i+3/2} = Psi(D_{i+1/2}/D_{i+3/2}).
// ---------------------------------------------------------------------------
template <class T>
void muscl(const Params& P, T vm1, T v0, T vp1, T vp2, T& L, T& R) {
  T d_m = v0 - vm1;    // D_{i-1/2}
  T d_0 = vp1 - v0;    // D_{i+1/2}
  T d_p = vp2 - vp1;   // D_{i+3/2}
  T e4 = T(P.eps / 4.0);
  T km = T(1.0 - P.kappa), kp = T(1.0 + P.kappa);
  L = v0 + e4 * (km * limited(P, d_0, d_m) + kp * limited(P, d_m, d_0));
  R = vp1 - e4 * (kp * limited(P, d_p, d_0) + km * limited(P, d_0, d_p));
}

template <class T>
T entropy_fix(T lam_abs, T delta) {
  if (val(lam_abs) < val(delta)) return (lam_abs * lam_abs + delta * delta) / (T(2.0) * delta);
  return lam_abs;
}

// ---------------------------------------------------------------------------
// Roe flux-difference splitting (Section 2): F^ = 1/2 (F(V_L).n + F(V_R).n)
// - 1/2 (|dF1| + |dF234| + |dF5|), returned multiplied by the face area |S|.
// F.n is the inviscid normal flux of Section 2: (rho V_n, rho u V_n + n_x p,
// rho v V_n + n_y p, rho w V_n + n_z p, rho h_t V_n).
// ---------------------------------------------------------------------------
template <class T>
void roe_flux(const Params& P, const T VL[5], const T VR[5], const double S[3], T out[5]) {
  const double g = P.gamma;
  double area = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  double nx = S[0] / area, ny = S[1] / area, nz = S[2] / area;

  T rL = VL[0], uL = VL[1], vL = VL[2], wL = VL[3], pL = VL[4];
  T rR = VR[0], uR = VR[1], vR = VR[2], wR = VR[3], pR = VR[4];
  T VnL = T(nx) * uL + T(ny) * vL + T(nz) * wL;
  T VnR = T(nx) * uR + T(ny) * vR + T(nz) * wR;
  T hL = T(g / (g - 1.0)) * pL / rL + T(0.5) * (uL * uL + vL * vL + wL * wL);
  T hR = T(g / (g - 1.0)) * pR / rR + T(0.5) * (uR * uR + vR * vR + wR * wR);

  T FL[5], FR[5];
  FL[0] = rL * VnL;
  FL[1] = rL * uL * VnL + T(nx) * pL;
  FL[2] = rL * vL * VnL + T(ny) * pL;
  FL[3] = rL * wL * VnL + T(nz) * pL;
  FL[4] = rL * hL * VnL;
  FR[0] = rR * VnR;
  FR[1] = rR * uR * VnR + T(nx) * pR;
  FR[2] = rR * vR * VnR + T(ny) * pR;
  FR[3] = rR * wR * VnR + T(nz) * pR;
  FR[4] = rR * hR * VnR;

  // Roe averages
  T Rt = sqrt_(rR / rL);
  T rt = sqrt_(rL * rR);
  T ut = (uL + Rt * uR) / (T(1.0) + Rt);
  T vt = (vL + Rt * vR) / (T(1.0) + Rt);
  T wt = (wL + Rt * wR) / (T(1.0) + Rt);
  T ht = (hL + Rt * hR) / (T(1.0) + Rt);
  T q2t = ut * ut + vt * vt + wt * wt;
  T ct = sqrt_(T(g - 1.0) * (ht - T(0.5) * q2t));
  T Vnt = T(nx) * ut + T(ny) * vt + T(nz) * wt;

  // jumps
  T dr = rR - rL, du = uR - uL, dv = vR - vL, dw = wR - wL, dp = pR - pL;
  T dVn = VnR - VnL;

  // eigenvalue magnitudes with Harten's entropy fix
  T delta = T(P.harten) * ct;
  T l1 = abs_(Vnt - ct), l2 = abs_(Vnt), l5 = abs_(Vnt + ct);
  if (P.harten > 0.0) {
    l1 = entropy_fix(l1, delta);
    l5 = entropy_fix(l5, delta);
    if (P.fix_all) l2 = entropy_fix(l2, delta);
  }

  T c2 = ct * ct;
  T a1 = l1 * (dp - rt * ct * dVn) / (T(2.0) * c2);   // |dF1| strength
  T a5 = l5 * (dp + rt * ct * dVn) / (T(2.0) * c2);   // |dF5| strength
  T a2 = l2 * (dr - dp / c2);                          // entropy wave
  T a3 = l2 * rt;                                      // shear waves

  T dF1[5], dF234[5], dF5[5];
  dF1[0] = a1;
  dF1[1] = a1 * (ut - T(nx) * ct);
  dF1[2] = a1 * (vt - T(ny) * ct);
  dF1[3] = a1 * (wt - T(nz) * ct);
  dF1[4] = a1 * (ht - Vnt * ct);
  dF5[0] = a5;
  dF5[1] = a5 * (ut + T(nx) * ct);
  dF5[2] = a5 * (vt + T(ny) * ct);
  dF5[3] = a5 * (wt + T(nz) * ct);
  dF5[4] = a5 * (ht + Vnt * ct);
  dF234[0] = a2;
  dF234[1] = a2 * ut + a3 * (du - T(nx) * dVn);
  dF234[2] = a2 * vt + a3 * (dv - T(ny) * dVn);
  dF234[3] = a2 * wt + a3 * (dw - T(nz) * dVn);
  dF234[4] = a2 * (T(0.5) * q2t) + a3 * (ut * du + vt * dv + wt * dw - Vnt * dVn);

  for (int n = 0; n < 5; ++n) {
    T Fh = T(0.5) * (FL[n] + FR[n]) - T(0.5) * (dF1[n] + dF234[n] + dF5[n]);
    out[n] = Fh * T(area);
  }
}

// ---------------------------------------------------------------------------
// Flux-vector splittings, the other two face fluxes SENSEI offers (Section 2):
// F^ = F+(V_L) + F-(V_R), times the face area.
// ---------------------------------------------------------------------------

// physical normal flux F.n of Section 2
template <class T>
void normal_flux(const Params& P, const T V[5], double nx, double ny, double nz, T F[5]) {
  T r = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
  T Vn = T(nx) * u + T(ny) * v + T(nz) * w;
  T ht = T(P.gamma / (P.gamma - 1.0)) * p / r + T(0.5) * (u * u + v * v + w * w);
  F[0] = r * Vn;
  F[1] = r * u * Vn + T(nx) * p;
  F[2] = r * v * Vn + T(ny) * p;
  F[3] = r * w * Vn + T(nz) * p;
  F[4] = r * ht * Vn;
}

// van Leer (1982): Mach-number splitting; sign = +1 for F+, -1 for F-
template <class T>
void vanleer_part(const Params& P, const T V[5], double nx, double ny, double nz, int sign, T F[5]) {
  const double g = P.gamma;
  T r = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
  T c = sqrt_(T(g) * p / r);
  T Vn = T(nx) * u + T(ny) * v + T(nz) * w;
  T M = Vn / c;
  if (val(M) >= 1.0 || val(M) <= -1.0) {
    const bool whole = (val(M) >= 1.0) == (sign > 0);
    if (whole) { normal_flux(P, V, nx, ny, nz, F); }
    else { for (int n = 0; n < 5; ++n) F[n] = T(0.0); }
    return;
  }
  T s = T((double)sign);
  T mp = M + s;                                   // M +- 1
  T fm = s * r * c * mp * mp / T(4.0);            // +- rho c (M +- 1)^2 / 4
  T a = (T(0.0) - Vn + s * T(2.0) * c) / T(g);    // (-V_n +- 2c) / gamma
  T e = T(g - 1.0) * Vn + s * T(2.0) * c;         // (gamma-1) V_n +- 2c
  F[0] = fm;
  F[1] = fm * (u + T(nx) * a);
  F[2] = fm * (v + T(ny) * a);
  F[3] = fm * (w + T(nz) * a);
  F[4] = fm * (e * e / T(2.0 * (g * g - 1.0)) + T(0.5) * (u * u + v * v + w * w - Vn * Vn));
}

// Steger and Warming (1981): eigenvalue splitting l+- = (l +- |l|)/2 of
// l1 = V_n - c, l2 = V_n, l5 = V_n + c
template <class T>
void steger_warming_part(const Params& P, const T V[5], double nx, double ny, double nz, int sign, T F[5]) {
  const double g = P.gamma;
  T r = V[0], u = V[1], v = V[2], w = V[3], p = V[4];
  T c = sqrt_(T(g) * p / r);
  T Vn = T(nx) * u + T(ny) * v + T(nz) * w;
  T s = T((double)sign);
  T l1 = T(0.5) * ((Vn - c) + s * abs_(Vn - c));
  T l2 = T(0.5) * (Vn + s * abs_(Vn));
  T l5 = T(0.5) * ((Vn + c) + s * abs_(Vn + c));
  T q2 = u * u + v * v + w * w;
  T H = c * c / T(g - 1.0) + T(0.5) * q2;
  T k = r / T(2.0 * g);
  T a2 = T(2.0 * (g - 1.0)) * l2;
  F[0] = k * (a2 + l1 + l5);
  F[1] = k * (a2 * u + l1 * (u - T(nx) * c) + l5 * (u + T(nx) * c));
  F[2] = k * (a2 * v + l1 * (v - T(ny) * c) + l5 * (v + T(ny) * c));
  F[3] = k * (a2 * w + l1 * (w - T(nz) * c) + l5 * (w + T(nz) * c));
  F[4] = k * (a2 * (T(0.5) * q2) + l1 * (H - c * Vn) + l5 * (H + c * Vn));
}

template <class T>
void face_flux_fn(const Params& P, const T VL[5], const T VR[5], const double S[3], T out[5]) {
  if (P.flux == 0) { roe_flux(P, VL, VR, S, out); return; }
  double area = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  double nx = S[0] / area, ny = S[1] / area, nz = S[2] / area;
  T Fp[5], Fm[5];
  if (P.flux == 1) {
    vanleer_part(P, VL, nx, ny, nz, +1, Fp);
    vanleer_part(P, VR, nx, ny, nz, -1, Fm);
  } else {
    steger_warming_part(P, VL, nx, ny, nz, +1, Fp);
    steger_warming_part(P, VR, nx, ny, nz, -1, Fm);
  }
  for (int n = 0; n < 5; ++n) out[n] = (Fp[n] + Fm[n]) * T(area);
}

// ---------------------------------------------------------------------------
// block geometry helpers
// ---------------------------------------------------------------------------
struct Blk {
  int ni, nj, nk;
  long sx, sy, sz;     // ghosted strides (i, j, k)
  long plane;          // ghosted cells per variable
  Blk(int a, int b, int c) : ni(a), nj(b), nk(c) {
    sx = 1; sy = a + 2 * G; sz = (long)(a + 2 * G) * (b + 2 * G);
    plane = sz * (c + 2 * G);
  }
  long at(int i, int j, int k) const { return (long)(k + G) * sz + (long)(j + G) * sy + (i + G); }
};

inline void cross_half(const double* xa, const double* xb, const double* xc, const double* xd, double* S) {
  double d1[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
  double d2[3] = {xd[0] - xb[0], xd[1] - xb[1], xd[2] - xb[2]};
  S[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
  S[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
  S[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
}

// Physical boundary kinds (codes shared with the boundary tables).
enum { BC_FIXED = 0, BC_SUPERSONIC_INFLOW = 1, BC_EXTRAPOLATE = 2, BC_SLIP_WALL = 3, BC_FARFIELD = 4,
       BC_NOSLIP_WALL = 5 };

// Slip-wall face flux (Section 7.2, V7): pressure only, p_w S.
template <class T>
void wall_flux(T p1, T p2, const double S[3], T out[5]) {
  T pw = T(1.5) * p1 - T(0.5) * p2;
  out[0] = T(0.0);
  out[1] = pw * T(S[0]);
  out[2] = pw * T(S[1]);
  out[3] = pw * T(S[2]);
  out[4] = T(0.0);
}

// Farfield face flux (Section 7.2, V7): F(V_b).S of the boundary state.
template <class T>
void farfield_flux(const Params& P, const T Vb[5], const double S[3], T out[5]) {
  const double a = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
  normal_flux(P, Vb, S[0] / a, S[1] / a, S[2] / a, out);
  for (int n = 0; n < 5; ++n) out[n] = out[n] * T(a);
}

// ---------------------------------------------------------------------------
// Laminar viscous flux (Section 2): F_v.n = (0, tau.n, Theta.n) with tau by
// Stokes's hypothesis and Theta = tau.u + k grad T (heat conduction and the
// work of the viscous stresses), k = mu c_p / Pr, c_p = gamma R/(gamma-1),
// T = p / (rho R); mu constant or by Sutherland's law.  Face gradients by
// Green's theorem over the auxiliary volume between the two cell centres
// (Section 2: "a Green's theorem approach" with a wider stencil).
// ---------------------------------------------------------------------------
template <class T>
T viscosity(const Params& P, T temp) {
  if (!P.sutherland) return T(P.mu);
  const T tr = temp / T(P.t_ref);
  return T(P.mu) * tr * sqrt_(tr) * T(P.t_ref + P.s_suth) / (temp + T(P.s_suth));
}

// Cell geometry of the auxiliary volumes: per cell of the block padded by one
// layer, Omega and the cell-averaged face vectors Sbar_d = (S_d,lo + S_d,hi)/2
// of the three face families; 10 planes of (ni+2)(nj+2)(nk+2) values.
struct Geo {
  const double* g;
  long np;                 // cells per plane
  int pi, pj;              // padded extents in i, j
  long at(int i, int j, int k) const { return ((long)(k + 1) * pj + (j + 1)) * pi + (i + 1); }
};

// Viscous flux times area of the face between cells L and R along axis a
// (cL, cR: ghosted state indices; sb, sc: ghosted strides of the tangential
// axes b, c; gL, gR: padded geometry indices), primitives V.
template <class T>
void viscous_face(const Params& P, const Blk& B, const std::vector<T>& V, const Geo& G, long cL, long cR, long sb,
                  long sc, long gL, long gR, int a, int b, int c, const double S[3], T out[5]) {
  const double R = P.r_gas;
  auto temp = [&](long x) { return V[4 * B.plane + x] / (V[x] * T(R)); };
  auto phi = [&](int m, long x) { return m < 3 ? V[(1 + m) * B.plane + x] : temp(x); };
  // auxiliary volume: Omega_f and the face vectors of its three families
  const double Om = 0.5 * (G.g[gL] + G.g[gR]);
  double A[3][3];
  for (int d = 0; d < 3; ++d)
    for (int x = 0; x < 3; ++x) A[d][x] = 0.5 * (G.g[(1 + 3 * d + x) * G.np + gL] + G.g[(1 + 3 * d + x) * G.np + gR]);
  // gradients of u, v, w, T
  T grad[4][3];
  for (int m = 0; m < 4; ++m) {
    const T da = phi(m, cR) - phi(m, cL);
    const T db = T(0.25) * ((phi(m, cL + sb) - phi(m, cL - sb)) + (phi(m, cR + sb) - phi(m, cR - sb)));
    T dc = T(0.0);
    if (P.dim == 3) dc = T(0.25) * ((phi(m, cL + sc) - phi(m, cL - sc)) + (phi(m, cR + sc) - phi(m, cR - sc)));
    for (int x = 0; x < 3; ++x) {
      T gx = da * T(A[a][x]) + db * T(A[b][x]);
      if (P.dim == 3) gx = gx + dc * T(A[c][x]);
      grad[m][x] = gx / T(Om);
    }
  }
  // face values
  T uf[3];
  for (int x = 0; x < 3; ++x) uf[x] = T(0.5) * (V[(1 + x) * B.plane + cL] + V[(1 + x) * B.plane + cR]);
  const T Tf = T(0.5) * (temp(cL) + temp(cR));
  const T mu = viscosity(P, Tf);
  const T kcond = mu * T(P.gamma * R / (P.gamma - 1.0) / P.prandtl);
  const T div = grad[0][0] + grad[1][1] + grad[2][2];
  T tau[3][3];
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 3; ++y) {
      T t = grad[x][y] + grad[y][x];
      if (x == y) t = t - T(2.0 / 3.0) * div;
      tau[x][y] = mu * t;
    }
  out[0] = T(0.0);
  T energy = T(0.0);
  for (int x = 0; x < 3; ++x) {
    const T f = tau[x][0] * T(S[0]) + tau[x][1] * T(S[1]) + tau[x][2] * T(S[2]);
    out[1 + x] = f;
    energy = energy + f * uf[x];
  }
  out[4] = energy + kcond * (grad[3][0] * T(S[0]) + grad[3][1] * T(S[1]) + grad[3][2] * T(S[2]));
}

// bcode: the six face maps of the block (imin, imax, jmin, jmax, kmin, kmax;
// each indexed by the two tangential cell indices in (i,j,k) order, first
// fastest) or nullptr; a slip-wall or farfield code replaces that boundary
// face's flux.
template <class T>
void residual_block(const Params& P, const Blk& B, const double* Sxi, const double* Seta,
                    const double* Szeta, const double* vol, const T* q, const double* src, T* R,
                    const signed char* const* bcode = nullptr, const double* geo = nullptr) {
  const int ni = B.ni, nj = B.nj, nk = B.nk;
  // primitives of every cell, ghosts included
  std::vector<T> V(5 * B.plane);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < B.plane; ++c) {
    T qc[5], vc[5];
    for (int n = 0; n < 5; ++n) qc[n] = q[n * B.plane + c];
    // cells that hold no data (edges/corners of the ghost frame) may be zero
    if (val(qc[0]) == 0.0) { for (int n = 0; n < 5; ++n) V[n * B.plane + c] = T(0.0); continue; }
    cons_to_prim(qc, P.gamma, vc);
    for (int n = 0; n < 5; ++n) V[n * B.plane + c] = vc[n];
  }
  const long nfx = (long)(ni + 1), nfy = (long)(nj + 1);
  const long n_xi = (long)nk * nj * nfx, n_eta = (long)nk * nfy * ni, n_zeta = (long)(nk + 1) * nj * ni;
  std::vector<T> Fx(5 * n_xi), Fy(5 * n_eta), Fz(P.dim == 3 ? 5 * n_zeta : 0);

  // code of the boundary face at tangential position (t0, t1) of block face bf
  auto code_at = [&](int bf, int t0, int t1) -> int {
    if (!bcode || !bcode[bf]) return BC_FIXED;
    const int ext0 = bf < 2 ? nj : ni;
    return bcode[bf][(long)t1 * ext0 + t0];
  };

  // face fluxes in one direction: face f between cells f-1 and f along the
  // axis; stencil cells cm2 .. cm2 + 3 stride.  side: 0 on the block's min
  // face (interior cells at cm2 + 2, 3 strides, first ghost at cm2 + stride),
  // 1 on its max face (interior at cm2 + stride, cm2; ghost at cm2 + 2 stride)
  auto face = [&](long cm2, long stride, const double* Sarr, long nfaces, long fidx, T* F, int code,
                  int side) {
    T out[5];
    double S[3] = {Sarr[fidx], Sarr[nfaces + fidx], Sarr[2 * nfaces + fidx]};
    if (code == BC_SLIP_WALL || code == BC_NOSLIP_WALL) {
      const long c1 = side == 0 ? cm2 + 2 * stride : cm2 + stride;
      const long c2 = side == 0 ? cm2 + 3 * stride : cm2;
      wall_flux(V[4 * B.plane + c1], V[4 * B.plane + c2], S, out);
    } else if (code == BC_FARFIELD) {
      const long g1 = side == 0 ? cm2 + stride : cm2 + 2 * stride;
      T Vb[5];
      for (int n = 0; n < 5; ++n) Vb[n] = V[n * B.plane + g1];
      farfield_flux(P, Vb, S, out);
    } else {
      T VL[5], VR[5];
      for (int n = 0; n < 5; ++n) {
        const T* Vn = &V[n * B.plane];
        muscl(P, Vn[cm2], Vn[cm2 + stride], Vn[cm2 + 2 * stride], Vn[cm2 + 3 * stride], VL[n], VR[n]);
      }
      face_flux_fn(P, VL, VR, S, out);
    }
    for (int n = 0; n < 5; ++n) F[n * nfaces + fidx] = out[n];
  };

#pragma omp parallel for schedule(static)
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i <= ni; ++i) {
        long f = ((long)k * nj + j) * nfx + i;
        int code = i == 0 ? code_at(0, j, k) : (i == ni ? code_at(1, j, k) : BC_FIXED);
        face(B.at(i - 2, j, k), B.sx, Sxi, n_xi, f, Fx.data(), code, i == 0 ? 0 : 1);
      }
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j <= nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long f = ((long)k * nfy + j) * ni + i;
        int code = j == 0 ? code_at(2, i, k) : (j == nj ? code_at(3, i, k) : BC_FIXED);
        face(B.at(i, j - 2, k), B.sy, Seta, n_eta, f, Fy.data(), code, j == 0 ? 0 : 1);
      }
  if (P.dim == 3) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nk; ++k)
      for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
          long f = ((long)k * nj + j) * ni + i;
          int code = k == 0 ? code_at(4, i, j) : (k == nk ? code_at(5, i, j) : BC_FIXED);
          face(B.at(i, j, k - 2), B.sz, Szeta, n_zeta, f, Fz.data(), code, k == 0 ? 0 : 1);
        }
  }
  // viscous face fluxes (each face once), when the laminar terms are on
  std::vector<T> Vx, Vy, Vz;
  const bool visc = P.visc && geo;
  if (visc) {
    Vx.assign(5 * n_xi, T(0.0));
    Vy.assign(5 * n_eta, T(0.0));
    if (P.dim == 3) Vz.assign(5 * n_zeta, T(0.0));
    Geo Gm{geo, (long)(ni + 2) * (nj + 2) * (nk + 2), ni + 2, nj + 2};
    auto vface = [&](int a, int i, int j, int k, long nfaces, long fidx, const double* Sarr, T* F) {
      // cells L (one step back along a) and R = (i, j, k)
      const long sa = a == 0 ? B.sx : (a == 1 ? B.sy : B.sz);
      const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
      const long sb = b == 0 ? B.sx : B.sy, sc = c == 1 ? B.sy : B.sz;
      const long cR = B.at(i, j, k), cL = cR - sa;
      const long gR = Gm.at(i, j, k);
      const long gL = gR - (a == 0 ? 1 : (a == 1 ? (long)(ni + 2) : (long)(ni + 2) * (nj + 2)));
      double S[3] = {Sarr[fidx], Sarr[nfaces + fidx], Sarr[2 * nfaces + fidx]};
      T out[5];
      viscous_face(P, B, V, Gm, cL, cR, sb, sc, gL, gR, a, b, c, S, out);
      for (int n = 0; n < 5; ++n) F[n * nfaces + fidx] = out[n];
    };
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j < nj; ++j)
        for (int i = 0; i <= ni; ++i) vface(0, i, j, k, n_xi, ((long)k * nj + j) * nfx + i, Sxi, Vx.data());
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j <= nj; ++j)
        for (int i = 0; i < ni; ++i) vface(1, i, j, k, n_eta, ((long)k * nfy + j) * ni + i, Seta, Vy.data());
    if (P.dim == 3) {
#pragma omp parallel for schedule(static)
      for (int k = 0; k <= nk; ++k)
        for (int j = 0; j < nj; ++j)
          for (int i = 0; i < ni; ++i) vface(2, i, j, k, n_zeta, ((long)k * nj + j) * ni + i, Szeta, Vz.data());
    }
  }

  // Eq. (governing), discretely: R = sum over faces of (F_i - F_v) |S|
  // (outward) - S Omega; per cell the inviscid pairs (xi, eta, zeta), then
  // the viscous pairs, then the source
  const long ncell = (long)ni * nj * nk;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long c = ((long)k * nj + j) * ni + i;
        long fx = ((long)k * nj + j) * nfx + i;
        long fy = ((long)k * nfy + j) * ni + i;
        long fz = ((long)k * nj + j) * ni + i;
        for (int n = 0; n < 5; ++n) {
          T r = (Fx[n * n_xi + fx + 1] - Fx[n * n_xi + fx]) +
                (Fy[n * n_eta + fy + ni] - Fy[n * n_eta + fy]);
          if (P.dim == 3) r = r + (Fz[n * n_zeta + fz + (long)ni * nj] - Fz[n * n_zeta + fz]);
          if (visc) {
            T rv = (Vx[n * n_xi + fx + 1] - Vx[n * n_xi + fx]) + (Vy[n * n_eta + fy + ni] - Vy[n * n_eta + fy]);
            if (P.dim == 3) rv = rv + (Vz[n * n_zeta + fz + (long)ni * nj] - Vz[n * n_zeta + fz]);
            r = r - rv;
          }
          if (src) r = r - T(src[n * ncell + c] * vol[c]);
          R[n * ncell + c] = r;
        }
      }
}

// One connection: ghosts of dst face at depth d <- src interior cells at depth d.
template <class T>
void exchange_one(const int* dims, const long* offs, T* q, const int* c) {
  int db = c[0], df = c[1], dlo0 = c[2], dlo1 = c[3], dhi0 = c[4], dhi1 = c[5];
  int sb = c[6], sf = c[7], slo0 = c[8], slo1 = c[9], t0 = c[10], t1 = c[11];
  Blk D(dims[3 * db], dims[3 * db + 1], dims[3 * db + 2]);
  Blk S(dims[3 * sb], dims[3 * sb + 1], dims[3 * sb + 2]);
  int da = df / 2, sa = sf / 2;
  int dext[3] = {D.ni, D.nj, D.nk}, sext[3] = {S.ni, S.nj, S.nk};
  int dtan[2], stan[2], n = 0, m = 0;
  for (int x = 0; x < 3; ++x) { if (x != da) dtan[n++] = x; if (x != sa) stan[m++] = x; }
  T* qd = q + offs[db];
  const T* qs = q + offs[sb];
  for (int b = 0; b < dhi1 - dlo1; ++b)
    for (int a = 0; a < dhi0 - dlo0; ++a)
      for (int d = 1; d <= G; ++d) {
        int dc[3], sc[3];
        dc[dtan[0]] = dlo0 + a;
        dc[dtan[1]] = dlo1 + b;
        dc[da] = (df % 2 == 0) ? -d : dext[da] - 1 + d;
        int st[2] = {slo0, slo1};
        st[std::abs(t0) - 1] += (t0 > 0 ? a : -a);
        st[std::abs(t1) - 1] += (t1 > 0 ? b : -b);
        sc[stan[0]] = st[0];
        sc[stan[1]] = st[1];
        sc[sa] = (sf % 2 == 0) ? d - 1 : sext[sa] - d;
        long di = D.at(dc[0], dc[1], dc[2]);
        long si = S.at(sc[0], sc[1], sc[2]);
        for (int v = 0; v < 5; ++v) qd[v * D.plane + di] = qs[v * S.plane + si];
      }
}

// ---------------------------------------------------------------------------
// Physical boundaries through ghost cells (Section 2; Section 7.2, V2/V3)
// ---------------------------------------------------------------------------

void prim_to_cons_d(const double V[5], double gamma, double q[5]) {
  q[0] = V[0];
  q[1] = V[0] * V[1];
  q[2] = V[0] * V[2];
  q[3] = V[0] * V[3];
  q[4] = V[4] / (gamma - 1.0) + 0.5 * V[0] * (V[1] * V[1] + V[2] * V[2] + V[3] * V[3]);
}

// Farfield boundary state from the interior state Vi, the free stream Vinf
// and the outward unit normal n: 1D Riemann invariants along n.
void farfield_state(double gamma, const double Vi[5], const double Vinf[5], const double n[3], double Vb[5]) {
  const double gm1 = gamma - 1.0;
  const double ci = std::sqrt(gamma * Vi[4] / Vi[0]);
  const double cinf = std::sqrt(gamma * Vinf[4] / Vinf[0]);
  const double vni = Vi[1] * n[0] + Vi[2] * n[1] + Vi[3] * n[2];
  const double vninf = Vinf[1] * n[0] + Vinf[2] * n[1] + Vinf[3] * n[2];
  if (vni >= ci) {          // supersonic outflow: everything from inside
    for (int m = 0; m < 5; ++m) Vb[m] = Vi[m];
    return;
  }
  if (vni <= -ci) {         // supersonic inflow: everything from the free stream
    for (int m = 0; m < 5; ++m) Vb[m] = Vinf[m];
    return;
  }
  const double rp = vni + 2.0 * ci / gm1;       // outgoing invariant (interior)
  const double rm = vninf - 2.0 * cinf / gm1;   // incoming invariant (free stream)
  const double vnb = 0.5 * (rp + rm);
  const double cb = 0.25 * gm1 * (rp - rm);
  const double* ref = vnb >= 0.0 ? Vi : Vinf;   // upwind side
  const double s = ref[4] / std::pow(ref[0], gamma);
  const double rhob = std::pow(cb * cb / (gamma * s), 1.0 / gm1);
  const double vnref = ref[1] * n[0] + ref[2] * n[1] + ref[3] * n[2];
  Vb[0] = rhob;
  for (int m = 0; m < 3; ++m) Vb[1 + m] = ref[1 + m] + (vnb - vnref) * n[m];
  Vb[4] = rhob * cb * cb / gamma;
}

// One boundary patch of a block: ghosts of face bf (0..5) over tangential
// cells [lo0,hi0) x [lo1,hi1) (tangential axes in (i,j,k) order).
// Sface: the block's face-vector array of the face's direction
// ([3][..] as the metrics store it).  state: primitive (rho,u,v,w,p).
void bc_fill_patch(const Params& P, const Blk& B, const double* Sface, int bf, int lo0, int lo1, int hi0,
                   int hi1, int kind, const double* state, double* q) {
  if (kind == BC_FIXED) return;
  const int ax = bf / 2, side = bf % 2;
  const int ext[3] = {B.ni, B.nj, B.nk};
  int tan[2], m = 0;
  for (int x = 0; x < 3; ++x)
    if (x != ax) tan[m++] = x;
  // face-vector array extents: one more face along the face's own axis
  int fe[3] = {B.ni, B.nj, B.nk};
  fe[ax] += 1;
  const long nfaces = (long)fe[0] * fe[1] * fe[2];
  double qs[5];
  if (kind == BC_SUPERSONIC_INFLOW) prim_to_cons_d(state, P.gamma, qs);
  for (int b = lo1; b < hi1; ++b)
    for (int a = lo0; a < hi0; ++a) {
      int c[3];
      c[tan[0]] = a;
      c[tan[1]] = b;
      // boundary face and its unit normal
      int fc[3] = {c[0], c[1], c[2]};
      fc[ax] = side == 0 ? 0 : ext[ax];
      const long fi = ((long)fc[2] * fe[1] + fc[1]) * fe[0] + fc[0];
      double S[3] = {Sface[fi], Sface[nfaces + fi], Sface[2 * nfaces + fi]};
      const double area = std::sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
      double nrm[3] = {S[0] / area, S[1] / area, S[2] / area};
      // first interior cell
      int c1[3] = {c[0], c[1], c[2]};
      c1[ax] = side == 0 ? 0 : ext[ax] - 1;
      const long i1 = B.at(c1[0], c1[1], c1[2]);
      double qb[5];
      if (kind == BC_FARFIELD) {
        double qi[5], Vi[5], Vb[5];
        for (int v = 0; v < 5; ++v) qi[v] = q[v * B.plane + i1];
        cons_to_prim(qi, P.gamma, Vi);
        const double sgn = side == 0 ? -1.0 : 1.0;   // S points +axis; outward on the max face
        double nout[3] = {sgn * nrm[0], sgn * nrm[1], sgn * nrm[2]};
        farfield_state(P.gamma, Vi, state, nout, Vb);
        prim_to_cons_d(Vb, P.gamma, qb);
      }
      for (int d = 1; d <= G; ++d) {
        int cg[3] = {c[0], c[1], c[2]};
        cg[ax] = side == 0 ? -d : ext[ax] - 1 + d;
        const long gi = B.at(cg[0], cg[1], cg[2]);
        if (kind == BC_SUPERSONIC_INFLOW) {
          for (int v = 0; v < 5; ++v) q[v * B.plane + gi] = qs[v];
        } else if (kind == BC_EXTRAPOLATE) {
          for (int v = 0; v < 5; ++v) q[v * B.plane + gi] = q[v * B.plane + i1];
        } else if (kind == BC_FARFIELD) {
          for (int v = 0; v < 5; ++v) q[v * B.plane + gi] = qb[v];
        } else if (kind == BC_NOSLIP_WALL) {
          // adiabatic no-slip wall: the mirrored cell with its velocity reversed
          int cm[3] = {c[0], c[1], c[2]};
          cm[ax] = side == 0 ? d - 1 : ext[ax] - d;
          const long mi = B.at(cm[0], cm[1], cm[2]);
          q[gi] = q[mi];
          for (int x = 1; x <= 3; ++x) q[x * B.plane + gi] = -q[x * B.plane + mi];
          q[4 * B.plane + gi] = q[4 * B.plane + mi];
        } else if (kind == BC_SLIP_WALL) {
          // mirror of the interior cell at the same depth, normal momentum reflected
          int cm[3] = {c[0], c[1], c[2]};
          cm[ax] = side == 0 ? d - 1 : ext[ax] - d;
          const long mi = B.at(cm[0], cm[1], cm[2]);
          double mom[3] = {q[1 * B.plane + mi], q[2 * B.plane + mi], q[3 * B.plane + mi]};
          const double mn = mom[0] * nrm[0] + mom[1] * nrm[1] + mom[2] * nrm[2];
          q[gi] = q[mi];
          for (int x = 0; x < 3; ++x) q[(1 + x) * B.plane + gi] = mom[x] - 2.0 * mn * nrm[x];
          q[4 * B.plane + gi] = q[4 * B.plane + mi];
        }
      }
    }
}

// ---------------------------------------------------------------------------
// Edge ghosts (Section 4 of the paper's GPU history: the corner and edge
// update), needed by the viscous stencil's tangential differences on a
// block's boundary faces: the cells with two ghost coordinates at depth 1.
// An edge cell takes the donor's cell when a connection of one of its two
// faces, extended by one cell along the face, reaches it (connections of the
// lower-numbered axis first, in table order); otherwise the mean of its two
// face-adjacent ghost cells.
// ---------------------------------------------------------------------------

// donor cell of dst tangential coordinates (u0, u1) (patch offsets may fall
// one cell outside the patch) at depth 1 of connection c; false if c does not
// belong to dst face df
bool conn_donor(const int* dims, const int* c, int df, int u0, int u1, int* sb, int* sc) {
  int dlo0 = c[2], dlo1 = c[3];
  int sbk = c[6], sf = c[7], slo0 = c[8], slo1 = c[9], t0 = c[10], t1 = c[11];
  if (c[1] != df) return false;
  const int a = u0 - dlo0, b = u1 - dlo1;
  const int sa = sf / 2;
  int stan[2], m = 0;
  for (int x = 0; x < 3; ++x)
    if (x != sa) stan[m++] = x;
  int st[2] = {slo0, slo1};
  st[std::abs(t0) - 1] += (t0 > 0 ? a : -a);
  st[std::abs(t1) - 1] += (t1 > 0 ? b : -b);
  const int sext[3] = {dims[3 * sbk], dims[3 * sbk + 1], dims[3 * sbk + 2]};
  sc[stan[0]] = st[0];
  sc[stan[1]] = st[1];
  sc[sa] = (sf % 2 == 0) ? 0 : sext[sa] - 1;
  *sb = sbk;
  return true;
}

void edge_fill(int nconn, const int* conns, const int* dims, const long* offs, int dim, double* q, int nblocks) {
  for (int bk = 0; bk < nblocks; ++bk) {
    Blk B(dims[3 * bk], dims[3 * bk + 1], dims[3 * bk + 2]);
    const int ext[3] = {B.ni, B.nj, B.nk};
    double* qb = q + offs[bk];
    const int npairs = dim == 3 ? 3 : 1;
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int pr = 0; pr < npairs; ++pr) {
      const int a = pairs[pr][0], b = pairs[pr][1], cx = 3 - a - b;
      const int nc = dim == 3 ? ext[cx] : 1;
      for (int sa = 0; sa < 2; ++sa)
        for (int sb = 0; sb < 2; ++sb)
          for (int t = 0; t < nc; ++t) {
            int e[3];
            e[a] = sa ? ext[a] : -1;
            e[b] = sb ? ext[b] : -1;
            e[cx] = t;
            bool done = false;
            // connections of face (a, sa) extended along b, then of (b, sb) along a
            for (int pass = 0; pass < 2 && !done; ++pass) {
              const int fa = pass == 0 ? a : b;          // the face's normal axis
              const int face = 2 * fa + (pass == 0 ? sa : sb);
              int tan[2], m = 0;
              for (int x = 0; x < 3; ++x)
                if (x != fa) tan[m++] = x;
              const int u0 = e[tan[0]], u1 = e[tan[1]];
              for (int cn = 0; cn < nconn && !done; ++cn) {
                const int* c = conns + 12 * cn;
                if (c[0] != bk || c[1] != face) continue;
                // the patch extended by one cell along the other edge axis
                int lo[2] = {c[2], c[3]}, hi[2] = {c[4], c[5]};
                const int other = pass == 0 ? b : a;
                for (int x = 0; x < 2; ++x)
                  if (tan[x] == other) { lo[x] -= 1; hi[x] += 1; }
                if (u0 < lo[0] || u0 >= hi[0] || u1 < lo[1] || u1 >= hi[1]) continue;
                int sbk, sc[3];
                conn_donor(dims, c, face, u0, u1, &sbk, sc);
                Blk S(dims[3 * sbk], dims[3 * sbk + 1], dims[3 * sbk + 2]);
                const double* qs = q + offs[sbk];
                const long di = B.at(e[0], e[1], e[2]), si = S.at(sc[0], sc[1], sc[2]);
                for (int v = 0; v < 5; ++v) qb[v * B.plane + di] = qs[v * S.plane + si];
                done = true;
              }
            }
            if (!done) {
              int f1[3] = {e[0], e[1], e[2]}, f2[3] = {e[0], e[1], e[2]};
              f1[b] = sb ? ext[b] - 1 : 0;      // ghost of face (a, sa)
              f2[a] = sa ? ext[a] - 1 : 0;      // ghost of face (b, sb)
              const long di = B.at(e[0], e[1], e[2]), i1 = B.at(f1[0], f1[1], f1[2]), i2 = B.at(f2[0], f2[1], f2[2]);
              for (int v = 0; v < 5; ++v)
                qb[v * B.plane + di] = 0.5 * (qb[v * B.plane + i1] + qb[v * B.plane + i2]);
            }
          }
    }
  }
}

}  // namespace

extern "C" {

// Edge-ghost fill of the packed state (in place), after the connections and
// the physical boundaries.
void oracle_edge_fill(int nconn, const int* conns, const int* dims, const long* offs, int dim, int nblocks,
                      double* q) {
  edge_fill(nconn, conns, dims, offs, dim, q, nblocks);
}

// Residual with the laminar viscous terms: geo is the block's padded
// auxiliary-volume geometry (10 planes of (ni+2)(nj+2)(nk+2): Omega, Sbar_xi,
// Sbar_eta, Sbar_zeta), codes as for oracle_residual_bc or NULL.
void oracle_residual_ns(const double* params, int ni, int nj, int nk, const double* Sxi, const double* Seta,
                        const double* Szeta, const double* vol, const double* geo, const double* q,
                        const double* src, const signed char* codes, double* R) {
  Params P = unpack(params);
  Blk B(ni, nj, nk);
  const signed char* maps[6];
  const long sz[6] = {(long)nj * nk, (long)nj * nk, (long)ni * nk, (long)ni * nk, (long)ni * nj, (long)ni * nj};
  long o = 0;
  for (int f = 0; f < 6; ++f) { maps[f] = codes ? codes + o : nullptr; o += sz[f]; }
  residual_block<double>(P, B, Sxi, Seta, Szeta, vol, q, src, R, codes ? maps : nullptr, geo);
}

// Operation counts of one viscous face (op-counting scalar), as the oracle
// states it: {add, mul, div, sqrt, abs, cmp}.
void oracle_viscous_opcount(const double* params, long* out) {
  Params P = unpack(params);
  P.dim = 3;
  Blk B(5, 5, 5);
  std::vector<Cnt> V(5 * B.plane, Cnt(1.0));
  std::vector<double> g(20, 1.0);
  Geo G{g.data(), 2, 2, 1};
  const double S[3] = {1.0, 0.1, 0.2};
  const long cL = B.at(2, 2, 2);
  Cnt o[5];
  g_ops = OpCount{0, 0, 0, 0, 0, 0};
  viscous_face<Cnt>(P, B, V, G, cL, cL + B.sx, B.sy, B.sz, 0, 1, 0, 1, 2, S, o);
  out[0] = g_ops.add; out[1] = g_ops.mul; out[2] = g_ops.div;
  out[3] = g_ops.sqrt; out[4] = g_ops.abs_; out[5] = g_ops.cmp;
}

// Viscous flux of one face from explicit stencil data, for the closed-form
// checks: V10 = primitives of L, R, L-b, L+b, R-b, R+b, L-c, L+c, R-c, R+c
// (10 x 5), geo2 = Omega, Sbar_xi, Sbar_eta, Sbar_zeta of L then R (2 x 10),
// a = the face's axis, S = its area vector.
void oracle_viscous_face(const double* params, const double* V10, const double* geo2, int a, const double* S,
                         double* out) {
  Params P = unpack(params);
  // a tiny block holding the 10 cells at the offsets the stencil uses
  Blk B(5, 5, 5);
  std::vector<double> V(5 * B.plane, 0.0);
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  int L[3] = {2, 2, 2}, Rc[3] = {2, 2, 2};
  Rc[a] = 3;
  auto put = [&](int slot, const int* cc, int db, int dc) {
    int x[3] = {cc[0], cc[1], cc[2]};
    x[b] += db;
    x[c] += dc;
    const long id = B.at(x[0], x[1], x[2]);
    for (int n = 0; n < 5; ++n) V[n * B.plane + id] = V10[5 * slot + n];
  };
  put(0, L, 0, 0); put(1, Rc, 0, 0);
  put(2, L, -1, 0); put(3, L, 1, 0); put(4, Rc, -1, 0); put(5, Rc, 1, 0);
  put(6, L, 0, -1); put(7, L, 0, 1); put(8, Rc, 0, -1); put(9, Rc, 0, 1);
  std::vector<double> g(20);
  for (int x = 0; x < 10; ++x) { g[2 * x] = geo2[x]; g[2 * x + 1] = geo2[10 + x]; }
  Geo G{g.data(), 2, 2, 1};
  const long sa = a == 0 ? B.sx : (a == 1 ? B.sy : B.sz);
  const long sb = b == 0 ? B.sx : B.sy, sc = c == 1 ? B.sy : B.sz;
  const long cL = B.at(L[0], L[1], L[2]);
  viscous_face(P, B, V, G, cL, cL + sa, sb, sc, 0, 1, a, b, c, S, out);
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

int oracle_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Face vectors and volumes (metric setup).  nodes: (nk+1)(nj+1)(ni+1)x3 or NULL
// for a Cartesian block with spacing h.  Sxi: [3][nk][nj][ni+1] (low face of
// cell i, pointing to +i), Seta: [3][nk][nj+1][ni], Szeta: [3][nk+1][nj][ni],
// vol: [nk][nj][ni].
void oracle_metrics(int ni, int nj, int nk, const double* nodes, const double* h,
                    double* Sxi, double* Seta, double* Szeta, double* vol) {
  const long n_xi = (long)nk * nj * (ni + 1), n_eta = (long)nk * (nj + 1) * ni,
             n_zeta = (long)(nk + 1) * nj * ni;
  if (!nodes) {
    for (long f = 0; f < n_xi; ++f) { Sxi[f] = h[1] * h[2]; Sxi[n_xi + f] = 0.0; Sxi[2 * n_xi + f] = 0.0; }
    for (long f = 0; f < n_eta; ++f) { Seta[f] = 0.0; Seta[n_eta + f] = h[0] * h[2]; Seta[2 * n_eta + f] = 0.0; }
    for (long f = 0; f < n_zeta; ++f) { Szeta[f] = 0.0; Szeta[n_zeta + f] = 0.0; Szeta[2 * n_zeta + f] = h[0] * h[1]; }
    for (long c = 0; c < (long)ni * nj * nk; ++c) vol[c] = h[0] * h[1] * h[2];
    return;
  }
  auto X = [&](int i, int j, int k) { return nodes + 3 * (((long)k * (nj + 1) + j) * (ni + 1) + i); };
  double S[3];
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i <= ni; ++i) {
        long f = ((long)k * nj + j) * (ni + 1) + i;
        cross_half(X(i, j, k), X(i, j + 1, k), X(i, j + 1, k + 1), X(i, j, k + 1), S);
        Sxi[f] = S[0]; Sxi[n_xi + f] = S[1]; Sxi[2 * n_xi + f] = S[2];
      }
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j <= nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long f = ((long)k * (nj + 1) + j) * ni + i;
        cross_half(X(i, j, k), X(i, j, k + 1), X(i + 1, j, k + 1), X(i + 1, j, k), S);
        Seta[f] = S[0]; Seta[n_eta + f] = S[1]; Seta[2 * n_eta + f] = S[2];
      }
  for (int k = 0; k <= nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        long f = ((long)k * nj + j) * ni + i;
        cross_half(X(i, j, k), X(i + 1, j, k), X(i + 1, j + 1, k), X(i, j + 1, k), S);
        Szeta[f] = S[0]; Szeta[n_zeta + f] = S[1]; Szeta[2 * n_zeta + f] = S[2];
      }
  // volume = 1/3 sum over the six faces of (face centroid . outward S)
  auto centroid = [&](const double* a, const double* b, const double* c, const double* d, double* m) {
    for (int x = 0; x < 3; ++x) m[x] = 0.25 * (a[x] + b[x] + c[x] + d[x]);
  };
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        double m[3], acc = 0.0;
        long fl = ((long)k * nj + j) * (ni + 1) + i;
        centroid(X(i, j, k), X(i, j + 1, k), X(i, j + 1, k + 1), X(i, j, k + 1), m);
        acc -= m[0] * Sxi[fl] + m[1] * Sxi[n_xi + fl] + m[2] * Sxi[2 * n_xi + fl];
        centroid(X(i + 1, j, k), X(i + 1, j + 1, k), X(i + 1, j + 1, k + 1), X(i + 1, j, k + 1), m);
        acc += m[0] * Sxi[fl + 1] + m[1] * Sxi[n_xi + fl + 1] + m[2] * Sxi[2 * n_xi + fl + 1];
        long gl = ((long)k * (nj + 1) + j) * ni + i, gh = gl + ni;
        centroid(X(i, j, k), X(i, j, k + 1), X(i + 1, j, k + 1), X(i + 1, j, k), m);
        acc -= m[0] * Seta[gl] + m[1] * Seta[n_eta + gl] + m[2] * Seta[2 * n_eta + gl];
        centroid(X(i, j + 1, k), X(i, j + 1, k + 1), X(i + 1, j + 1, k + 1), X(i + 1, j + 1, k), m);
        acc += m[0] * Seta[gh] + m[1] * Seta[n_eta + gh] + m[2] * Seta[2 * n_eta + gh];
        long zl = ((long)k * nj + j) * ni + i, zh = zl + (long)nj * ni;
        centroid(X(i, j, k), X(i + 1, j, k), X(i + 1, j + 1, k), X(i, j + 1, k), m);
        acc -= m[0] * Szeta[zl] + m[1] * Szeta[n_zeta + zl] + m[2] * Szeta[2 * n_zeta + zl];
        centroid(X(i, j, k + 1), X(i + 1, j, k + 1), X(i + 1, j + 1, k + 1), X(i, j + 1, k + 1), m);
        acc += m[0] * Szeta[zh] + m[1] * Szeta[n_zeta + zh] + m[2] * Szeta[2 * n_zeta + zh];
        vol[((long)k * nj + j) * ni + i] = acc / 3.0;
      }
}

// Connected-boundary ghost fill for every connection (rows of 12 ints, see
// the connection table layout), applied in table order.
void oracle_exchange(int nconn, const int* conns, const int* dims, const long* offs, double* q) {
  for (int c = 0; c < nconn; ++c) exchange_one<double>(dims, offs, q, conns + 12 * c);
}

// Residual of one block: R = sum_faces F^ |S| - S Omega (interior cells,
// [5][nk][nj][ni]).  q: ghosted conserved state [5][nk+4][nj+4][ni+4];
// src: source per unit volume at cell centroids [5][nk][nj][ni] or NULL.
void oracle_residual(const double* params, int ni, int nj, int nk, const double* Sxi,
                     const double* Seta, const double* Szeta, const double* vol,
                     const double* q, const double* src, double* R) {
  Params P = unpack(params);
  Blk B(ni, nj, nk);
  residual_block<double>(P, B, Sxi, Seta, Szeta, vol, q, src, R);
}

// Residual with overwritten boundary-face fluxes: codes holds the six face
// maps of the block concatenated in face order (sizes nj*nk, nj*nk, ni*nk,
// ni*nk, ni*nj, ni*nj; the first tangential index fastest).
void oracle_residual_bc(const double* params, int ni, int nj, int nk, const double* Sxi,
                        const double* Seta, const double* Szeta, const double* vol,
                        const double* q, const double* src, const signed char* codes, double* R) {
  Params P = unpack(params);
  Blk B(ni, nj, nk);
  const signed char* maps[6];
  const long sz[6] = {(long)nj * nk, (long)nj * nk, (long)ni * nk, (long)ni * nk, (long)ni * nj, (long)ni * nj};
  long o = 0;
  for (int f = 0; f < 6; ++f) { maps[f] = codes ? codes + o : nullptr; o += sz[f]; }
  residual_block<double>(P, B, Sxi, Seta, Szeta, vol, q, src, R, codes ? maps : nullptr);
}

// Ghost fill of one physical boundary patch of one block (in place).
void oracle_bc_fill(const double* params, int ni, int nj, int nk, const double* Sxi, const double* Seta,
                    const double* Szeta, int face, int lo0, int lo1, int hi0, int hi1, int kind,
                    const double* state, double* q) {
  Params P = unpack(params);
  Blk B(ni, nj, nk);
  const double* Sface = face / 2 == 0 ? Sxi : (face / 2 == 1 ? Seta : Szeta);
  bc_fill_patch(P, B, Sface, face, lo0, lo1, hi0, hi1, kind, state, q);
}

// Pieces of the boundary treatment for the closed-form checks.
void oracle_farfield_state(double gamma, const double* Vi, const double* Vinf, const double* n, double* Vb) {
  farfield_state(gamma, Vi, Vinf, n, Vb);
}
void oracle_wall_flux(double p1, double p2, const double* S, double* out) { wall_flux<double>(p1, p2, S, out); }

// Jacobian-vector product of the residual: dR = (dR/dq) dq (forward mode).
void oracle_residual_jvp(const double* params, int ni, int nj, int nk, const double* Sxi,
                         const double* Seta, const double* Szeta, const double* vol,
                         const double* q, const double* dq, const double* src, double* R,
                         double* dR) {
  Params P = unpack(params);
  Blk B(ni, nj, nk);
  std::vector<Dual> qd(5 * B.plane), Rd(5L * ni * nj * nk);
  for (long x = 0; x < 5 * B.plane; ++x) qd[x] = Dual(q[x], dq[x]);
  residual_block<Dual>(P, B, Sxi, Seta, Szeta, vol, qd.data(), src, Rd.data());
  for (long x = 0; x < 5L * ni * nj * nk; ++x) { R[x] = Rd[x].v; dR[x] = Rd[x].d; }
}

// Tangent of the ghost exchange (linear: the same copy applied to dq).
void oracle_exchange_tangent(int nconn, const int* conns, const int* dims, const long* offs, double* dq) {
  for (int c = 0; c < nconn; ++c) exchange_one<double>(dims, offs, dq, conns + 12 * c);
}

// RK stage update for one block: Q^(m) = Q^(0) - (alpha dt / Omega) R on the
// interior; ghost cells of the output take Q^(0)'s ghosts.
void oracle_rk_update(int ni, int nj, int nk, double alpha_dt, const double* vol,
                      const double* q0, const double* R, double* qout) {
  Blk B(ni, nj, nk);
  std::memcpy(qout, q0, sizeof(double) * 5 * B.plane);
  const long ncell = (long)ni * nj * nk;
  for (int n = 0; n < 5; ++n)
    for (int k = 0; k < nk; ++k)
      for (int j = 0; j < nj; ++j)
        for (int i = 0; i < ni; ++i) {
          long c = ((long)k * nj + j) * ni + i;
          double fac = alpha_dt / vol[c];
          qout[n * B.plane + B.at(i, j, k)] = q0[n * B.plane + B.at(i, j, k)] - fac * R[n * ncell + c];
        }
}

// Pieces exposed for the closed-form checks.
void oracle_roe_flux(const double* params, const double* VL, const double* VR, const double* S,
                     double* out) {
  Params P = unpack(params);
  roe_flux<double>(P, VL, VR, S, out);
}

// Face flux of the configured function (Roe, van Leer or Steger-Warming).
void oracle_face_flux(const double* params, const double* VL, const double* VR, const double* S, double* out) {
  Params P = unpack(params);
  face_flux_fn<double>(P, VL, VR, S, out);
}

void oracle_muscl(const double* params, const double* v4, double* LR) {
  Params P = unpack(params);
  muscl<double>(P, v4[0], v4[1], v4[2], v4[3], LR[0], LR[1]);
}

double oracle_limited(const double* params, double a, double b) {
  Params P = unpack(params);
  return limited<double>(P, a, b);
}

void oracle_cons_to_prim(double gamma, const double* q, double* V) { cons_to_prim<double>(q, gamma, V); }

// Operation counts of one face evaluation (5 MUSCL components + Roe flux):
// out = {add, mul, div, sqrt, abs, compare}.
void oracle_face_opcount(const double* params, const double* V4x5, const double* S, long* out) {
  Params P = unpack(params);
  g_ops = OpCount{0, 0, 0, 0, 0, 0};
  Cnt VL[5], VR[5], F[5];
  for (int n = 0; n < 5; ++n) {
    Cnt L, R;
    muscl<Cnt>(P, Cnt(V4x5[4 * n]), Cnt(V4x5[4 * n + 1]), Cnt(V4x5[4 * n + 2]), Cnt(V4x5[4 * n + 3]), L, R);
    VL[n] = L; VR[n] = R;
  }
  roe_flux<Cnt>(P, VL, VR, S, F);
  out[0] = g_ops.add; out[1] = g_ops.mul; out[2] = g_ops.div; out[3] = g_ops.sqrt;
  out[4] = g_ops.abs_; out[5] = g_ops.cmp;
}

}  // extern "C"
