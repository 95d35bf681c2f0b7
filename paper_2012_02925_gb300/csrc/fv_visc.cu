// Laminar viscous terms (Section 2) for the binary64 and double-float forms:
// F_v.S = (0, tau.S, Theta.S) with Stokes's-hypothesis stresses
// tau = mu (grad u + grad u^T - 2/3 div u I), Theta = tau.u_f + k grad T,
// k = mu c_p / Pr, T = p / (rho R), and face gradients by Green's theorem
// over the auxiliary volume between the two cell centres (Section 2: the
// viscous flux needs a wider stencil than the inviscid one):
//   grad phi = (phi_R - phi_L) G_a + D_b G_b + D_c G_c,
//   D_b = ((phi_L,b+ - phi_L,b-) + (phi_R,b+ - phi_R,b-)) / 4,
// G_d = the mean of the two cells' averaged face vectors of family d divided
// by their mean volume (a static per-face record built with the metrics).
//
// One kernel per stage computes every face of every direction.  A CTA owns
// 32 x 8 face positions of a block and marches them along k through a ring
// of three padded-cell planes in shared memory holding (u, v, w, T) of each
// cell, computed once per plane from the conserved state; each thread then
// evaluates the xi, eta and zeta faces at its position (the faces on the
// low sides of its cell, plus the high-side faces of the block's last cells)
// from the ring.  The conserved state of the next plane is copied
// asynchronously into a staging plane while the faces are computed.  The
// fluxes go to per-face records (4 values, 32 bytes) that the fused stage
// kernel subtracts from each face's inviscid flux.
#include <cuda_pipeline.h>

#include "fv_arith.cuh"
#include "fv_internal.h"

namespace {

// storage type of each arithmetic form with its loads and stores
template <class T> struct VT;
template <> struct VT<double> {
  using type = double;
  static __device__ __forceinline__ double get(double v) { return v; }
  static __device__ __forceinline__ double put(double v) { return v; }
  static __device__ __forceinline__ void st4(double* p, long long f, const double v[4]) {
    double2* q = reinterpret_cast<double2*>(p + 4 * f);
    q[0] = make_double2(v[0], v[1]);
    q[1] = make_double2(v[2], v[3]);
  }
  static __device__ __forceinline__ void ld12(const double* p, long long f, double o[12]) {
    const double2* q = reinterpret_cast<const double2*>(p + 12 * f);
#pragma unroll
    for (int x = 0; x < 6; ++x) {
      const double2 a = __ldg(q + x);
      o[2 * x] = a.x;
      o[2 * x + 1] = a.y;
    }
  }
};
template <> struct VT<df64> {
  using type = float2;
  static __device__ __forceinline__ df64 get(float2 v) { return mk(v.x, v.y); }
  static __device__ __forceinline__ float2 put(df64 v) { return make_float2(v.hi, v.lo); }
  static __device__ __forceinline__ void st4(float2* p, long long f, const df64 v[4]) {
    float4* q = reinterpret_cast<float4*>(p + 4 * f);
    q[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    q[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
  }
  static __device__ __forceinline__ void ld12(const float2* p, long long f, df64 o[12]) {
    const float4* q = reinterpret_cast<const float4*>(p + 12 * f);
#pragma unroll
    for (int x = 0; x < 6; ++x) {
      const float4 a = __ldg(q + x);
      o[2 * x] = mk(a.x, a.y);
      o[2 * x + 1] = mk(a.z, a.w);
    }
  }
};

constexpr int TX = FV_VISC_TX, TY = FV_VISC_TY, KC = FV_VISC_KC;
constexpr int W = TX + 2, H = TY + 2;

// the viscous constants in the arithmetic of the form
template <class T>
struct ViscK {
  T mu, kfac, itref, tref_s, s_suth;
};

// F_v.S of one face from the differences of (u, v, w, T) along the face's
// own axis (da) and the tangential axes (db, dc), the face values of the
// velocity (uf) and of T (Tf), and the face's geometry record g
// (G_a, G_b, G_c, S).  tau is symmetric: its six distinct entries are formed
// once and mu multiplies tau.S, not each entry; the sums of products are
// compensated dot products in double-float.
template <class T, bool THREE>
__device__ __forceinline__ void face_flux(const ViscK<T>& K, int suth, const T da[4], const T db[4], const T dc[4],
                                          const T uf[3], T Tf, const T g[12], T fv[4]) {
  using S = Sc<T>;
  T grad[4][3];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int x = 0; x < 3; ++x)
      grad[m][x] = THREE ? S::dot3(da[m], g[x], db[m], g[3 + x], dc[m], g[6 + x]) : S::dot2(da[m], g[x], db[m], g[3 + x]);
  T mu = K.mu;
  if (suth) {
    const T tr = Tf * K.itref;
    mu = mu * tr * S::sqrt(tr) * K.tref_s * S::rcp(Tf + K.s_suth);
  }
  const T d23 = S::c(2.0 / 3.0) * (grad[0][0] + grad[1][1] + grad[2][2]);
  const T t00 = S::twice(grad[0][0]) - d23, t11 = S::twice(grad[1][1]) - d23, t22 = S::twice(grad[2][2]) - d23;
  const T t01 = grad[0][1] + grad[1][0], t02 = grad[0][2] + grad[2][0], t12 = grad[1][2] + grad[2][1];
  fv[0] = mu * S::dot3(t00, g[9], t01, g[10], t02, g[11]);
  fv[1] = mu * S::dot3(t01, g[9], t11, g[10], t12, g[11]);
  fv[2] = mu * S::dot3(t02, g[9], t12, g[10], t22, g[11]);
  fv[3] = S::dot4(fv[0], uf[0], fv[1], uf[1], fv[2], uf[2], mu * K.kfac,
                  S::dot3(grad[3][0], g[9], grad[3][1], g[10], grad[3][2], g[11]));
}

template <class T, bool THREE>
__global__ void __launch_bounds__(TX * TY, 2) visc_faces_kernel(const FvViscArgs a) {
  using S = Sc<T>;
  using V = VT<T>;
  using MT = typename V::type;
  constexpr int NP = THREE ? 3 : 1;
  __shared__ MT ring[NP][4][H][W];
  __shared__ double stg[THREE ? 5 : 1][THREE ? H * W : 1];   // staged state of the next plane

  const FvViscTile tile = a.tiles[blockIdx.x];
  const FvBlockDev& B = a.blocks[tile.block];
  const int ni = B.ni, nj = B.nj, nk = B.nk;
  const long long qoff = B.qoff, jst = B.jstride, kst = B.kstride, pl = B.plane;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i = tile.i0 + tx, j = tile.j0 + ty;
  const int k0 = tile.k0, k1 = THREE ? min(tile.k0 + KC, nk + 1) : 1;
  const double* __restrict__ q = a.q;
  const T gm1 = S::c(a.vp.gamma - 1.0), iR = S::c(1.0 / a.vp.r_gas), zero = S::c(0.0);
  ViscK<T> K;
  K.mu = S::c(a.vp.mu);
  K.kfac = S::c(a.vp.kfac);
  K.itref = S::c(1.0 / a.vp.t_ref);
  K.tref_s = S::c(a.vp.t_ref + a.vp.s_suth);
  K.s_suth = S::c(a.vp.s_suth);
  const int suth = a.vp.sutherland;

  // plane kk's cells handled by this thread: e = tid + r * TX * TY; the
  // cell's state index, or -1 outside the padded block
  constexpr int NE = (W * H + TX * TY - 1) / (TX * TY);
  auto cell_of = [&](int e, int kk) -> long long {
    const int x = e % W, y = e / W;
    const int ci = tile.i0 - 1 + x, cj = tile.j0 - 1 + y;
    if (e >= W * H || kk < -1 || kk > nk || ci > ni || cj > nj) return -1;
    return qoff + (long long)(kk + 2) * kst + (long long)(cj + 2) * jst + (ci + 2);
  };
  // Double-float: T goes into the ring as T - tref, tref a binary32 value
  // (the T of the tile's first interior cell).  The T gradient divides
  // differences of T by the cell size, so double-float's ~48-bit
  // significand of T itself cost the 128^3 laminar energy residual 2e-12 of
  // its terms' scale.  The deviation is formed without that loss: its
  // numerator rho^2 R (T - tref) = (gamma - 1)(E rho - |m|^2 / 2) - tref R
  // rho^2 in binary64 (products only: no binary64 division), then divided by
  // rho^2 R in double-float, whose relative error now applies to the small
  // deviation (binary64 T: no reference).
  constexpr bool TDEV = std::is_same<T, df64>::value;
  const double gm1d = a.vp.gamma - 1.0;
  double tref_d = 0.0;
  if constexpr (TDEV) {
    const int ri = min(tile.i0, ni - 1), rj = min(tile.j0, nj - 1), rk = THREE ? min(k0, nk - 1) : 0;
    const long long c = qoff + (long long)(rk + 2) * kst + (long long)(rj + 2) * jst + (ri + 2);
    const double r = q[c], m1 = q[c + pl], m2 = q[c + 2 * pl], m3 = q[c + 3 * pl];
    tref_d = (double)(float)(gm1d * fma(q[c + 4 * pl], r, -0.5 * (m1 * m1 + m2 * m2 + m3 * m3)) /
                             (r * r * a.vp.r_gas));
  }
  const double tref_rd = tref_d * a.vp.r_gas;
  const T tref = S::from_d(tref_d);
  // (u, v, w, T) of one cell from its conserved state into ring slot sl;
  // the never-filled corners of the ghost frame (density 0) and cells
  // outside the padded block get zeros: no face reads them
  auto put_vars = [&](int sl, int e, bool in, double r, double m1, double m2, double m3, double en) {
    T u = zero, v = zero, w = zero, t = zero;
    if (in && r > 0.0) {
      const T rho = S::from_d(r);
      const T ri = S::rcp(rho);
      u = S::from_d(m1) * ri;
      v = S::from_d(m2) * ri;
      w = S::from_d(m3) * ri;
      if constexpr (TDEV) {
        const double num = fma(gm1d, fma(en, r, -0.5 * (m1 * m1 + m2 * m2 + m3 * m3)), -(tref_rd * r) * r);
        t = S::from_d(num) * ri * ri * iR;
      } else {
        const T p = gm1 * (S::from_d(en) - S::c(0.5) * rho * (u * u + v * v + w * w));
        t = p * ri * iR;
      }
    }
    MT* d = &ring[sl][0][0][0] + e;
    d[0] = V::put(u);
    d[H * W] = V::put(v);
    d[2 * H * W] = V::put(w);
    d[3 * H * W] = V::put(t);
  };
  auto load_plane = [&](int sl, int kk) {
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      const int e = tid + r * TX * TY;
      if (e >= W * H) break;
      const long long c = cell_of(e, kk);
      if (c >= 0) put_vars(sl, e, true, q[c], q[c + pl], q[c + 2 * pl], q[c + 3 * pl], q[c + 4 * pl]);
      else put_vars(sl, e, false, 0.0, 0.0, 0.0, 0.0, 0.0);
    }
  };
  // the same in two halves: the asynchronous copy of the state into the
  // staging plane, then (after the faces) the conversion of the cells this
  // thread copied
  auto prefetch_plane = [&](int kk) {
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      const int e = tid + r * TX * TY;
      const long long c = cell_of(e, kk);
      if (c < 0) continue;
#pragma unroll
      for (int n = 0; n < 5; ++n) __pipeline_memcpy_async(&stg[n][e], q + c + n * pl, sizeof(double));
    }
    __pipeline_commit();
  };
  auto convert_plane = [&](int sl, int kk) {
    __pipeline_wait_prior(0);
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      const int e = tid + r * TX * TY;
      if (e >= W * H) break;
      const bool in = cell_of(e, kk) >= 0;
      put_vars(sl, e, in, in ? stg[0][e] : 0.0, in ? stg[1][e] : 0.0, in ? stg[2][e] : 0.0, in ? stg[3][e] : 0.0,
               in ? stg[4][e] : 0.0);
    }
  };

  if (THREE) {
    for (int kk = k0 - 1; kk <= k0 + 1; ++kk) load_plane((kk + 1) % 3, kk);
  } else {
    load_plane(0, 0);
  }
  __syncthreads();

  constexpr int VS = H * W, SL = 4 * VS;     // variable and ring-slot strides
  for (int k = k0; k < k1; ++k) {
    const int sm = THREE ? k % 3 : 0, s0 = THREE ? (k + 1) % 3 : 0, sp = THREE ? (k + 2) % 3 : 0;
    const bool more = THREE && k + 1 < k1;
    if (more) prefetch_plane(k + 2);      // overlaps the faces below
    // this position's cell (variable 0) and the offsets of the planes k-1
    // and k+1 from it
    const MT* C = &ring[s0][0][ty + 1][tx + 1];
    const int dkm = (sm - s0) * SL, dkp = (sp - s0) * SL;
    // the xi, eta and zeta faces at this position through one copy of the
    // face code (three inlined copies overflow the instruction cache)
#pragma unroll 1
    for (int dir = 0; dir < (THREE ? 3 : 2); ++dir) {
      const bool valid = dir == 0 ? (i <= ni && j < nj && k < nk)
                                  : (dir == 1 ? (i < ni && j <= nj && k < nk) : (i < ni && j < nj && k <= nk));
      if (!valid) continue;
      // L (offset oL) and the tangential neighbours: xi face b = eta,
      // c = zeta; eta face b = xi, c = zeta; zeta face b = xi, c = eta
      const int oL = dir == 0 ? -1 : (dir == 1 ? -W : dkm);
      const int obp = dir == 0 ? W : 1, obm = -obp;
      const int ocp = dir == 2 ? W : dkp, ocm = dir == 2 ? -W : dkm;
      const int ei = ni + (dir == 0), ej = nj + (dir == 1);
      const long long f = B.vface_off[dir] + (long long)i + (long long)ei * (j + (long long)ej * k);
      T g[12];
      V::ld12(reinterpret_cast<const MT*>(a.fgeo[dir]), f, g);
      T da[4], db[4], dc[4], uf[3], Tf;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const MT* c = C + m * VS;
        const T pL = V::get(c[oL]), pR = V::get(c[0]);
        da[m] = pR - pL;
        db[m] = S::quarter((V::get(c[oL + obp]) - V::get(c[oL + obm])) + (V::get(c[obp]) - V::get(c[obm])));
        dc[m] = zero;
        if (THREE)
          dc[m] = S::quarter((V::get(c[oL + ocp]) - V::get(c[oL + ocm])) + (V::get(c[ocp]) - V::get(c[ocm])));
        if (m < 3) uf[m] = S::halve(pL + pR);
        else Tf = TDEV ? S::halve(pL + pR) + tref : S::halve(pL + pR);
      }
      T fv[4];
      face_flux<T, THREE>(K, suth, da, db, dc, uf, Tf, g, fv);
      V::st4(reinterpret_cast<MT*>(a.fv[dir]), f, fv);
    }
    if (more) {
      __syncthreads();
      convert_plane(sm, k + 2);   // plane k-1's slot takes plane k+2
      __syncthreads();
    }
  }
}

}  // namespace

int fv_visc_faces(const FvViscArgs& a, int precision, cudaStream_t s) {
  if (a.ntiles == 0) return 0;
  const dim3 block(TX, TY);
  const bool three = a.vp.dim == 3;
  if (precision == 0) {
    if (three) visc_faces_kernel<double, true><<<a.ntiles, block, 0, s>>>(a);
    else visc_faces_kernel<double, false><<<a.ntiles, block, 0, s>>>(a);
  } else {
    if (three) visc_faces_kernel<df64, true><<<a.ntiles, block, 0, s>>>(a);
    else visc_faces_kernel<df64, false><<<a.ntiles, block, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
