// Laminar viscous terms (Section 2): F_v.S = (0, tau.S, Theta.S) with
// Stokes's-hypothesis stresses tau = mu (grad u + grad u^T - 2/3 div u I),
// Theta = tau.u_f + k grad T, k = mu c_p / Pr, T = p / (rho R), and face
// gradients by Green's theorem over the auxiliary volume between the two
// cell centres (Section 2: the viscous flux needs a wider stencil than the
// inviscid one).
//
// Two kernels per stage, each in the arithmetic of the form (binary64,
// double-float, binary32): the face variables (u, v, w, T) of every cell of
// the blocks padded by one layer (ghosts and edge ghosts included), then one
// thread per face of one direction gathering the ten cells of its stencil and
// the auxiliary-volume geometry of its two cells.  The fluxes go to a
// per-face array that the fused stage kernel differences per cell.
#include "fv_arith.cuh"
#include "fv_internal.h"

namespace {

// storage type of each arithmetic form (metrics, geometry, face variables,
// fluxes) with its load and store
template <class T> struct VMetric;
template <> struct VMetric<double> {
  using type = double;
  static __device__ __forceinline__ double ld(const double* m, long long i) { return __ldg(m + i); }
  static __device__ __forceinline__ void st(double* m, long long i, double v) { m[i] = v; }
};
template <> struct VMetric<df64> {
  using type = float2;
  static __device__ __forceinline__ df64 ld(const float2* m, long long i) {
    const float2 v = __ldg(m + i);
    return mk(v.x, v.y);
  }
  static __device__ __forceinline__ void st(float2* m, long long i, df64 v) { m[i] = make_float2(v.hi, v.lo); }
};
template <> struct VMetric<float> {
  using type = float;
  static __device__ __forceinline__ float ld(const float* m, long long i) { return __ldg(m + i); }
  static __device__ __forceinline__ void st(float* m, long long i, float v) { m[i] = v; }
};

// Per-cell records: the face variables (u, v, w, T) and the geometry
// (Omega, Sbar_xi, Sbar_eta, Sbar_zeta, 2 pads) of a padded cell lie
// together, 4 and 12 values of the storage type, read with 16-byte loads.
template <class T> struct VRec;
template <> struct VRec<double> {
  static __device__ __forceinline__ void ld4(const double* p, long long c, double o[4]) {
    const double2* q = reinterpret_cast<const double2*>(p + 4 * c);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  static __device__ __forceinline__ void st4(double* p, long long c, const double v[4]) {
    double2* q = reinterpret_cast<double2*>(p + 4 * c);
    q[0] = make_double2(v[0], v[1]);
    q[1] = make_double2(v[2], v[3]);
  }
  static __device__ __forceinline__ void ld10(const double* p, long long c, double o[10]) {
    const double2* q = reinterpret_cast<const double2*>(p + 12 * c);
#pragma unroll
    for (int x = 0; x < 5; ++x) {
      const double2 a = __ldg(q + x);
      o[2 * x] = a.x; o[2 * x + 1] = a.y;
    }
  }
};
template <> struct VRec<df64> {
  static __device__ __forceinline__ void ld4(const float2* p, long long c, df64 o[4]) {
    const float4* q = reinterpret_cast<const float4*>(p + 4 * c);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    o[0] = mk(a.x, a.y); o[1] = mk(a.z, a.w); o[2] = mk(b.x, b.y); o[3] = mk(b.z, b.w);
  }
  static __device__ __forceinline__ void st4(float2* p, long long c, const df64 v[4]) {
    float4* q = reinterpret_cast<float4*>(p + 4 * c);
    q[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    q[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
  }
  static __device__ __forceinline__ void ld10(const float2* p, long long c, df64 o[10]) {
    const float4* q = reinterpret_cast<const float4*>(p + 12 * c);
#pragma unroll
    for (int x = 0; x < 5; ++x) {
      const float4 a = __ldg(q + x);
      o[2 * x] = mk(a.x, a.y); o[2 * x + 1] = mk(a.z, a.w);
    }
  }
};
template <> struct VRec<float> {
  static __device__ __forceinline__ void ld4(const float* p, long long c, float o[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p + 4 * c));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
  static __device__ __forceinline__ void st4(float* p, long long c, const float v[4]) {
    *reinterpret_cast<float4*>(p + 4 * c) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void ld10(const float* p, long long c, float o[10]) {
    const float4* q = reinterpret_cast<const float4*>(p + 12 * c);
    const float4 a = __ldg(q), b = __ldg(q + 1), d = __ldg(q + 2);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    o[8] = d.x; o[9] = d.y;
  }
};

// last block whose offset (pad_off, or vface_off[dir] when dir >= 0) is <= x
__device__ __forceinline__ int find_block(const FvBlockDev* __restrict__ B, int n, long long x, int dir) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long o = dir < 0 ? B[mid].pad_off : B[mid].vface_off[dir];
    if (o <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// (u, v, w, T) of every padded cell; cells that were never filled (the
// corners of the ghost frame, density 0) get zeros - no stencil reads them
template <class T>
__global__ void visc_vars_kernel(const FvViscArgs a) {
  using S = Sc<T>;
  using V = VMetric<T>;
  typename V::type* wv = reinterpret_cast<typename V::type*>(a.wvar);
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < a.pad_total;
       x += (long long)gridDim.x * blockDim.x) {
    const FvBlockDev& B = a.blocks[find_block(a.blocks, a.nblocks, x, -1)];
    const long long loc = x - B.pad_off;
    const int pi = B.ni + 2, pj = B.nj + 2;
    const int i = (int)(loc % pi) - 1, j = (int)((loc / pi) % pj) - 1, k = (int)(loc / ((long long)pi * pj)) - 1;
    const long long qi = B.qoff + (long long)(k + 2) * B.kstride + (long long)(j + 2) * B.jstride + (i + 2);
    const double r = a.q[qi];
    if (!(r > 0.0)) {
      const T z[4] = {S::c(0.0), S::c(0.0), S::c(0.0), S::c(0.0)};
      VRec<T>::st4(wv, x, z);
      continue;
    }
    const T rho = S::from_d(r);
    const T ri = S::rcp(rho);
    const T u = S::from_d(a.q[qi + B.plane]) * ri;
    const T v = S::from_d(a.q[qi + 2 * B.plane]) * ri;
    const T w = S::from_d(a.q[qi + 3 * B.plane]) * ri;
    const T p = S::c(a.vp.gamma - 1.0) * (S::from_d(a.q[qi + 4 * B.plane]) - S::c(0.5) * rho * (u * u + v * v + w * w));
    const T temp = p * ri * S::c(1.0 / a.vp.r_gas);
    const T rec[4] = {u, v, w, temp};
    VRec<T>::st4(wv, x, rec);
  }
}

template <class T>
__global__ void visc_faces_kernel(const FvViscArgs a, const int dir) {
  using S = Sc<T>;
  using V = VMetric<T>;
  using MT = typename V::type;
  const MT* metric = reinterpret_cast<const MT*>(a.metric);
  const MT* geo = reinterpret_cast<const MT*>(a.geo);    // [pad cells][12]
  const MT* wv = reinterpret_cast<const MT*>(a.wvar);    // [pad cells][4]
  MT* fv = reinterpret_cast<MT*>(a.fv);
  const long long P = a.pad_total;
  const int b_ax = dir == 0 ? 1 : 0, c_ax = dir == 2 ? 1 : 2;
  const bool three = a.vp.dim == 3;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < a.vstride;
       f += (long long)gridDim.x * blockDim.x) {
    const FvBlockDev& B = a.blocks[find_block(a.blocks, a.nblocks, f, dir)];
    const long long loc = f - B.vface_off[dir];
    const int ei = B.ni + (dir == 0), ej = B.nj + (dir == 1);
    const int i = (int)(loc % ei), j = (int)((loc / ei) % ej), k = (int)(loc / ((long long)ei * ej));
    const long long pi = B.ni + 2, pij = pi * (B.nj + 2);
    const long long pR = B.pad_off + (k + 1) * pij + (long long)(j + 1) * pi + (i + 1);
    const long long sa = dir == 0 ? 1 : (dir == 1 ? pi : pij);
    const long long sb = b_ax == 0 ? 1 : pi, sc = c_ax == 1 ? pi : pij;
    const long long pL = pR - sa;
    // the face's area vector
    T Sx, Sy, Sz;
    if (B.cartesian) {
      const T A = S::from_d(B.cart_area[dir]);
      Sx = S::from_d(B.cart_n[dir][0]) * A;
      Sy = S::from_d(B.cart_n[dir][1]) * A;
      Sz = S::from_d(B.cart_n[dir][2]) * A;
    } else {
      const long long fi = 4 * (B.face_off[dir] + loc);     // (n_x, n_y, n_z, |S|) record
      const T A = VMetric<T>::ld(metric, fi + 3);
      Sx = VMetric<T>::ld(metric, fi) * A;
      Sy = VMetric<T>::ld(metric, fi + 1) * A;
      Sz = VMetric<T>::ld(metric, fi + 2) * A;
    }
    // auxiliary volume: mean volume and mean averaged face vectors of L and R
    const T half = S::c(0.5), quarter = S::c(0.25);
    T gl[10], gr[10];
    VRec<T>::ld10(geo, pL, gl);
    VRec<T>::ld10(geo, pR, gr);
    const T iOm = S::rcp(half * (gl[0] + gr[0]));
    // families of the face's own axis (a) and of the tangential axes b, c
    T Aa[3], Ab[3], Ac[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Aa[x] = half * (dir == 0 ? gl[1 + x] + gr[1 + x] : (dir == 1 ? gl[4 + x] + gr[4 + x] : gl[7 + x] + gr[7 + x]));
      Ab[x] = half * (b_ax == 0 ? gl[1 + x] + gr[1 + x] : gl[4 + x] + gr[4 + x]);
      Ac[x] = half * (c_ax == 1 ? gl[4 + x] + gr[4 + x] : gl[7 + x] + gr[7 + x]);
    }
    // the stencil: L, R and their neighbours along b (and c)
    T wL[4], wR[4], wLbm[4], wLbp[4], wRbm[4], wRbp[4];
    VRec<T>::ld4(wv, pL, wL);
    VRec<T>::ld4(wv, pR, wR);
    VRec<T>::ld4(wv, pL - sb, wLbm);
    VRec<T>::ld4(wv, pL + sb, wLbp);
    VRec<T>::ld4(wv, pR - sb, wRbm);
    VRec<T>::ld4(wv, pR + sb, wRbp);
    T wLcm[4], wLcp[4], wRcm[4], wRcp[4];
    if (three) {
      VRec<T>::ld4(wv, pL - sc, wLcm);
      VRec<T>::ld4(wv, pL + sc, wLcp);
      VRec<T>::ld4(wv, pR - sc, wRcm);
      VRec<T>::ld4(wv, pR + sc, wRcp);
    }
    // gradients of u, v, w, T
    T grad[4][3];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const T da = wR[m] - wL[m];
      const T db = quarter * ((wLbp[m] - wLbm[m]) + (wRbp[m] - wRbm[m]));
      T dc = S::c(0.0);
      if (three) dc = quarter * ((wLcp[m] - wLcm[m]) + (wRcp[m] - wRcm[m]));
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        T g = da * Aa[x] + db * Ab[x];
        if (three) g = g + dc * Ac[x];
        grad[m][x] = g * iOm;
      }
    }
    // face values, viscosity, conductivity
    T uf[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) uf[x] = half * (wL[x] + wR[x]);
    const T Tf = half * (wL[3] + wR[3]);
    T mu = S::c(a.vp.mu);
    if (a.vp.sutherland) {
      const T tr = Tf * S::c(1.0 / a.vp.t_ref);
      mu = mu * tr * S::sqrt(tr) * S::c(a.vp.t_ref + a.vp.s_suth) * S::rcp(Tf + S::c(a.vp.s_suth));
    }
    const T kc = mu * S::c(a.vp.kfac);
    const T div = grad[0][0] + grad[1][1] + grad[2][2];
    const T Sv[3] = {Sx, Sy, Sz};
    T energy = S::c(0.0);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      T fx = S::c(0.0);
#pragma unroll
      for (int y = 0; y < 3; ++y) {
        T t = grad[x][y] + grad[y][x];
        if (x == y) t = t - S::c(2.0 / 3.0) * div;
        fx = fx + mu * t * Sv[y];
      }
      V::st(fv, x * a.vstride + f, fx);
      energy = energy + fx * uf[x];
    }
    energy = energy + kc * (grad[3][0] * Sx + grad[3][1] * Sy + grad[3][2] * Sz);
    V::st(fv, 3 * a.vstride + f, energy);
  }
}

int grid_of(long long n, int threads) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > (long long)nsm * 16 ? (long long)nsm * 16 : g));
}

}  // namespace

int fv_visc_vars(const FvViscArgs& a, int precision, cudaStream_t s) {
  const int t = 256, g = grid_of(a.pad_total, t);
  if (precision == 0) visc_vars_kernel<double><<<g, t, 0, s>>>(a);
  else if (precision == 1) visc_vars_kernel<df64><<<g, t, 0, s>>>(a);
  else visc_vars_kernel<float><<<g, t, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int fv_visc_faces(const FvViscArgs& a, int dir, int precision, cudaStream_t s) {
  if (a.vstride == 0) return 0;
  const int t = 128, g = grid_of(a.vstride, t);
  if (precision == 0) visc_faces_kernel<double><<<g, t, 0, s>>>(a, dir);
  else if (precision == 1) visc_faces_kernel<df64><<<g, t, 0, s>>>(a, dir);
  else visc_faces_kernel<float><<<g, t, 0, s>>>(a, dir);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
