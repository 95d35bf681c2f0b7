// Fused residual + Runge-Kutta stage kernel (one template for every form).
//
// One CTA owns a TX x TY column of cells of one block and marches it through
// k.  Per k-plane it
//   1. stages the primitive variables of the newest plane (with a two-cell
//      i/j halo) in shared memory, a ring of four planes for the zeta stencil;
//   2. evaluates every face the tile needs exactly once - the (TX+1) x TY xi
//      faces and TX x (TY+1) eta faces of the plane and the TX x TY zeta faces
//      above it - as one balanced list spread over all threads;
//   3. sums, per cell, R = (xi pair) + (eta pair) + (zeta pair) - S*Omega in
//      that order (Section 2, Eq. (governing) discretised) and applies
//      Q^(m) = Q^(0) - alpha_m dt / Omega * R (explicit M-step RK, Section 2),
//      or writes R itself.
// Nothing per face is written to global memory (the V4 design of Section 7.2
// stored limiter and flux arrays; here they live in registers and shared
// memory only).  Tiles come from a table, so one launch covers every block of
// a multi-block problem.
#pragma once
#include <cuda_pipeline.h>
#include <type_traits>
#include "fv_face.cuh"
#include "fv_viscface.cuh"

template <class T> struct MetricStore;
// Face metrics are one (n_x, n_y, n_z, |S|) record per face, read with
// 16-byte loads (ld4); ld reads one value (the viscous face fluxes).
template <> struct MetricStore<double> {
  using type = double;
  static __device__ __forceinline__ double ld(const double* p, long long i) { return __ldg(p + i); }
  static __device__ __forceinline__ void ld4(const double* p, long long f, double& a, double& b, double& c,
                                             double& d) {
    const double2* q = reinterpret_cast<const double2*>(p + 4 * f);
    const double2 x = __ldg(q), y = __ldg(q + 1);
    a = x.x; b = x.y; c = y.x; d = y.y;
  }
};
template <> struct MetricStore<df64> {
  using type = float2;
  static __device__ __forceinline__ df64 ld(const float2* p, long long i) {
    float2 v = __ldg(p + i);
    return mk(v.x, v.y);
  }
  static __device__ __forceinline__ void ld4(const float2* p, long long f, df64& a, df64& b, df64& c, df64& d) {
    const float4* q = reinterpret_cast<const float4*>(p + 4 * f);
    const float4 x = __ldg(q), y = __ldg(q + 1);
    a = mk(x.x, x.y); b = mk(x.z, x.w); c = mk(y.x, y.y); d = mk(y.z, y.w);
  }
};
template <> struct MetricStore<float> {
  using type = float;
  static __device__ __forceinline__ float ld(const float* p, long long i) { return __ldg(p + i); }
  static __device__ __forceinline__ void ld4(const float* p, long long f, float& a, float& b, float& c, float& d) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p + 4 * f));
    a = x.x; b = x.y; c = x.z; d = x.w;
  }
};

// accumulation type: binary32 face fluxes are summed in double-float
template <class T> struct Acc {
  using type = T;
  static __device__ __forceinline__ T diff(T a, T b) { return a - b; }
  static __device__ __forceinline__ T from_d(double x) { return Sc<T>::from_d(x); }
};
template <> struct Acc<float> {
  using type = df64;
  static __device__ __forceinline__ df64 diff(float a, float b) { return two_sum(a, -b); }
  static __device__ __forceinline__ df64 from_d(double x) { return fv_d2df(x); }
};

// Q^(0) - fac * R in binary64, with fac = alpha dt / Omega
__device__ __forceinline__ double rk_apply(double q0, double alpha_dt, double invvol, double R) {
  return q0 - (alpha_dt * invvol) * R;
}
__device__ __forceinline__ double rk_apply(double q0, df64 fac, df64 R) {
  df64 d = fac * R;
  return q0 - fv_df2d(d);
}

// NV: variables per ring cell (the primitives, and with the fused viscous
// terms a sixth: T - tref); SHARE: the per-cell slope planes (below);
// NSLOT3: planes in the 3-D ring
template <class T, int TX, int TY, int NV = 5, bool SHARE = false, int NSLOT3 = 4>
struct StageSmem {
  static constexpr int W = TX + 4, H = TY + 4, PL = W * H;
  static constexpr int NXI = (TX + 1) * TY, NETA = TX * (TY + 1), NZETA = TX * TY;
  static constexpr int NHX = (TX + 2) * TY, NHY = TX * (TY + 2);
  static constexpr __host__ __device__ size_t typed(bool three_d) {
    return sizeof(T) * (size_t)((three_d ? NSLOT3 : 1) * NV * PL + 5 * NXI + 5 * NETA + (three_d ? 2 * 5 * NZETA : 0) +
                                (SHARE ? 5 * NHX + 5 * NHY + (three_d ? 2 * 5 * NZETA : 0) : 0));
  }
  // with prefetch: + a binary64 staging plane that cp.async fills while the
  // faces of the previous plane are computed
  static constexpr __host__ __device__ size_t bytes(bool three_d, bool prefetch) {
    return ((typed(three_d) + 15) / 16) * 16 + (prefetch && three_d ? sizeof(double) * 5 * PL : 0);
  }
};

// The default scheme (kappa = -1, eps = 1, van Leer) puts V_i + h_i on cell
// i's upper face and V_i - h_i on its lower face, h_i = Psi(a/b) b / 2 of the
// cell's forward difference a and backward difference b: van Leer's Psi
// makes h symmetric in a and b, so the two faces share one limiter
// evaluation, done once per cell and direction in a slope pass before the
// faces (about 0.56 of the per-face stencil's limiter work with the tile
// halo).  Built for the binary64 form, which the FP64 unit bounds (128^3
// block: 0.625 -> 0.716 Gcell/s); the double-float and binary32 forms are
// bound by issue and latency at their occupancy, and the slope planes, the
// third barrier per plane and the lost resident CTA made them slower
// (2.75 -> 2.62 and 9.84 -> 8.26 Gcell/s), so they keep the per-face stencil.
template <class T, bool FAST, bool VISC>
__host__ __device__ constexpr bool stage_share() {
  return FAST && std::is_same<T, double>::value;
}
// planes in the 3-D ring: with shared slopes a pass reads planes k .. k+2
// only, unless a slip-wall zeta face on a block's upper side reads k - 1
template <class T, bool FAST, bool VISC, bool BC>
__host__ __device__ constexpr int stage_slots() {
  return stage_share<T, FAST, VISC>() && !BC ? 3 : 4;
}
template <class T, int TX, int TY, bool FAST, bool VISC, bool BC>
using StageSmemOf = StageSmem<T, TX, TY, (VISC && std::is_same<T, float>::value) ? 6 : 5,
                              stage_share<T, FAST, VISC>(), stage_slots<T, FAST, VISC, BC>()>;

// resident CTAs per SM the register allocation must allow (shared memory
// permits this many for the compiled shapes)
template <class T, int NT, bool VISC>
constexpr int stage_min_ctas() {
  return sizeof(T) == 4 ? (VISC ? (NT <= 128 ? 6 : 3) : (NT <= 128 ? 8 : 4)) : (NT <= 128 ? 4 : (NT <= 256 ? 2 : 1));
}

// VISC: the laminar viscous terms.  The binary32 form evaluates them in the
// face loop (FUSED_VISC); the wider forms subtract the per-face fluxes of the
// separate viscous kernel from each face's inviscid flux in the face loop
// (VISC_PAIRS: one record load per face after the inviscid flux; loaded
// before it, the record's registers slowed the flux by 4 %).  Without VISC
// neither code path exists in the kernel.  BC: the boundary-code lookup and
// the overwritten wall and farfield fluxes; without it (no block has such a
// face) their code is not compiled in, which on the 128^3 block made both
// the double-float and the binary32 kernels 10 % faster.
template <class T, int TX, int TY, int NT, bool DIM3, bool PF, bool FAST, bool VISC, bool BC>
__global__ void __launch_bounds__(NT, (stage_min_ctas<T, NT, VISC>())) fv_stage_kernel(const FvStageArgs args) {
  constexpr bool FUSED_VISC = VISC && std::is_same<T, float>::value;
  constexpr bool VISC_PAIRS = VISC && !std::is_same<T, float>::value;
  using S = Sc<T>;
  using CC = typename std::conditional<FAST, FaceCFast<T>, FaceC<T>>::type;
  using AT = typename Acc<T>::type;
  using MT = typename MetricStore<T>::type;
  constexpr int NV = FUSED_VISC ? 6 : 5;
  constexpr bool SHARE = stage_share<T, FAST, VISC>();
  using SM = StageSmemOf<T, TX, TY, FAST, VISC, BC>;
  constexpr int W = SM::W, PL = SM::PL;
  constexpr int NXI = SM::NXI, NETA = SM::NETA, NZETA = SM::NZETA;
  constexpr int NHX = SM::NHX, NHY = SM::NHY;
  constexpr int NSLOT = DIM3 ? stage_slots<T, FAST, VISC, BC>() : 1;
  constexpr int NFACE = NXI + NETA + (DIM3 ? NZETA : 0);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Vs = reinterpret_cast<T*>(smem_raw);        // [NSLOT][NV][H][W]
  T* Fx = Vs + NSLOT * NV * PL;                   // [5][TY][TX+1]
  T* Fy = Fx + 5 * NXI;                           // [5][TY+1][TX]
  T* Fz = Fy + 5 * NETA;                          // [2][5][TY][TX] (3-D)
  T* Hx = Fz + (DIM3 ? 2 * 5 * NZETA : 0);        // SHARE: [5][TY][TX+2], cells x = -1 .. TX
  T* Hy = Hx + 5 * NHX;                           // SHARE: [5][TY+2][TX], rows y = -1 .. TY
  T* Hz = Hy + 5 * NHY;                           // SHARE: [2][5][TY][TX] (3-D), planes by parity
  double* stg = reinterpret_cast<double*>(smem_raw + ((SM::typed(DIM3) + 15) / 16) * 16);  // [5][H][W] (PF)
  // ring slot of plane kk (kk >= -2)
  auto ring = [&](int kk) -> T* {
    const int sl = NSLOT == 4 ? (kk & 3) : (NSLOT == 3 ? (kk + 6) % 3 : 0);
    return Vs + sl * NV * PL;
  };

  const int tid = threadIdx.x;
  const CC C = CC::from(make_face_consts<T>(args.fp));
  const ViscC<T> VK = make_visc_consts<T>(args.vp);
  const typename VGeo<T>::type* geo = reinterpret_cast<const typename VGeo<T>::type*>(args.geo);
  const MT* mxi = reinterpret_cast<const MT*>(args.metric[0]);
  const MT* meta = reinterpret_cast<const MT*>(args.metric[1]);
  const MT* mzeta = reinterpret_cast<const MT*>(args.metric[2]);

  // Tiles 0..gridDim-1 go to the CTAs in order; later ones are handed out
  // dynamically (largest first, as the table is sorted) through a counter
  // that the last CTA to finish resets for the next launch.
  __shared__ int s_next;
  for (int tile = blockIdx.x; tile < args.ntiles;) {
    const FvTile td = args.tiles[tile];
    const FvBlockDev& B = args.blocks[td.block];
    const int ni = B.ni, nj = B.nj, nk = B.nk;
    const int i0 = td.i0, j0 = td.j0, k0 = td.kk & 0xffff, k1 = td.kk >> 16;
    const long long js = B.jstride, ks = B.kstride, pl = B.plane;
    const double* qin = args.qin + B.qoff;
    const bool cart = B.cartesian != 0;

    // Per-thread work descriptors, fixed for the whole tile (only the plane
    // index changes along k): the halo cells this thread stages ...
    constexpr int LROUNDS = (PL + NT - 1) / NT;
    int loff[LROUNDS];                // (j+2)*js + (i+2), or -1 outside the ghosted block
#pragma unroll
    for (int r = 0; r < LROUNDS; ++r) {
      const int it = tid + r * NT;
      const int rr = it / W, c = it - rr * W;
      const int j = j0 - 2 + rr, i = i0 - 2 + c;
      loff[r] = (it < PL && i < ni + 2 && j < nj + 2) ? (int)((j + 2) * js + (i + 2)) : -1;
    }
    // The fused viscous terms difference T across one cell, so the ring's
    // sixth variable holds T - tref (tref: the binary32 T of the tile's first
    // interior cell) with its numerator rho^2 R (T - tref) =
    // (gamma - 1)(E rho - |m|^2 / 2) - tref R rho^2 formed in double-float
    // from the binary64 state: the binary32 T itself would carry 2^-24 of T
    // into every gradient (128^3 laminar energy residual: 2.6e-5 of its
    // terms' scale)
    float tref = 0.0f;
    df64 trefR = mk(0.0f, 0.0f);
    if constexpr (FUSED_VISC) {
      const int ri = min(i0, ni - 1), rj = min(j0, nj - 1), rk = DIM3 ? min(max(k0, 0), nk - 1) : 0;
      const double* c = qin + (long long)(rk + 2) * ks + (long long)(rj + 2) * js + (ri + 2);
      const double r = c[0], m1 = c[pl], m2 = c[2 * pl], m3 = c[3 * pl];
      tref = (float)((args.vp.gamma - 1.0) * fma(c[4 * pl], r, -0.5 * (m1 * m1 + m2 * m2 + m3 * m3)) /
                     (r * r * args.vp.r_gas));
      trefR = fv_d2df((double)tref * args.vp.r_gas);
    }
    const df64 gm1_df = Sc<df64>::c(args.vp.gamma - 1.0);
    const float iR_f = (float)(1.0 / args.vp.r_gas);
    auto t_dev = [&](const double* qd, float rho) -> float {
      const df64 r = fv_d2df(qd[0]), m1 = fv_d2df(qd[1]), m2 = fv_d2df(qd[2]), m3 = fv_d2df(qd[3]);
      const df64 e = fv_d2df(qd[4]);
      const df64 num = gm1_df * (e * r - Sc<df64>::halve(Sc<df64>::dot3(m1, m1, m2, m2, m3, m3))) - (trefR * r) * r;
      const float ri = __fdividef(1.0f, rho);
      return FADD(num.hi, num.lo) * ri * ri * iR_f;
    };
    // stage plane kk (ghosted index kk + 2 in memory) into its ring slot
    auto load_plane = [&](int kk) {
      T* dst = ring(kk);
      const double* base = qin + (long long)(kk + 2) * ks;
#pragma unroll
      for (int r = 0; r < LROUNDS; ++r) {
        if (loff[r] < 0) continue;
        const double* src = base + loff[r];
        double qd[5];
        T q[5], V[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
          qd[n] = __ldg(src + n * pl);
          q[n] = S::from_d(qd[n]);
        }
        prim_from_cons(C, q, V);
#pragma unroll
        for (int n = 0; n < 5; ++n) dst[n * PL + tid + r * NT] = V[n];
        if constexpr (FUSED_VISC) dst[5 * PL + tid + r * NT] = t_dev(qd, V[0]);
      }
    };

    // asynchronous copy of plane kk's raw binary64 state into the staging
    // plane; every thread later converts exactly the cells it copied
    auto prefetch_plane = [&](int kk) {
      const double* base = qin + (long long)(kk + 2) * ks;
#pragma unroll
      for (int r = 0; r < LROUNDS; ++r) {
        if (loff[r] < 0) continue;
#pragma unroll
        for (int n = 0; n < 5; ++n)
          __pipeline_memcpy_async(stg + n * PL + tid + r * NT, base + loff[r] + n * pl, sizeof(double));
      }
      __pipeline_commit();
    };
    auto convert_staged = [&](int kk) {
      __pipeline_wait_prior(0);
      T* dst = ring(kk);
#pragma unroll
      for (int r = 0; r < LROUNDS; ++r) {
        if (loff[r] < 0) continue;
        const int it = tid + r * NT;
        double qd[5];
        T q[5], V[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
          qd[n] = stg[n * PL + it];
          q[n] = S::from_d(qd[n]);
        }
        prim_from_cons(C, q, V);
#pragma unroll
        for (int n = 0; n < 5; ++n) dst[n * PL + it] = V[n];
        if constexpr (FUSED_VISC) dst[5 * PL + it] = t_dev(qd, V[0]);
      }
    };

    // Evaluate one face from its stencil cells s0..s3 (ring/plane pointers),
    // direction `dir` and face index f, storing the 5 fluxes at dst[n * dstr].
    // code: 0, or the boundary kind whose flux overwrites this face (slip
    // wall, farfield); side: 0 on the block's min face, 1 on its max face
    // vis: the viscous stencil (VISC only): tangential neighbours of L = s1
    // and R = s2, and the padded-cell index of R (L is one step back)
    struct VisArgs {
      const T *Lbm, *Lbp, *Rbm, *Rbp, *Lcm, *Lcp, *Rcm, *Rcp;
      long long gR, gstep;
    };
    // hL, hR, hs (SHARE): the half-slopes of s1 and s2, components hs apart
    auto do_face = [&](const T* s0, const T* s1, const T* s2, const T* s3, const T* hL, const T* hR, int hs,
                       int dir, long long f, T* dst, int dstr, int code, int side, const VisArgs& vis) {
      T nx, ny, nz, A;
      if (cart) {
        nx = S::from_d(B.cart_n[dir][0]); ny = S::from_d(B.cart_n[dir][1]);
        nz = S::from_d(B.cart_n[dir][2]); A = S::from_d(B.cart_area[dir]);
      } else {
        const MT* m = dir == 0 ? mxi : (dir == 1 ? meta : mzeta);
        MetricStore<T>::ld4(m, f, nx, ny, nz, A);
      }
      T out[5];
      if (code == FV_BCK_SLIP_WALL || code == FV_BCK_NOSLIP_WALL) {
        // nearest interior cells: s2, s3 on a min face, s1, s0 on a max face
        wall_face_flux(C, (side ? s1 : s2)[4 * PL], (side ? s0 : s3)[4 * PL], nx, ny, nz, A, out);
      } else if (code == FV_BCK_FARFIELD) {
        const T* gc = side ? s2 : s1;   // first ghost layer: the boundary state
        T Vb[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) Vb[n] = gc[n * PL];
        normal_face_flux(C, Vb, nx, ny, nz, A, out);
      } else if constexpr (SHARE) {
        T VL[5], VR[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
          VL[n] = s1[n * PL] + hL[n * hs];
          VR[n] = s2[n * PL] - hR[n * hs];
        }
        face_riemann(C, VL, VR, nx, ny, nz, A, out);
      } else {
        face_flux(C, s0, s1, s2, s3, PL, nx, ny, nz, A, out);
      }
      if constexpr (FUSED_VISC) {
        // F_i - F_v: the cell sums below then carry the viscous pairs too
        T gl[10], gr[10], fvv[4];
        VGeo<T>::ld10(geo, vis.gR - vis.gstep, gl);
        VGeo<T>::ld10(geo, vis.gR, gr);
        viscous_face_flux(VK, s1, s2, vis.Lbm, vis.Lbp, vis.Rbm, vis.Rbp, vis.Lcm, vis.Lcp, vis.Rcm, vis.Rcp, PL,
                          DIM3, gl, gr, dir, dir == 0 ? 1 : 0, dir == 2 ? 1 : 2, nx * A, ny * A, nz * A, tref, fvv);
#pragma unroll
        for (int n = 0; n < 4; ++n) out[1 + n] = out[1 + n] - fvv[n];
      }
      if constexpr (VISC_PAIRS) {
        // F_i - F_v, as the fused binary32 path stores it; the separate
        // viscous kernel's F_v.S of this face (same face order as the
        // metrics, all blocks)
        T fva, fvb, fvc, fvd;
        const MT* vr = reinterpret_cast<const MT*>(args.fv[dir == 0 ? 0 : (dir == 1 ? 1 : 2)]);
        MetricStore<T>::ld4(vr, B.vface_off[dir] + (f - B.face_off[dir]), fva, fvb, fvc, fvd);
        out[1] = out[1] - fva;
        out[2] = out[2] - fvb;
        out[3] = out[3] - fvc;
        out[4] = out[4] - fvd;
      }
#pragma unroll
      for (int n = 0; n < 5; ++n) dst[n * dstr] = out[n];
    };
    // ... and, for each face item it = tid + r*NT, the face it evaluates:
    // direction, stencil offset inside a plane (xi, eta) or column offset
    // (zeta), metric index without its k term and destination slot
    // (dir < 0: unused or outside).  Decoded on the fly: holding these in
    // registers for the whole tile costs more occupancy than the decode.
    // and (SHARE) the index of the face's lower cell in its direction's slope plane
    auto face_item = [&](int it, int& dir, int& off, int& dst, int& hoff, long long& met) {
      dir = -1;
      if (it < NXI) {
        // the TX faces x < TX of every row first, row by row, then the last
        // face of each row: a warp then reads whole rows of the plane
        // without shared-memory bank conflicts
        int y, x;                                              // face between cells x-1 and x
        if (it < TX * TY) {
          y = it / TX; x = it - y * TX;
        } else {
          y = it - TX * TY; x = TX;
        }
        const int i = i0 + x, j = j0 + y;
        if (i <= ni && j < nj) {
          dir = 0; off = (y + 2) * W + x; dst = y * (TX + 1) + x; hoff = y * (TX + 2) + x;
          met = B.face_off[0] + (long long)j * (ni + 1) + i;
        }
      } else if (it < NXI + NETA) {
        const int e = it - NXI;
        const int y = e / TX, x = e - y * TX;                   // face between rows y-1 and y
        const int i = i0 + x, j = j0 + y;
        if (i < ni && j <= nj) {
          dir = 1; off = y * W + (x + 2); dst = e; hoff = e;
          met = B.face_off[1] + (long long)j * ni + i;
        }
      } else if (DIM3 && it < NFACE) {
        const int e = it - NXI - NETA;
        const int y = e / TX, x = e - y * TX;
        if (i0 + x < ni && j0 + y < nj) {
          dir = 2; off = (y + 2) * W + (x + 2); dst = e; hoff = e;
          met = B.face_off[2] + (long long)(j0 + y) * ni + (i0 + x);
        }
      }
    };
    // SHARE: the half-slopes h = vanleer_half(forward, backward difference)
    // of the cells the faces read - in xi and eta those of plane kp (cells
    // x = -1 .. TX, rows y = -1 .. TY, inside the ghosted block), in zeta
    // that of plane kz (from planes kz-1 .. kz+1, into the slot of kz's
    // parity); inplane = false: zeta only
    auto slopes = [&](int kp, int kz, bool inplane) {
      constexpr int NH = NHX + NHY + (DIM3 ? NZETA : 0);
      const T* Pk = ring(kp);
      for (int it = inplane ? tid : NHX + NHY + tid; it < NH; it += NT) {
        const T *cm, *c0, *cp;
        T* hd;
        int hs;
        if (it < NHX) {
          const int y = it / (TX + 2), x = it - y * (TX + 2);   // cell x - 1 of row y
          if (j0 + y >= nj || i0 + x > ni + 1) continue;
          c0 = Pk + (y + 2) * W + (x + 1);
          cm = c0 - 1;
          cp = c0 + 1;
          hd = Hx + it;
          hs = NHX;
        } else if (it < NHX + NHY) {
          const int e = it - NHX;
          const int y = e / TX, x = e - y * TX;                 // cell x of row y - 1
          if (j0 + y > nj + 1 || i0 + x >= ni) continue;
          c0 = Pk + (y + 1) * W + (x + 2);
          cm = c0 - W;
          cp = c0 + W;
          hd = Hy + e;
          hs = NHY;
        } else {
          const int e = it - NHX - NHY;
          const int y = e / TX, x = e - y * TX;
          if (j0 + y >= nj || i0 + x >= ni) continue;
          const int off = (y + 2) * W + (x + 2);
          cm = ring(kz - 1) + off;
          c0 = ring(kz) + off;
          cp = ring(kz + 1) + off;
          hd = Hz + (kz & 1) * 5 * NZETA + e;
          hs = NZETA;
        }
#pragma unroll
        for (int n = 0; n < 5; ++n) {
          const T v0 = c0[n * PL];
          hd[n * hs] = vanleer_half(cp[n * PL] - v0, v0 - cm[n * PL]);
        }
      }
    };
    const long long kfx = (long long)nj * (ni + 1), kfy = (long long)(nj + 1) * ni, kfz = (long long)nj * ni;
    // zeta face between planes kf-1 and kf (stencil kf-2 .. kf+1) at column offset c
    if (DIM3) {
      // planes k0-2 .. k0 now; plane k0+1 arrives in the first pass below
      for (int s = -2; s <= 0; ++s) load_plane(k0 + s);
      if (PF) prefetch_plane(k0 + 1);
      if constexpr (SHARE) {
        // the zeta slope of plane k0-1; the first pass overwrites k0-2
        __syncthreads();
        slopes(k0 - 1, k0 - 1, false);
        __syncthreads();
      }
    } else {
      load_plane(0);
      __syncthreads();
    }

    // In 3D the first pass (k = k0 - 1) evaluates only the zeta faces below
    // plane k0; every later pass is one plane.
    for (int k = DIM3 ? k0 - 1 : k0; k < k1; ++k) {
      if (DIM3) {
        if (PF) {
          convert_staged(k + 2);
          __syncthreads();
          if (k + 1 < k1) prefetch_plane(k + 3);   // overlaps the faces below
        } else {
          load_plane(k + 2);
          __syncthreads();
        }
      }
      const T* P = ring(k);
      if constexpr (SHARE) {
        slopes(k, k + 1, !DIM3 || k >= k0);
        __syncthreads();
      }
      // ---- every face of this plane (and the zeta faces above it), once;
      // one call site of the face code for all three directions ----
      for (int it = tid; it < NFACE; it += NT) {
        int d, off, dst, hoff;
        long long met;
        face_item(it, d, off, dst, hoff, met);
        if (d < 0 || (DIM3 && k < k0 && d != 2)) continue;
        const T *s0, *s1, *s2, *s3, *hL, *hR;
        int hs;
        T* dp;
        int dstr;
        long long f;
        if (DIM3 && d == 2) {
          // zeta face between planes k and k+1: stencil k-1 .. k+2 from the ring
          // (with a 3-plane ring s0 aliases plane k+2; only the
          // per-face stencil and the wall flux, which keep 4 planes, read it)
          s0 = ring(k - 1) + off;
          s1 = ring(k) + off;
          s2 = ring(k + 1) + off;
          s3 = ring(k + 2) + off;
          dp = Fz + ((k + 1) & 1) * 5 * NZETA + dst;
          dstr = NZETA;
          f = met + (k + 1) * kfz;
          hL = Hz + (k & 1) * 5 * NZETA + hoff;
          hR = Hz + ((k + 1) & 1) * 5 * NZETA + hoff;
          hs = NZETA;
        } else {
          const int st = d == 0 ? 1 : W;
          s0 = P + off;
          s1 = s0 + st;
          s2 = s1 + st;
          s3 = s2 + st;
          dp = (d == 0 ? Fx : Fy) + dst;
          dstr = d == 0 ? NXI : NETA;
          f = met + k * (d == 0 ? kfx : kfy);
          hL = (d == 0 ? Hx : Hy) + hoff;
          hR = hL + (d == 0 ? 1 : TX);
          hs = d == 0 ? NHX : NHY;
        }
        // physical boundary face with an overwritten flux?
        int code = 0, side = 0;
        if (BC && B.bcmap) {
          if (d == 0) {
            const int fy = dst / (TX + 1), fi = i0 + dst - fy * (TX + 1);
            if (fi == 0 || fi == ni) {
              side = fi != 0;
              code = B.bcmap[(side ? (long long)nj * nk : 0) + (long long)k * nj + (j0 + fy)];
            }
          } else if (d == 1) {
            const int fy = dst / TX, fj = j0 + fy;
            if (fj == 0 || fj == nj) {
              side = fj != 0;
              code = B.bcmap[2LL * nj * nk + (side ? (long long)ni * nk : 0) + (long long)k * ni + (i0 + dst - fy * TX)];
            }
          } else {
            const int fk = k + 1;
            if (fk == 0 || fk == nk) {
              side = fk != 0;
              const int fy = dst / TX;
              code = B.bcmap[2LL * nj * nk + 2LL * ni * nk + (side ? (long long)ni * nj : 0) +
                             (long long)(j0 + fy) * ni + (i0 + dst - fy * TX)];
            }
          }
        }
        VisArgs vis;
        if constexpr (FUSED_VISC) {
          // cell R of the face in block coordinates, and its tangential
          // neighbours (and L's) in the plane ring
          int ri, rj, rk;
          if (d == 0) {
            const int fy = dst / (TX + 1);
            ri = i0 + dst - fy * (TX + 1); rj = j0 + fy; rk = k;
          } else {
            const int fy = dst / TX;
            ri = i0 + dst - fy * TX; rj = j0 + fy; rk = d == 2 ? k + 1 : k;
          }
          const long long pi = ni + 2, pij = pi * (nj + 2);
          vis.gR = B.pad_off + (rk + 1) * pij + (long long)(rj + 1) * pi + (ri + 1);
          vis.gstep = d == 0 ? 1 : (d == 1 ? pi : pij);
          const int sb = d == 0 ? W : 1;
          vis.Lbm = s1 - sb; vis.Lbp = s1 + sb; vis.Rbm = s2 - sb; vis.Rbp = s2 + sb;
          if (d == 2) {
            vis.Lcm = s1 - W; vis.Lcp = s1 + W; vis.Rcm = s2 - W; vis.Rcp = s2 + W;
          } else {
            const long long oL = s1 - P, oR = s2 - P;
            const T* Pm = ring(k - 1);
            const T* Pp = ring(k + 1);
            vis.Lcm = Pm + oL; vis.Lcp = Pp + oL; vis.Rcm = Pm + oR; vis.Rcp = Pp + oR;
          }
        }
        do_face(s0, s1, s2, s3, hL, hR, hs, d, f, dp, dstr, code, side, vis);
      }
      __syncthreads();
      if (DIM3 && k < k0) continue;
      // ---- per cell: flux differences in a fixed order, then the RK update ----
      for (int cc = tid; cc < TX * TY; cc += NT) {
        const int y = cc / TX, x = cc - y * TX;
        const int i = i0 + x, j = j0 + y;
        if (i < ni && j < nj) {
          const long long cell = ((long long)k * nj + j) * ni + i;
          const long long q_idx = (long long)(k + 2) * ks + (long long)(j + 2) * js + (i + 2);
          const long long ncell_b = (long long)ni * nj * nk;
          AT R[5];
          const long long src_off = 5 * B.cell_off + cell;
#pragma unroll
          for (int n = 0; n < 5; ++n) {
            const T x1 = Fx[n * NXI + y * (TX + 1) + x + 1], x0 = Fx[n * NXI + y * (TX + 1) + x];
            const T y1 = Fy[n * NETA + (y + 1) * TX + x], y0 = Fy[n * NETA + y * TX + x];
            if constexpr (std::is_same<T, float>::value) {
              // exact pair differences, then the high parts summed with
              // error-free transformations and the low parts in binary32
              const df64 rx = two_sum(x1, -x0), ry = two_sum(y1, -y0);
              df64 h = two_sum(rx.hi, ry.hi);
              float lo = FADD(FADD(rx.lo, ry.lo), h.lo);
              if (DIM3) {
                const df64 rz = two_sum(Fz[((k + 1) & 1) * 5 * NZETA + n * NZETA + cc],
                                        -Fz[(k & 1) * 5 * NZETA + n * NZETA + cc]);
                const df64 h2 = two_sum(h.hi, rz.hi);
                lo = FADD(FADD(lo, rz.lo), h2.lo);
                h.hi = h2.hi;
              }
              if (args.srcvol2) {
                const float2 sv = __ldg(args.srcvol2 + src_off + n * ncell_b);
                const df64 t = two_sum(h.hi, -sv.x);
                lo = FADD(FSUB(lo, sv.y), t.lo);
                h.hi = t.hi;
              }
              R[n] = quick_two_sum(h.hi, lo);
            } else {
              AT r = Acc<T>::diff(x1, x0) + Acc<T>::diff(y1, y0);
              if (DIM3)
                r = r + Acc<T>::diff(Fz[((k + 1) & 1) * 5 * NZETA + n * NZETA + cc],
                                     Fz[(k & 1) * 5 * NZETA + n * NZETA + cc]);
              if constexpr (std::is_same<AT, df64>::value) {
                if (args.srcvol2) {
                  const float2 sv = __ldg(args.srcvol2 + src_off + n * ncell_b);
                  r = r - mk(sv.x, sv.y);
                }
              } else {
                if (args.srcvol) r = r - __ldg(args.srcvol + src_off + n * ncell_b);
              }
              R[n] = r;
            }
          }
          if (args.mode == FV_MODE_RK) {
            // the same binary64 product the host forms when dt is passed by value
            const double alpha_dt = args.dt_dev ? args.alpha * *args.dt_dev : args.alpha_dt;
            const double iv = cart ? B.cart_invvol : __ldg(args.invvol + B.cell_off + cell);
            const double* q0 = args.q0 + B.qoff + q_idx;
            double* qo = args.qout + B.qoff + q_idx;
            if constexpr (std::is_same<AT, double>::value) {
#pragma unroll
              for (int n = 0; n < 5; ++n) qo[n * pl] = rk_apply(q0[n * pl], alpha_dt, iv, R[n]);
            } else if constexpr (std::is_same<T, float>::value) {
              // binary32 increment (its rounding is far below the error of
              // the binary32 face fluxes it sums), one binary64 add
              const float fac = FMUL(fv_d2f_rn(alpha_dt), fv_d2f_rn(iv));
#pragma unroll
              for (int n = 0; n < 5; ++n) qo[n * pl] = q0[n * pl] - fv_f2d(FMUL(fac, FADD(R[n].hi, R[n].lo)));
            } else {
              const df64 fac = fv_d2df(alpha_dt) * fv_d2df(iv);
#pragma unroll
              for (int n = 0; n < 5; ++n) qo[n * pl] = rk_apply(q0[n * pl], fac, R[n]);
            }
            if (args.rmon) {
              // the residual monitor's copy of R, in the accumulator's own
              // storage (no binary64 conversion on the FP64 unit)
              const long long mi = B.cell_off + cell;
              if constexpr (std::is_same<AT, double>::value) {
#pragma unroll
                for (int n = 0; n < 5; ++n) static_cast<double*>(args.rmon)[n * args.ncell_total + mi] = R[n];
              } else {
#pragma unroll
                for (int n = 0; n < 5; ++n)
                  static_cast<float2*>(args.rmon)[n * args.ncell_total + mi] = make_float2(R[n].hi, R[n].lo);
              }
            }
          } else {
            double* ro = args.rout;
            if (args.rout_varmajor) {
#pragma unroll
              for (int n = 0; n < 5; ++n) ro[n * args.ncell_total + B.cell_off + cell] = Sc<AT>::to_d(R[n]);
            } else {
#pragma unroll
              for (int n = 0; n < 5; ++n) ro[5 * B.cell_off + n * ncell_b + cell] = Sc<AT>::to_d(R[n]);
            }
          }
        }
      }
    }
    __syncthreads();   // smem is reused by the next tile
    if (tid == 0) s_next = (int)gridDim.x + atomicAdd(args.tile_counter, 1);
    __syncthreads();
    tile = s_next;
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(args.tile_counter + 1, 1) == (int)gridDim.x - 1) {
      args.tile_counter[0] = 0;
      args.tile_counter[1] = 0;
      __threadfence();
    }
  }
}

// The dynamic shared-memory limit is raised once by occupancy_t (at handle
// creation), so a launch is a plain enqueue that stream capture accepts.
template <class T, int TX, int TY, int NT, bool PF, bool FAST, bool VISC, bool BC>
static int launch_stage_t(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  const size_t smem = StageSmemOf<T, TX, TY, FAST, VISC, BC>::bytes(l.three_d != 0, PF);
  if (l.three_d) {
    fv_stage_kernel<T, TX, TY, NT, true, PF, FAST, VISC, BC><<<l.grid, NT, smem, s>>>(a);
  } else {
    fv_stage_kernel<T, TX, TY, NT, false, false, FAST, VISC, BC><<<l.grid, NT, smem, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <class T, int TX, int TY, int NT, bool PF, bool FAST, bool VISC, bool BC>
static int occupancy_t(bool three_d, size_t* smem_out) {
  const size_t smem = StageSmemOf<T, TX, TY, FAST, VISC, BC>::bytes(three_d, PF);
  int n = 0;
  if (three_d) {
    auto k = fv_stage_kernel<T, TX, TY, NT, true, PF, FAST, VISC, BC>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, smem);
  } else {
    auto k = fv_stage_kernel<T, TX, TY, NT, false, false, FAST, VISC, BC>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, smem);
  }
  if (smem_out) *smem_out = smem;
  return n;
}

// Compiled tile shapes (TX, TY, threads, prefetch); the shape ids of
// fv_config.tile are 1-based indices into this list.  The prefetching shapes
// are built for the binary32-flux form only (their staging plane would cost
// the wider forms a resident CTA).
#define FV_SHAPES(X)      \
  X(1, 32, 8, 256, false) \
  X(2, 32, 4, 128, false) \
  X(3, 16, 8, 128, false) \
  X(4, 30, 8, 256, false) \
  X(5, 32, 8, 288, false) \
  X(6, 32, 8, 256, true)  \
  X(7, 32, 4, 128, true)  \
  X(8, 32, 7, 256, false) \
  X(9, 32, 6, 256, false) \
  X(10, 16, 12, 192, false) \
  X(11, 16, 4, 128, false)

// FAST selects the compile-time default scheme (FaceCFast); each
// translation unit instantiates one combination of FAST, VISC and BC.
template <class T, bool FAST, bool VISC, bool BC>
int fv_dispatch_launch(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s) {
  constexpr bool allow_pf = std::is_same<T, float>::value;
#define FV_LAUNCH_CASE(ID, TX, TY, NT, PF)                                     \
  if (l.shape == ID) {                                                          \
    if (PF && !allow_pf) return -2;                                             \
    return launch_stage_t<T, TX, TY, NT, PF && allow_pf, FAST, VISC, BC>(a, l, s); \
  }
  FV_SHAPES(FV_LAUNCH_CASE)
#undef FV_LAUNCH_CASE
  return -2;
}

template <class T, bool FAST, bool VISC, bool BC>
int fv_dispatch_occupancy(const FvLaunch& l, size_t* smem) {
  constexpr bool allow_pf = std::is_same<T, float>::value;
  const bool d3 = l.three_d != 0;
#define FV_OCC_CASE(ID, TX, TY, NT, PF)                                         \
  if (l.shape == ID) {                                                          \
    if (PF && !allow_pf) return 0;                                              \
    return occupancy_t<T, TX, TY, NT, PF && allow_pf, FAST, VISC, BC>(d3, smem); \
  }
  FV_SHAPES(FV_OCC_CASE)
#undef FV_OCC_CASE
  return 0;
}
