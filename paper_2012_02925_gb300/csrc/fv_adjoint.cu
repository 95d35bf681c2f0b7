// Discrete adjoint (vector-Jacobian product) of one Runge-Kutta stage; the
// face VJPs in binary64 or double-float arithmetic, everything else binary64.  Stage map: Q^(m) = Q^(0) - alpha_m dt / Omega * R(X(Q^(m-1)))
// with X the ghost exchange.  For a cotangent lam of Q^(m):
//   mu_c   = -alpha_m dt / Omega_c * lam_c              (cotangent of R_c)
//   Fbar_f = mu_L(f) - mu_R(f)                          (R_L holds +F_f, R_R holds -F_f)
//   qbar   = sum over faces of (dF_f/dq)^T Fbar_f        (face_vjp, 4-cell stencil)
//   ghost cotangents are added into their donor cells (transpose of X),
//   fixed ghosts are constants.
// Deterministic: per-face contributions go to a scratch array and every cell
// gathers its (up to 12) contributions in a fixed order; connections are
// transposed one launch at a time in table order.
#include "fv_adjoint.cuh"
#include "fv_internal.h"

namespace {

__device__ __forceinline__ long long ghost_index(const FvBlockDev& B, int i, int j, int k) {
  return (long long)(k + FV_GHOST) * B.kstride + (long long)(j + FV_GHOST) * B.jstride + (i + FV_GHOST);
}

// faces of direction `dir` in block B: index f over (n_dir + 1) x (other two
// extents); the face's VJP in arithmetic T, inputs and outputs binary64
// NT threads per CTA; PARK: values dead across the Roe part parked in shared
// memory (ADJ_PARK per thread); LOCK: the CTA's warps pass barriers at fixed
// points of every face VJP (every thread runs the same number of faces, the
// last ones repeating the final face without storing it)
template <class T, int NT, int MINB, bool PARK, bool LOCK>
__global__ void __launch_bounds__(NT, MINB) adj_face_kernel(const FvBlockDev B, int dir, const double* __restrict__ qin,
                                                       const double* __restrict__ lam_out,
                                                       const double* __restrict__ invvol, double alpha_dt,
                                                       const double* __restrict__ metric, long long mstride,
                                                       const AdjParams PP, double* __restrict__ contrib) {
  using S = Sc<T>;
  const AdjC<T> P = adj_consts<T>(PP);
  const int ei = B.ni + (dir == 0), ej = B.nj + (dir == 1), ek = B.nk + (dir == 2);
  const long long nf = (long long)ei * ej * ek;
  const long long ncell_b = (long long)B.ni * B.nj * B.nk;
  const double* lam = lam_out + 5 * B.cell_off;
  const double* qb = qin + B.qoff;
  for (long long base = blockIdx.x * (long long)NT; base < nf; base += (long long)gridDim.x * NT) {
    const bool valid = base + threadIdx.x < nf;
    if (!LOCK && !valid) break;
    const long long f = valid ? base + threadIdx.x : nf - 1;
    const int i = (int)(f % ei), j = (int)((f / ei) % ej), k = (int)(f / ((long long)ei * ej));
    const int g = dir == 0 ? i : (dir == 1 ? j : k);            // face between cells g-1 and g
    const int n_dir = dir == 0 ? B.ni : (dir == 1 ? B.nj : B.nk);
    const long long stride = dir == 0 ? 1 : (dir == 1 ? B.jstride : B.kstride);
    const long long c1 = ghost_index(B, i - (dir == 0), j - (dir == 1), k - (dir == 2));   // cell g-1
    T q[4][5];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int n = 0; n < 5; ++n) q[s][n] = S::from_d(qb[c1 + (s - 1) * stride + n * B.plane]);
    // cotangent of the face flux from the two cells' residual cotangents
    double Fd[5] = {0, 0, 0, 0, 0};
    if (g - 1 >= 0) {
      const int il = i - (dir == 0), jl = j - (dir == 1), kl = k - (dir == 2);
      const long long cl = ((long long)kl * B.nj + jl) * B.ni + il;
      const double fac = -alpha_dt * (B.cartesian ? B.cart_invvol : invvol[B.cell_off + cl]);
#pragma unroll
      for (int n = 0; n < 5; ++n) Fd[n] += fac * lam[n * ncell_b + cl];
    }
    if (g < n_dir) {
      const long long cr = ((long long)k * B.nj + j) * B.ni + i;
      const double fac = -alpha_dt * (B.cartesian ? B.cart_invvol : invvol[B.cell_off + cr]);
#pragma unroll
      for (int n = 0; n < 5; ++n) Fd[n] -= fac * lam[n * ncell_b + cr];
    }
    T Fb[5];
#pragma unroll
    for (int n = 0; n < 5; ++n) Fb[n] = S::from_d(Fd[n]);
    T nx, ny, nz, A;
    if (B.cartesian) {
      nx = S::from_d(B.cart_n[dir][0]); ny = S::from_d(B.cart_n[dir][1]); nz = S::from_d(B.cart_n[dir][2]);
      A = S::from_d(B.cart_area[dir]);
    } else {
      const long long fi = B.face_off[dir] + f;
      nx = S::from_d(metric[4 * fi]); ny = S::from_d(metric[4 * fi + 1]);
      nz = S::from_d(metric[4 * fi + 2]); A = S::from_d(metric[4 * fi + 3]);
    }
    T qbar[4][5], F[5];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int n = 0; n < 5; ++n) qbar[s][n] = S::c(0.0);
    if constexpr (PARK) {
      extern __shared__ __align__(16) unsigned char adj_smem[];
      T* park = reinterpret_cast<T*>(adj_smem) + threadIdx.x;
      face_vjp<T, NT, LOCK>(P, q, nx, ny, nz, A, Fb, qbar, F, park);
    } else {
      face_vjp<T, 0, LOCK>(P, q, nx, ny, nz, A, Fb, qbar, F);
    }
    if (!valid) continue;
    double* out = contrib + f * 20;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int n = 0; n < 5; ++n) out[s * 5 + n] = S::to_d(qbar[s][n]);
  }
}

// every ghosted cell: sum its face contributions, xi then eta then zeta,
// faces in increasing order within a direction
__global__ void adj_gather_kernel(const FvBlockDev B, const double* __restrict__ cx, const double* __restrict__ cy,
                                  const double* __restrict__ cz, int three_d, double* __restrict__ lamg) {
  const int gi = B.ni + 2 * FV_GHOST, gj = B.nj + 2 * FV_GHOST, gk = B.nk + 2 * FV_GHOST;
  const long long n = (long long)gi * gj * gk;
  double* out = lamg + B.qoff;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(x % gi) - FV_GHOST, j = (int)((x / gi) % gj) - FV_GHOST, k = (int)(x / ((long long)gi * gj)) - FV_GHOST;
    const bool ii = i >= 0 && i < B.ni, jj = j >= 0 && j < B.nj, kk = k >= 0 && k < B.nk;
    double acc[5] = {0, 0, 0, 0, 0};
    if (jj && kk) {
      for (int s = 3; s >= 0; --s) {              // faces g = i+2-s in increasing order
        const int g = i + 2 - s;
        if (g < 0 || g > B.ni) continue;
        const double* c = cx + ((((long long)k * B.nj + j) * (B.ni + 1)) + g) * 20 + s * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] += c[v];
      }
    }
    if (ii && kk) {
      for (int s = 3; s >= 0; --s) {
        const int g = j + 2 - s;
        if (g < 0 || g > B.nj) continue;
        const double* c = cy + ((((long long)k * (B.nj + 1) + g) * B.ni) + i) * 20 + s * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] += c[v];
      }
    }
    if (three_d && ii && jj) {
      for (int s = 3; s >= 0; --s) {
        const int g = k + 2 - s;
        if (g < 0 || g > B.nk) continue;
        const double* c = cz + ((((long long)g * B.nj + j) * B.ni) + i) * 20 + s * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] += c[v];
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) out[x + v * B.plane] = acc[v];
  }
}

// transpose of one connection: donor interior cell += ghost cotangent
__global__ void adj_transpose_kernel(const FvBlockDev* __restrict__ blocks, const FvConnDev c, double* lamg) {
  const long long nitems = 2LL * c.L0 * c.L1;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < nitems; it += (long long)gridDim.x * blockDim.x) {
    long long local = it;
    const int a = (int)(local % c.L0);
    local /= c.L0;
    const int b = (int)(local % c.L1);
    const int d = (int)(local / c.L1) + 1;
    const FvBlockDev& D = blocks[c.dst_block];
    const FvBlockDev& S = blocks[c.src_block];
    const int da = c.dst_face >> 1, sa = c.src_face >> 1;
    const int dext[3] = {D.ni, D.nj, D.nk}, sext[3] = {S.ni, S.nj, S.nk};
    int dc[3], sc[3];
    const int dt0 = da == 0 ? 1 : 0, dt1 = da == 2 ? 1 : 2;
    const int st0 = sa == 0 ? 1 : 0, st1 = sa == 2 ? 1 : 2;
    dc[dt0] = c.dlo0 + a;
    dc[dt1] = c.dlo1 + b;
    dc[da] = (c.dst_face & 1) ? dext[da] - 1 + d : -d;
    int st[2] = {c.slo0, c.slo1};
    const int u0 = (c.t0 < 0 ? -c.t0 : c.t0) - 1, u1 = (c.t1 < 0 ? -c.t1 : c.t1) - 1;
    st[u0] += c.t0 > 0 ? a : -a;
    st[u1] += c.t1 > 0 ? b : -b;
    sc[st0] = st[0];
    sc[st1] = st[1];
    sc[sa] = (c.src_face & 1) ? sext[sa] - d : d - 1;
    const long long di = D.qoff + ghost_index(D, dc[0], dc[1], dc[2]);
    const long long si = S.qoff + ghost_index(S, sc[0], sc[1], sc[2]);
#pragma unroll
    for (int v = 0; v < 5; ++v) lamg[si + v * S.plane] += lamg[di + v * D.plane];
  }
}

// lam_in <- interior of lamg; lam_q0 += lam_out
__global__ void adj_finish_kernel(const FvBlockDev B, const double* __restrict__ lamg, const double* __restrict__ lam_out,
                                  double* __restrict__ lam_in, double* __restrict__ lam_q0) {
  const long long nc = (long long)B.ni * B.nj * B.nk;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < 5 * nc; x += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(x / nc);
    const long long c = x - v * nc;
    const int i = (int)(c % B.ni), j = (int)((c / B.ni) % B.nj), k = (int)(c / ((long long)B.ni * B.nj));
    const long long o = 5 * B.cell_off + x;
    lam_in[o] = lamg[B.qoff + ghost_index(B, i, j, k) + v * B.plane];
    lam_q0[o] += lam_out[o];
  }
}

int grid_of(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

}  // namespace

int fv_adjoint_faces(const FvBlockDev& B, int dir, const double* qin, const double* lam_out, const double* invvol,
                     double alpha_dt, const double* metric, long long mstride, const FvFaceParams& fp,
                     int double_float, double* contrib, cudaStream_t s) {
  AdjParams P;
  P.gm1 = fp.gamma - 1.0;
  P.g_gm1 = fp.gamma / (fp.gamma - 1.0);
  P.e4km = fp.eps * 0.25 * (1.0 - fp.kappa);
  P.e4kp = fp.eps * 0.25 * (1.0 + fp.kappa);
  P.harten = fp.harten;
  P.va_d2 = fp.va_delta2;
  P.limiter = fp.limiter;
  P.fix_all = fp.fix_all;
  const long long nf = (long long)(B.ni + (dir == 0)) * (B.nj + (dir == 1)) * (B.nk + (dir == 2));
  // The double-float sweep parks its cell primitives, MUSCL states and
  // Jacobian in shared memory across the Roe part (55 KB per CTA of 128
  // threads), runs the MUSCL forward as a loop, is capped at 128 registers
  // for 4 CTAs per SM (~200 bytes spill) and the warps of a CTA pass
  // barriers at five points of each face.  96^3 VJP stage on GB300: 2.52 ms
  // (168 registers, 430 bytes spilled, 3 CTAs) -> 2.29 (parked, 3 CTAs, no
  // spill) -> 2.03 (parked, 4 CTAs) -> 1.97 (barriers) -> 1.80 ms (MUSCL
  // loop); one CTA of 384 threads (168 registers, no spill) took 2.34 ms,
  // two of 256 1.98 ms.  The binary64 sweep is bound by the FP64 unit and
  // keeps its registers.
  if (double_float) {
    constexpr int NT = 128, MB = 4;
    constexpr bool LOCK = true;
    constexpr int smem = ADJ_PARK * sizeof(df64) * NT;
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(adj_face_kernel<df64, NT, MB, true, LOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    adj_face_kernel<df64, NT, MB, true, LOCK><<<grid_of(nf, NT), NT, smem, s>>>(B, dir, qin, lam_out, invvol, alpha_dt,
                                                                             metric, mstride, P, contrib);
  } else {
    adj_face_kernel<double, 128, 1, false, false><<<grid_of(nf, 128), 128, 0, s>>>(B, dir, qin, lam_out, invvol,
                                                                                  alpha_dt, metric, mstride, P, contrib);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int fv_adjoint_gather(const FvBlockDev& B, const double* cx, const double* cy, const double* cz, int three_d,
                      double* lamg, cudaStream_t s) {
  const long long n = (long long)(B.ni + 4) * (B.nj + 4) * (B.nk + 4);
  adj_gather_kernel<<<grid_of(n, 256), 256, 0, s>>>(B, cx, cy, cz, three_d, lamg);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int fv_adjoint_transpose(const FvBlockDev* d_blocks, const FvConnDev& c, double* lamg, cudaStream_t s) {
  const long long n = 2LL * c.L0 * c.L1;
  adj_transpose_kernel<<<grid_of(n, 256), 256, 0, s>>>(d_blocks, c, lamg);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int fv_adjoint_finish(const FvBlockDev& B, const double* lamg, const double* lam_out, double* lam_in, double* lam_q0,
                      cudaStream_t s) {
  const long long n = 5LL * B.ni * B.nj * B.nk;
  adj_finish_kernel<<<grid_of(n, 256), 256, 0, s>>>(B, lamg, lam_out, lam_in, lam_q0);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
