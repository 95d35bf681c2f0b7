// Internal data structures shared by the host runtime and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define FV_GHOST 2

// One structured block as the kernels see it.  State buffers hold, per
// block, 5 variable planes of (nk+4) x (nj+4) rows of `pitch` doubles
// (i fastest, ghost cells inline, interior cell (i,j,k) at
// ((k+2)*(nj+4) + (j+2))*pitch + (i+2)).
struct FvBlockDev {
  int ni, nj, nk, pitch;
  long long jstride, kstride;   // = pitch, pitch*(nj+4)
  long long plane;              // distance between variable planes (elements)
  long long qoff;               // block offset inside a state buffer (elements)
  long long cell_off;           // first interior cell in cell-indexed arrays
  long long face_off[3];        // first face in the per-direction metric arrays
  int cartesian;                // metrics are per-block constants
  int pad_;
  // codes of the boundary faces whose flux is overwritten (slip wall,
  // farfield): six face maps (imin, imax, jmin, jmax, kmin, kmax; sizes
  // nj*nk, nj*nk, ni*nk, ni*nk, ni*nj, ni*nj; first tangential index
  // fastest) back to back, or null when the block has none
  const signed char* bcmap;
  long long pad_off;            // viscous terms: first cell of the block padded by one layer
  long long vface_off[3];       // viscous terms: first face per direction (every block)
  double cart_n[3][3];          // Cartesian unit normal of each face family
  double cart_area[3];          // Cartesian face areas
  double cart_invvol;           // Cartesian 1/volume
};

// One unit of work of the fused stage kernel: a TX x TY column of cells of a
// block, marched from k0 to k1-1.
struct FvTile {
  int block, i0, j0, kk;        // kk = k0 | (k1 << 16)
};

struct FvConnDev {
  int dst_block, dst_face, dlo0, dlo1, L0, L1;
  int src_block, src_face, slo0, slo1, t0, t1;
  long long item_off;           // first work item (a, b, depth) of this connection
};

// One unit of work of the exchange kernel: items a0..a0+FV_XCH_TA-1 x
// b0..b0+FV_XCH_TB-1 (both depths) of connection `conn`, clipped to its patch.
struct FvXchTile {
  int conn, a0, b0, pad_;
};
constexpr int FV_XCH_TA = 32, FV_XCH_TB = 16;

// Physical boundary kinds as the kernels see them (the values of fv_bc_kind).
constexpr int FV_BCK_FIXED = 0, FV_BCK_SUPERSONIC_INFLOW = 1, FV_BCK_EXTRAPOLATE = 2, FV_BCK_SLIP_WALL = 3,
              FV_BCK_FARFIELD = 4, FV_BCK_NOSLIP_WALL = 5;

// One physical boundary patch; work items (a, b) = tangential cells.
struct FvBcDev {
  int block, face, lo0, lo1, L0, L1, kind, pad_;
  long long item_off;           // first work item of this patch
  double state[5];              // primitive (rho, u, v, w, p)
  double qstate[5];             // the same, conserved
  double cstate;                // its speed of sound
};

struct FvViscParams {
  double gamma, mu, r_gas, kfac;   // kfac = gamma r_gas / ((gamma - 1) Pr): k = mu kfac
  double t_ref, s_suth;
  int sutherland, dim;
};

struct FvFaceParams {
  double gamma, eps, kappa, harten, va_delta2;
  int limiter, fix_all, flux;
};

enum { FV_MODE_RK = 0, FV_MODE_RESIDUAL = 1 };

struct FvStageArgs {
  const FvBlockDev* blocks;
  const FvTile* tiles;
  int ntiles;
  int* tile_counter;            // {next dynamic tile, CTAs finished}; zero between launches
  int mode;
  const double* qin;            // Q^(m-1)
  const double* q0;             // Q^(0)
  double* qout;                 // Q^(m)
  const void* metric[3];        // per direction: one (n_x, n_y, n_z, |S|) record per face
  long long mstride[3];         // per direction: faces in all blocks
  const double* invvol;         // 1/Omega per interior cell
  const double* srcvol;         // S*Omega, [block][5][cells], or null
  const float2* srcvol2;        // the same as double-float (hi, lo) pairs, or null
  const void* fv[3];            // viscous face fluxes per direction, one (momentum x, y, z, energy) record
                                // per face in the form's storage type (binary64, binary32 pairs), or null
  FvViscParams vp;              // the binary32 form's fused viscous terms (VISC kernels)
  const void* geo;              // and their 12-entry (Omega, Sbar_xi, Sbar_eta, Sbar_zeta, pads) geometry record
                                // per cell of every block padded by one layer, binary32
  double* rout;                 // residual output or null
  int rout_varmajor;            // 0: [block][5][cells]; 1: [5][all cells]
  void* rmon;                   // RK mode: the residual also stored here, [5][all cells], as binary64
                                // (binary64 form) or (hi, lo) binary32 pairs (other forms); or null
  long long ncell_total;
  double alpha_dt;              // alpha_m * dt (dt_dev null)
  const double* dt_dev;         // or: dt read from device memory (a replayed graph), alpha_dt = alpha * *dt_dev
  double alpha;                 // alpha_m
  FvFaceParams fp;
};

// Kernel launchers, one translation unit per compiled variant.
struct FvLaunch {
  int shape;                    // compiled tile shape id (1-based)
  int tx, ty, threads;          // tile shape
  int grid;                     // CTAs (persistent)
  int three_d;
  int fast;                     // the kernel with the default scheme compiled in
  int visc;                     // the kernel with the laminar viscous terms (fused for binary32, the
                                // separate kernel's pairs for the other forms)
  int bc;                       // the kernel with the boundary-face flux overwrites
};

// The default scheme (Roe flux, van Leer limiter, eps = 1, kappa = -1,
// Harten fix on the acoustic waves only) has kernels with its switches fixed
// at compile time.
inline bool fv_default_scheme(int flux, int limiter, double eps, double kappa, double harten, int fix_all) {
  return flux == 0 && limiter == 1 && eps == 1.0 && kappa == -1.0 && harten > 0.0 && fix_all == 0;
}

// Stage kernel variants, fv_stage_<name>.cu each: the form (fp64, df64,
// fp32 = binary32 flux), _fast = default scheme compiled in,
// _visc = laminar viscous terms, _bc = boundary-face flux overwrites.
// launch: enqueue on a stream; occupancy: CTAs per SM for the launch's tile
// shape (0 = shape not compiled) and its dynamic shared memory.
#define FV_STAGE_VARIANTS(X)                                                                  \
  X(fp64) X(fp64_bc) X(fp64_visc) X(fp64_visc_bc) X(fp64_fast) X(fp64_fast_bc) X(fp64_fast_visc)  \
  X(fp64_fast_visc_bc) X(df64) X(df64_bc) X(df64_visc) X(df64_visc_bc) X(df64_fast) X(df64_fast_bc) \
  X(df64_fast_visc) X(df64_fast_visc_bc) X(fp32) X(fp32_bc) X(fp32_visc) X(fp32_visc_bc) X(fp32_fast) \
  X(fp32_fast_bc) X(fp32_fast_visc) X(fp32_fast_visc_bc)
#define FV_DECLARE_STAGE_VARIANT(NAME)                                                       \
  int fv_launch_stage_##NAME(const FvStageArgs& a, const FvLaunch& l, cudaStream_t s);     \
  int fv_stage_occupancy_##NAME(const FvLaunch& l, size_t* smem_bytes);
FV_STAGE_VARIANTS(FV_DECLARE_STAGE_VARIANT)
#undef FV_DECLARE_STAGE_VARIANT

// tile shapes compiled into fv_stage_kernel: {TX, TY, threads, prefetch}
constexpr int FV_NUM_SHAPES = 11;
constexpr int FV_SHAPE_TABLE[FV_NUM_SHAPES][4] = {{32, 8, 256, 0}, {32, 4, 128, 0}, {16, 8, 128, 0},
                                                  {30, 8, 256, 0}, {32, 8, 288, 0}, {32, 8, 256, 1},
                                                  {32, 4, 128, 1}, {32, 7, 256, 0}, {32, 6, 256, 0},
                                                  {16, 12, 192, 0}, {16, 4, 128, 0}};

// Discrete-adjoint kernels (fv_adjoint.cu): binary64 data; the face VJPs in
// binary64 (double_float = 0) or double-float arithmetic.
int fv_adjoint_faces(const FvBlockDev& B, int dir, const double* qin, const double* lam_out, const double* invvol,
                     double alpha_dt, const double* metric, long long mstride, const FvFaceParams& fp,
                     int double_float, double* contrib, cudaStream_t s);
int fv_adjoint_gather(const FvBlockDev& B, const double* cx, const double* cy, const double* cz, int three_d,
                      double* lamg, cudaStream_t s);
int fv_adjoint_transpose(const FvBlockDev* d_blocks, const FvConnDev& c, double* lamg, cudaStream_t s);
int fv_adjoint_finish(const FvBlockDev& B, const double* lamg, const double* lam_out, double* lam_in, double* lam_q0,
                      cudaStream_t s);

// ---------------------------------------------------------------------------
// Laminar viscous terms (fv_visc.cu)
// ---------------------------------------------------------------------------


// Padded-cell geometry of the auxiliary volumes for the binary32 form's
// fused path: a 12-entry record per cell (Omega, Sbar_xi, Sbar_eta,
// Sbar_zeta, 2 pads) in binary32, read with 16-byte loads.
//
// The binary64 and double-float forms use the separate kernel below.  Its
// static geometry is one 12-entry record per face of each direction:
// G_a, G_b, G_c (the auxiliary volume's face vectors of the face's own
// family a and of the two tangential families, each divided by the
// auxiliary volume) and the face's area vector S, in the form's storage type
// (binary64, or (hi, lo) binary32 pairs for double-float).

// One unit of work of the viscous face kernel: face positions
// i0..i0+31 x j0..j0+7 of a block, marched over k0..k0+7 (one plane in 2D).
struct FvViscTile {
  int block, i0, j0, k0;
};
constexpr int FV_VISC_TX = 32, FV_VISC_TY = 8, FV_VISC_KC = 8;

struct FvViscArgs {
  const FvBlockDev* blocks;
  const FvViscTile* tiles;
  int ntiles;
  const double* q;                 // state buffer (ghosts, edge ghosts filled)
  const void* fgeo[3];             // per direction: the face geometry records
  void* fv[3];                     // per direction: viscous fluxes, one 4-value record per face
  FvViscParams vp;
};

// F_v.S of every face of every direction (binary64: precision 0,
// double-float: 1)
int fv_visc_faces(const FvViscArgs& a, int precision, cudaStream_t s);

// ---------------------------------------------------------------------------
// Residual norms (fv_monitor.cu)
// ---------------------------------------------------------------------------

// r: [5][ncell] residual as binary64 (binary64 != 0) or (hi, lo) binary32
// pairs; partials: 15 * nparts doubles of scratch (nparts = FV_NORM_PARTS
// CTAs per SM); out: 15 doubles on the device = per variable
// sqrt(mean R^2), max |R|, non-finite flag count.
constexpr int FV_NORM_PARTS = 8;
int fv_monitor_reduce(const void* r, int binary64, long long ncell, double* partials, int nparts, double* out,
                      cudaStream_t s);
