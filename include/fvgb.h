/*
 * fvgb - explicit finite-volume Euler residual and Runge-Kutta stage of a
 * multi-block structured-grid solver, on one GPU (C ABI).
 *
 * The method is the one of Xue, Jackson and Roy, "An improved framework of
 * GPU computing for CFD applications on structured grids using OpenACC"
 * (arXiv 2012.02925):
 *   - cell-centred conserved variables Q = (rho, rho u, rho v, rho w, rho e_t)
 *     and the weak form of Eq. (governing), Section 2;
 *   - MUSCL reconstruction of the primitive variables with slope limiter,
 *     Eq. (flux) of Section 7.2 (V4);
 *   - Roe's flux-difference splitting as the face flux, Section 2;
 *   - two ghost layers per block face; connected faces take their ghosts from
 *     the neighbouring block each sub-step, Section 2 and Section 4;
 *   - physical boundaries enforced through the ghost cells (slip wall,
 *     supersonic inflow, extrapolated outflow, farfield), Section 2 and
 *     Section 7.2 (V2/V3), with the wall and farfield face fluxes overwritten
 *     after the enforcement, Section 7.2 (V7);
 *   - explicit M-step Runge-Kutta time marching, Section 2;
 *   - optionally the laminar viscous flux F_v of Section 2 (Stokes's-hypothesis
 *     stresses, heat conduction and the work of the stresses), with face
 *     gradients by Green's theorem over an auxiliary volume (a wider stencil
 *     that needs the edge ghost cells, Section 2 and the corner/edge update
 *     of Section 4).
 *
 * Conventions used by every call:
 *   - A block has interior cells i in [0,ni), j in [0,nj), k in [0,nk) and two
 *     ghost layers on every side.
 *   - "Packed ghosted state": for each block in order, 5 variable planes of
 *     (nk+4) x (nj+4) x (ni+4) doubles (i fastest), interior cell (i,j,k) at
 *     ((k+2)(nj+4) + (j+2))(ni+4) + (i+2) of its plane.  fv_state_size() gives
 *     the total number of doubles.
 *   - "Packed interior field": for each block in order, 5 planes of
 *     nk x nj x ni doubles.  fv_field_size() gives the total.
 *   - Faces are numbered imin, imax, jmin, jmax, kmin, kmax = 0..5.
 *   - Pointers named *_dev are device pointers; pointers documented as "host
 *     or device" may be either (the copy direction is inferred through
 *     unified addressing).  The caller owns every pointer it passes; the
 *     library reads or writes it only during the call's stream work.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *     work and return without synchronising unless documented otherwise.
 *   - Every call returns an fv_status; the message of the last failure on a
 *     handle is fv_last_error(handle).  No call aborts, traps or throws.
 */
#ifndef FVGB_H
#define FVGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FV_OK = 0,
  FV_ERR_INVALID_ARG = 1,   /* bad handle, size, range, overlap, stage, ... */
  FV_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  FV_ERR_OOM = 3,           /* device allocation failed */
  FV_ERR_NONFINITE = 4,     /* a residual norm found NaN or Inf */
  FV_ERR_TIMEOUT = 5,       /* reserved: a bounded device wait expired */
  FV_ERR_UNSUPPORTED = 6    /* option not built (tile shape, precision, ...) */
} fv_status;

/* Arithmetic of the face computations.  The state in memory is always IEEE
 * binary64 and the residual sum and RK update keep binary64 accuracy. */
typedef enum {
  FV_PREC_FP64 = 0,      /* every operation in IEEE binary64 */
  FV_PREC_DF64 = 1,      /* face arithmetic in double-float (pairs of binary32,
                            ~48-bit significand) on the FP32 pipe */
  FV_PREC_FP32FLUX = 2   /* limiter / reconstruction / Roe flux in binary32;
                            flux differences, source, RK update in double-float
                            / binary64 */
} fv_precision;

typedef enum { FV_LIM_NONE = 0, FV_LIM_VANLEER = 1, FV_LIM_VANALBADA = 2 } fv_limiter;

/* Face flux (Section 2: Roe's flux-difference splitting, Steger-Warming and
 * van Leer flux-vector splitting are SENSEI's inviscid fluxes). */
typedef enum { FV_FLUX_ROE = 0, FV_FLUX_VANLEER = 1, FV_FLUX_STEGER_WARMING = 2 } fv_flux;

typedef struct fv_ctx* fv_handle;

/* One block.  nodes: HOST pointer to (nk+1)(nj+1)(ni+1) x 3 doubles
 * (xyz fastest, then i, j, k) for a curvilinear block, or NULL for a
 * Cartesian block with origin x0 and spacing h.  Copied during
 * fv_create_blocks. */
typedef struct {
  int ni, nj, nk;
  const double* nodes;
  double x0[3];
  double h[3];
} fv_block_desc;

/* Ghost layers of dst_face of dst_block are filled from src_block (Section 2:
 * ghost cells of connected boundaries carry the neighbouring block's data;
 * Section 5: self-connection is allowed).  The dst patch covers tangential
 * cell indices [dst_lo[0], dst_hi[0]) x [dst_lo[1], dst_hi[1]) (tangential
 * axes in i, j, k order without the face normal).  src_lo holds the src
 * tangential indices of the cell that dst corner dst_lo maps to;
 * transform[t] = +-1 or +-2 names the src tangential axis (1-based, signed)
 * along which one step of dst tangential axis t moves.  Ghost depth d = 1, 2
 * takes the src interior cell at depth d from src_face.  Momentum components
 * are copied unrotated (one global Cartesian frame). */
typedef struct {
  int dst_block, dst_face;
  int dst_lo[2], dst_hi[2];
  int src_block, src_face;
  int src_lo[2];
  int transform[2];
} fv_connection;

/* Physical boundary kinds (Section 2 names slip walls, supersonic/subsonic
 * inflow and outflow and farfield boundaries, enforced through ghost cells).
 * Readings of what the paper does not spell out:
 *   FIXED: ghosts keep the values of the state set by the caller.
 *   SUPERSONIC_INFLOW: both ghost layers hold the prescribed state.
 *   EXTRAPOLATE (supersonic outflow): both layers copy the first interior cell.
 *   SLIP_WALL: ghost at depth d mirrors the interior cell at depth d, with the
 *     momentum reflected about the boundary face's unit normal n:
 *     m_g = m - 2 (m.n) n (density and total energy copied).  The wall face
 *     flux is overwritten with pressure only, (0, p_w S, 0) with
 *     p_w = (3 p_1 - p_2)/2 from the two nearest interior cells.
 *   FARFIELD: both layers hold the characteristic state V_b built from the
 *     first interior cell V_i and the free stream V_f along the outward unit
 *     normal: supersonic (|V_n,i| >= c_i) takes everything from V_i (outflow)
 *     or V_f (inflow); otherwise V_n,b = (R+ + R-)/2 and
 *     c_b = (gamma-1)(R+ - R-)/4 with R+ = V_n,i + 2 c_i/(gamma-1),
 *     R- = V_n,f - 2 c_f/(gamma-1), and the entropy p/rho^gamma and the
 *     tangential velocity of the upwind side.  The farfield face flux is
 *     overwritten with the physical flux F(V_b).S.
 *   NOSLIP_WALL (adiabatic, for the viscous terms): ghost at depth d mirrors
 *     the interior cell at depth d with its momentum reversed (m_g = -m;
 *     density and total energy copied, so the temperature is mirrored); the
 *     inviscid face flux is overwritten as for SLIP_WALL, the viscous flux is
 *     evaluated from the ghosts. */
typedef enum {
  FV_BC_FIXED = 0,
  FV_BC_SUPERSONIC_INFLOW = 1,
  FV_BC_EXTRAPOLATE = 2,
  FV_BC_SLIP_WALL = 3,
  FV_BC_FARFIELD = 4,
  FV_BC_NOSLIP_WALL = 5
} fv_bc_kind;

/* One physical boundary patch: face `face` (0..5) of block `block` over the
 * tangential cells [lo[0], hi[0]) x [lo[1], hi[1]) (tangential axes in i, j, k
 * order without the face normal, as for connections).  state: primitive
 * (rho, u, v, w, p) of a supersonic inflow or of the farfield free stream
 * (ignored by the other kinds). */
typedef struct {
  int block, face;
  int lo[2], hi[2];
  int kind;
  double state[5];
} fv_bc_patch;

/* Method parameters.  Readings of points the paper leaves open:
 *   limiter: van Leer Psi(r) = (r+|r|)/(1+|r|); van Albada in the smooth
 *     product form Psi(a/b) b = b (a^2+ab)/(a^2+b^2+va_delta2); NONE: Psi = 1.
 *   eps, kappa: MUSCL parameters of Eq. (flux) (eps=1, kappa=-1 by default).
 *   harten: Harten entropy-fix width as a fraction of the Roe sound speed, on
 *     the acoustic eigenvalues (and on V_n too when fix_all); 0 = off.
 *   dim: 2 (nk must be 1; no zeta fluxes) or 3.
 *   n_stages, alpha: Q^(m) = Q^(0) - alpha[m-1] dt / Omega R(Q^(m-1)),
 *     m = 1..n_stages (2..8).
 *   tile: 0 = automatic; else an index into the compiled tile shapes
 *     (1: 32x8 cells / 256 threads, 2: 32x4 / 128, 3: 16x8 / 128, 4: 30x8 / 256,
 *     5: 32x8 / 288, 6: 32x8 / 256 and 7: 32x4 / 128 with the next k-plane
 *     prefetched by cp.async - 6 and 7 for FV_PREC_FP32FLUX only -, 8: 32x7 / 256,
 *     9: 32x6 / 256, 10: 16x12 / 192, 11: 16x4 / 128).
 *   kchunk: k-planes per tile; 0 = automatic (about three tiles per resident
 *     CTA slot); -w = about w tiles per resident CTA slot.  Tiles are handed
 *     to persistent CTAs largest first through a device counter.
 *   flux: fv_flux (Roe by default); van Leer F+- split by the normal Mach
 *     number, Steger-Warming by the eigenvalues; F^ = F+(V_L) + F-(V_R).
 *   visc: 1 adds the laminar viscous flux F_v.S = (0, tau.S, Theta.S),
 *     tau = mu (grad u + grad u^T - 2/3 div u I), Theta = tau.u_f + k grad T,
 *     k = mu c_p / prandtl, c_p = gamma r_gas / (gamma - 1), T = p/(rho r_gas);
 *     mu constant (sutherland = 0) or mu (T/t_ref)^1.5 (t_ref + s_suth)/(T + s_suth).
 *     Face values are the means of the two cells; the face gradient of
 *     phi in (u, v, w, T) on the face between L and R along axis a is
 *     [(phi_R - phi_L) A_a + D_b A_b + D_c A_c] / Omega_f with
 *     D_b = ((phi_L,b+ - phi_L,b-) + (phi_R,b+ - phi_R,b-))/4, A_d the mean of
 *     the two cells' averaged face vectors of family d and Omega_f the mean
 *     volume (no c term in 2D).  Ghost cells of a connected face take the
 *     donor cell's geometry, other ghosts that of the adjacent interior cell;
 *     the depth-1 edge ghosts take the donor cell of a connection extended by
 *     one cell along its face, else the mean of their two face-adjacent
 *     ghosts.  R = sum of the inviscid pairs - sum of the viscous pairs - S Omega. */
typedef struct {
  double gamma, eps, kappa, harten, va_delta2;
  int limiter, fix_all, dim, n_stages;
  double alpha[8];
  int precision;
  int tile;
  int kchunk;
  int flux;
  int visc;
  double mu, prandtl, r_gas;
  int sutherland;
  double t_ref, s_suth;
} fv_config;

/* Fill *cfg with the defaults: gamma 1.4, eps 1, kappa -1, van Leer,
 * harten 0.1, fix_all 0, va_delta2 1e-12, dim 3, 4 stages with
 * alpha = (1/4, 1/3, 1/2, 1), FV_PREC_FP64, automatic tiles, Roe flux,
 * inviscid (visc 0; for visc 1: prandtl 0.72, r_gas 287, t_ref 273.15,
 * s_suth 110.4, mu to be set). */
void fv_config_default(fv_config* cfg);

/* Create the solver state on the current CUDA device: validates blocks and
 * connections (ranges inside the faces, no ghost cell filled twice), computes
 * the face vectors S = 1/2 (x_c - x_a) x (x_d - x_b), unit normals, areas and
 * volumes (1/3 sum of face-centroid . S) on the device, builds the tile and
 * connection tables and allocates three state buffers (Q^(0) and two stage
 * buffers).  Blocking.  *out receives the handle (NULL on failure).  The
 * error text of a failed create is available from fv_last_error(NULL). */
int fv_create_blocks(const fv_block_desc* blocks, int nblocks, const fv_connection* conns, int nconn,
                     const fv_config* cfg, fv_handle* out);

/* Release every device resource of the handle (synchronises the device). */
int fv_destroy(fv_handle h);

/* Message of the last failing call on `h` (or of the last failed create when
 * h is NULL).  Owned by the library; valid until the next call on `h`. */
const char* fv_last_error(fv_handle h);

/* Sizes (in doubles) of the packed ghosted state and of the packed interior
 * field; number of interior cells. -1 for a bad handle. */
int64_t fv_state_size(fv_handle h);
int64_t fv_field_size(fv_handle h);
int64_t fv_cell_count(fv_handle h);

/* Set Q^(0) (and both stage buffers, so that fixed ghost values are present
 * in all of them) from a packed ghosted state (host or device).  Ghost cells
 * not covered by a connection keep these values for the life of the state
 * (fixed / Dirichlet ghosts). */
int fv_set_state(fv_handle h, const double* q, void* stream);

/* Upload overlapped with computation: fv_stage_state copies a packed ghosted
 * state (host or device; pinned host memory for an asynchronous copy) into a
 * handle-owned staging buffer on `stream` - typically a copy stream, so that
 * the upload of the next step's input runs while the current step computes -
 * and fv_set_state_staged then sets it as fv_set_state does, on `stream`
 * (device-to-device).  The caller orders the two streams (the staged copy
 * must be complete before fv_set_state_staged reads it, and that read before
 * the next fv_stage_state overwrites it) and keeps the host buffer alive
 * until the copy is done.  The first fv_stage_state allocates the staging
 * buffer (the packed state's size; blocking).  fv_set_state_staged before
 * any fv_stage_state: FV_ERR_INVALID_ARG. */
int fv_stage_state(fv_handle h, const double* q, void* stream);
int fv_set_state_staged(fv_handle h, void* stream);

/* Overwrite one state buffer (0 = Q^(0), 1, 2 = stage buffers) with a packed
 * ghosted state (host or device); the other buffers are untouched.  Used to
 * replay a stage from a checkpoint (the adjoint's forward recomputation). */
int fv_set_buffer(fv_handle h, int buffer, const double* q, void* stream);

/* Copy buffer `buffer` (0 = Q^(0), the current solution; 1, 2 = stage
 * buffers) out as a packed ghosted state (host or device destination).  With
 * a host destination the call synchronises `stream`. */
int fv_get_state(fv_handle h, int buffer, double* q, void* stream);

/* Source term per unit volume at the cell centroids as a packed interior
 * field (host or device), S of Eq. (governing); the library stores S * Omega.
 * NULL removes the source. */
int fv_set_source(fv_handle h, const double* s, void* stream);

/* Physical boundaries of the handle (replacing any earlier set; n = 0 clears
 * them).  patches: HOST array of n fv_bc_patch, copied.  Validates block and
 * face indices (faces 4, 5 only when dim = 3), patch ranges inside the face,
 * the kind, a finite state with rho > 0 and p > 0 for SUPERSONIC_INFLOW and
 * FARFIELD, and at least two interior cells along the normal of a SLIP_WALL
 * face; FV_ERR_INVALID_ARG otherwise (the old set stays).  A CUDA or
 * allocation failure after validation leaves no patches set.  Patches are filled
 * in order after the connections, so a later patch wins where two overlap.
 * Discards cached step graphs.  Blocking. */
int fv_set_boundaries(fv_handle h, const fv_bc_patch* patches, int n);

/* Ghost fill of state buffer `buffer`: first the connections - for every
 * connection, ghost cells at depth 1 and 2 of the dst patch <- src interior
 * cells at the same depth (Section 2, Section 4; Section 7.2 V1 packs such
 * slabs for MPI - on one device the copy is direct) - then the physical
 * boundary patches (fv_set_boundaries).  One kernel launch for each of the
 * two parts that is present. */
int fv_exchange_ghosts(fv_handle h, int buffer, void* stream);

/* Residual R = sum over faces of F^(V_L, V_R) |S| - S Omega of buffer
 * `buffer` as it stands (no exchange), written to r_dev as a packed interior
 * field (device pointer, fv_field_size doubles).  Sum order per cell: xi pair,
 * eta pair, zeta pair, source.  Slip-wall and farfield boundary faces carry
 * their overwritten fluxes (fv_bc_kind). */
int fv_residual(fv_handle h, int buffer, double* r_dev, void* stream);

/* Runge-Kutta stage m (1..n_stages) with time step dt: fill the ghosts of
 * Q^(m-1) (fv_exchange_ghosts), evaluate R(Q^(m-1)) and write
 * Q^(m) = Q^(0) - alpha_m dt / Omega R.
 * Buffers: stage 1 reads Q^(m-1) = Q^(0) from buffer 0; stage m < n_stages
 * writes buffer 1 when m is odd and buffer 2 when m is even; the last stage
 * writes buffer 0 in place; stage m > 1 reads what stage m-1 wrote.  Kernel
 * launches: connections, physical boundaries, fused residual + update; with
 * visc also the edge ghosts and (binary64, double-float) the viscous face
 * kernel before the fused kernel; stage 1 with the residual monitor on (see
 * fv_set_monitor) also its two reduction kernels. */
int fv_rk_stage(fv_handle h, int stage, double dt, void* stream);

/* A whole time step: stages 1..n_stages (Section 2's M-step scheme).  With
 * use_graph != 0 the stage sequence is captured once per stream as a CUDA
 * graph and replayed; the graph reads dt from a device slot of its own, which
 * a one-thread kernel on `stream` rewrites whenever dt differs from the
 * previous step's, so a changing dt (CFL-based stepping) re-captures nothing.
 * At most 8 streams keep a graph; a ninth evicts the least recently used one
 * (after a device synchronisation).  The first step on a stream allocates 8
 * bytes and instantiates its graph (blocking). */
int fv_rk_step(fv_handle h, double dt, int use_graph, void* stream);

/* Number of RK-step graphs fv_rk_step currently holds (one per stream it has
 * stepped on, at most 8); -1 for a NULL handle. */
int fv_graph_count(fv_handle h);

/* Residual norms of buffer `buffer` (after a ghost exchange of it): per
 * variable L2 = sqrt(mean over all interior cells of R^2) in out_host[0..4]
 * and Linf = max |R| in out_host[5..9] (host pointer, 10 doubles).
 * Synchronises `stream`.  Returns FV_ERR_NONFINITE when any R is NaN/Inf. */
int fv_residual_norms(fv_handle h, int buffer, double* out_host, void* stream);

/* Residual monitor (the residual histories of Sections 8.1-8.3, recorded
 * without a separate residual evaluation).  on != 0: from now on every RK
 * stage 1 (fv_rk_stage(h, 1, ...), the first stage of fv_rk_step) also
 * stores the residual it computes, R(Q^(0)) - the residual of the state the
 * step starts from, the one fv_residual_norms(h, 0, ...) would give before
 * the step - and reduces it to the norms fv_monitor_norms returns.  The
 * first call with on != 0 allocates the monitor's device memory (5 cells x
 * 8 bytes per cell and a few KB; blocking); any call discards cached step
 * graphs.  on = 0 stops the recording (the memory stays until fv_destroy). */
int fv_set_monitor(fv_handle h, int on);

/* Norms recorded by the latest monitored stage 1, as fv_residual_norms
 * defines them (out_host[0..4] L2, [5..9] Linf; host pointer, 10 doubles).
 * Synchronises `stream` (the stream the step ran on).  FV_ERR_INVALID_ARG if
 * the monitor is off or no monitored stage has been launched since it was
 * turned on; FV_ERR_NONFINITE (out_host still written) when that residual
 * had NaN/Inf entries. */
int fv_monitor_norms(fv_handle h, double* out_host, void* stream);

/* Autotuner of the batched launch (not in the paper): times `reps` launches
 * of RK stage 1 with step dt for every compiled tile shape and a set of
 * k-chunk lengths (planes per tile; automatic = enough tiles to fill the
 * resident CTA slots about three times), keeps the fastest and discards
 * cached step graphs.  Reads Q^(0), overwrites stage buffer 1: call it between
 * steps.  Synchronises `stream`. */
int fv_autotune(fv_handle h, double dt, int reps, void* stream);

/* Current launch configuration: out4 = {tile shape (0 = automatic), k-chunk
 * (0 = automatic), number of tiles, persistent CTAs}. */
int fv_get_launch(fv_handle h, int* out4);

/* Discrete-adjoint vector-Jacobian product of one RK stage m with step dt.
 * Stage map: Q^(m) = Q^(0) - alpha_m dt / Omega R(X(Q^(m-1))) with X the
 * ghost exchange.  Inputs: qin_dev = the stage input Q^(m-1) (packed ghosted
 * state, device), lam_out_dev = dJ/dQ^(m) (packed interior field).  Outputs:
 * lam_in_dev (packed interior field) <- (dQ^(m)/dQ^(m-1))^T lam_out,
 * including the transpose of the exchange (ghost cotangents added into their
 * donor cells); lam_q0_dev (packed interior field) += lam_out.  qin_dev is
 * not modified.  Fixed ghost cells are constants.  Built for FV_PREC_FP64
 * handles with the Roe flux, no physical boundary patches and visc = 0
 * (FV_ERR_UNSUPPORTED otherwise). */
int fv_adjoint_vjp(fv_handle h, int stage, double dt, const double* qin_dev, const double* lam_out_dev,
                   double* lam_in_dev, double* lam_q0_dev, void* stream);

/* Arithmetic of fv_adjoint_vjp's per-face sweeps (not in the paper):
 * FV_PREC_FP64 (the default) or FV_PREC_DF64 - double-float on the binary32
 * units, relative error ~1e-14 per operation, several times faster on parts
 * whose binary64 rate is a small fraction of the binary32 rate.  States,
 * cotangents, the gather, the exchange transpose and the accumulation stay
 * binary64.  FV_ERR_INVALID_ARG for any other value. */
int fv_set_adjoint_arith(fv_handle h, int precision);

/* ---------------------------------------------------------------------------
 * Cross-device halo: connections whose two sides live on different devices
 * (ranks) after the blocks are split and aggregated onto processors
 * (Section 4: Cartesian splitting, over-decomposition and aggregation;
 * Section 5: decomposing and re-linking connected boundaries).  Section 7.2
 * V1 packs such boundary data into contiguous send buffers and unpacks
 * received ones on the GPU, V5/V6 exchange them with non-blocking calls, all
 * posted before the wait, and V10 (GPUDirect) sends device buffers directly.
 * The library does the device half: fv_halo_pack gathers this handle's donor
 * cells into a send buffer and fv_halo_unpack scatters a receive buffer into
 * this handle's ghost cells; the transfer itself is the caller's (e.g.
 * NCCL/torch.distributed point-to-point calls on the device buffers).
 *
 * Each slab is one fv_connection as fv_create_blocks defines it, with only
 * the local side's block index meaningful:
 *   send[i]: src_block (this handle's block), src_face, src_lo, transform,
 *            and dst_face, dst_lo, dst_hi (the receiver's patch, which fixes
 *            the item order and count); dst_block is ignored;
 *   recv[i]: dst_block (this handle's block), dst_face, dst_lo, dst_hi;
 *            src_block, src_face, src_lo and transform are ignored.
 * A slab holds n = 2 L0 L1 ghost cells (depth 1 and 2, L0 = dst_hi[0] -
 * dst_lo[0], L1 = dst_hi[1] - dst_lo[1]) in the order (a, b, depth), a
 * fastest, as 5 variable planes of n doubles; slabs lie back to back in table
 * order.  A sender and its receiver must list a connection with the same
 * dst patch, in the same position of their tables' segments for each other.
 * fv_set_halo validates the tables (FV_ERR_INVALID_ARG: ranges, transforms,
 * recv patches overlapping each other or this handle's own connections),
 * replaces any previous tables and synchronises the device; the device
 * tables it allocates are freed by fv_destroy.  Blocks whose ghosts come from
 * a recv slab must not also have them fixed by fv_set_state's caller. */
int fv_set_halo(fv_handle h, const fv_connection* send, int nsend, const fv_connection* recv, int nrecv);

/* Doubles in the send (recv == 0) or receive (recv != 0) buffer: 5 x the
 * slab cells of the table; -1 for a NULL handle. */
int64_t fv_halo_size(fv_handle h, int recv);

/* Gather the send slabs' donor cells (depth 1, 2 inside the src face) of
 * state buffer `buffer` (0, 1, 2 as fv_rk_stage numbers them) into send_dev
 * (device, fv_halo_size(h, 0) doubles).  One kernel launch on `stream`;
 * nothing when the table is empty. */
int fv_halo_pack(fv_handle h, int buffer, double* send_dev, void* stream);

/* Scatter recv_dev (device, fv_halo_size(h, 1) doubles, as a sender's
 * fv_halo_pack wrote it) into the recv slabs' ghost cells of state buffer
 * `buffer`.  One kernel launch on `stream`. */
int fv_halo_unpack(fv_handle h, int buffer, const double* recv_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Arithmetic throughput probe (measurement support; no paper counterpart).
 * The paper's P100/V100 ran binary64 at half the binary32 rate; the stage
 * kernel's arithmetic roofline on another part needs that part's measured
 * rates.  Runs short probe kernels on the current device (8 CTAs of 256
 * threads per SM, 8 independent dependency chains per thread) and writes to
 * out_host (host pointer, n_out >= FV_PROBE_NRATES doubles) operations per
 * second of: [0] binary64 FMA, [1] add, [2] multiply, [3] the compiler's IEEE
 * reciprocal 1.0/x, [4] IEEE square root, [5] binary32 FMA, and the
 * double-float operations of the stage kernel's other form: [6] add,
 * [7] multiply, [8] quotient, [9] square root, [10] absolute value,
 * [11] the binary64 face code's reciprocal (see fv_check_rcp64) and [12] its
 * square root (see fv_check_sqrt64).
 * Allocates and frees 2 KB, synchronises `stream`, takes ~50 ms.
 * FV_ERR_INVALID_ARG for a NULL pointer or short array, FV_ERR_CUDA if a
 * launch fails.
 * ------------------------------------------------------------------------- */
#define FV_PROBE_NRATES 13

int fv_probe_alu_rates(double* out_host, int n_out, void* stream);

/* Test support for the binary64 face code's reciprocal (a Newton-type
 * refinement of the hardware's approximate reciprocal, within one unit in
 * the last place of 1/x): for each of the n doubles at x_dev (device) writes
 * out_dev[2i] = that reciprocal and out_dev[2i+1] = the compiler's IEEE
 * 1.0 / x[i] (device, 2n doubles), asynchronously on `stream`.
 * FV_ERR_INVALID_ARG for NULL pointers or n <= 0, FV_ERR_CUDA if the launch
 * fails. */
int fv_check_rcp64(const double* x_dev, int64_t n, double* out_dev, void* stream);

/* Test support for the binary64 face code's square root (the hardware's
 * approximate reciprocal square root corrected by the binomial series of
 * (1 - e)^(-1/2), within one unit in the last place of sqrt(x) for positive
 * normal x): out_dev[2i] = that square root, out_dev[2i+1] = the compiler's
 * IEEE sqrt(x[i]).  Arguments, stream and errors as fv_check_rcp64. */
int fv_check_sqrt64(const double* x_dev, int64_t n, double* out_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Allocation-free residual norms.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory while they
 * run - code under a framework's caching allocator (where cudaMalloc would
 * synchronise the device or fragment the pool), real-time or embedded hosts
 * that forbid allocation after start-up, and plugins that only receive
 * memory from their host application.
 *
 * field_dev: device pointer to 5 contiguous planes of n doubles (variable v at
 *   field_dev + v*n), e.g. the packed interior field that fv_residual writes
 *   for a one-block handle.  n must satisfy 1 <= n <= FV_NOALLOC_MAX_N.
 * out_dev: device pointer to 11 doubles: per-variable L2 = sqrt(mean of
 *   squares) in [0..4], Linf in [5..9], and in [10] the number of variables
 *   that hold NaN or Inf.  Written asynchronously on `stream`.
 * Partial sums (one slot per FV_NOALLOC_CHUNK elements) live in a fixed
 * 120 KiB device array inside the library: it is held on every GPU that loads
 * the library until the process exits, it is shared by every call, and calls
 * whose kernels overlap on the GPU race on it (serialise them on one stream).
 * The first call on a device looks up that array's device address; the
 * address is kept until the process exits, so after a cudaDeviceReset() of a
 * device this entry point must not be called on that device again.  Nothing is
 * allocated or freed.  The launch status returned is that of this call's
 * own launches (an error left by an earlier, unrelated call is neither
 * reported nor cleared).
 * Returns FV_ERR_INVALID_ARG for NULL pointers or n outside
 * [1, FV_NOALLOC_MAX_N], FV_ERR_CUDA when the address lookup or a launch
 * fails, FV_ERR_UNSUPPORTED for device ordinals above 63.
 * ------------------------------------------------------------------------- */
#define FV_NOALLOC_CHUNK 65536
#define FV_NOALLOC_MAX_N (1024LL * FV_NOALLOC_CHUNK)

int fv_field_norms_noalloc(const double* field_dev, int64_t n, double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FVGB_H */
