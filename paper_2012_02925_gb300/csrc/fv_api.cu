// Host runtime of the C ABI declared in include/fvgb.h, and the small kernels
// around the fused stage kernel: metrics, ghost exchange, residual norms,
// source scaling.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/fvgb.h"
#include "fv_internal.h"

namespace {

thread_local std::string g_create_error;

// streams whose RK-step graph fv_rk_step keeps at one time
constexpr int FV_MAX_GRAPHS = 8;

}  // namespace

struct fv_ctx {
  fv_config cfg;
  int nblocks = 0, nconn = 0;
  std::vector<FvBlockDev> hb;
  std::vector<fv_connection> conns;
  FvBlockDev* d_blocks = nullptr;
  FvTile* d_tiles = nullptr;
  int ntiles = 0;
  int* d_tile_counter = nullptr;    // dynamic tile scheduling of the stage kernel
  FvLaunch launch{};
  FvConnDev* d_conns = nullptr;
  long long conn_items = 0;
  FvXchTile* d_xtiles = nullptr;    // exchange kernel work units of d_conns
  int nxtiles = 0;
  double* buf[3] = {nullptr, nullptr, nullptr};
  long long state_elems = 0;        // internal layout, doubles per buffer
  long long ext_state_elems = 0;    // packed ghosted layout
  long long ncell = 0;              // interior cells, all blocks
  void* metric[3] = {nullptr, nullptr, nullptr};
  long long nfaces[3] = {0, 0, 0};
  double* invvol = nullptr;
  double* vol = nullptr;
  double* srcvol = nullptr;
  float2* srcvol2 = nullptr;        // S*Omega as double-float pairs (non-binary64 forms)
  double* scratch_r = nullptr;      // residual (variable-major) for norms
  double* stage_buf = nullptr;      // a packed state staged by fv_stage_state
  bool staged = false;
  double* partials = nullptr;       // per-CTA norm partials
  double* d_norm = nullptr;         // 11 doubles
  double* adj_contrib = nullptr;    // adjoint: per-face input cotangents (20 per face)
  double* adj_lamg = nullptr;       // adjoint: ghosted cotangent of Q^(m-1)
  double* adj_qx = nullptr;         // adjoint: X(Q^(m-1)), the exchanged stage input
  int adj_df64 = 0;                 // adjoint face VJPs in double-float arithmetic (fv_set_adjoint_arith)
  std::vector<FvConnDev> hconns;
  // cross-device halo slabs (fv_set_halo): send = this device's donor side,
  // recv = this device's ghost side; item offsets count slab items
  FvConnDev* d_hsend = nullptr;
  FvConnDev* d_hrecv = nullptr;
  int nhsend = 0, nhrecv = 0;
  long long hsend_items = 0, hrecv_items = 0;
  FvXchTile* d_hstiles = nullptr;   // their exchange kernel work units
  FvXchTile* d_hrtiles = nullptr;
  int nhstiles = 0, nhrtiles = 0;
  std::vector<fv_bc_patch> bcs;     // physical boundary patches as set
  FvBcDev* d_bcs = nullptr;
  int nbc = 0;
  long long bc_items = 0;
  signed char* d_bcmap = nullptr;   // overwritten-flux face maps of all blocks
  // laminar viscous terms
  long long pad_total = 0;          // cells of all blocks padded by one layer
  long long nvfaces[3] = {0, 0, 0}; // faces per direction, every block
  double* geo = nullptr;            // auxiliary-volume geometry [10][pad_total], binary64 (setup only)
  void* geo_t = nullptr;            // binary32 form: the same as per-cell records [pad_total][12]
  void* fgeo[3] = {nullptr, nullptr, nullptr};    // other forms: face records (G_a, G_b, G_c, S) [nvfaces[d]][12]
  FvViscTile* d_vtiles = nullptr;   // work units of the viscous face kernel
  int nvtiles = 0;
  void* fvis[3] = {nullptr, nullptr, nullptr};    // viscous face fluxes [nvfaces[d]][4], storage type
  struct EdgeItem { long long dst, dplane, s1, s1plane, s2, s2plane; };
  EdgeItem* d_edges = nullptr;      // depth-1 edge ghost fills
  long long nedges = 0;
  // residual monitor: RK stage 1 stores its residual (rmon) and reduces it
  // into mon_norm (see fv_set_monitor)
  int monitor = 0;
  bool mon_ran = false;
  void* rmon = nullptr;
  double* mon_partials = nullptr;
  double* mon_norm = nullptr;
  int device = 0, nsm = 0;
  // fv_rk_step's graphs, one per stream, each with its own device slot for
  // dt (set by a one-thread kernel on that stream when dt changes, so that a
  // new dt neither re-captures nor instantiates anything); at most
  // FV_MAX_GRAPHS streams, the least recently used evicted
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    double* dt_dev = nullptr;
    double dt = 0.0;
    unsigned long long used = 0;
  };
  std::map<cudaStream_t, StepGraph> graphs;
  unsigned long long graph_clock = 0;
  std::string err;
};

namespace {

int fail(fv_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

int cuda_fail(fv_ctx* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? FV_ERR_OOM : FV_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                          \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

inline long long ghosted_cells(int ni, int nj, int nk) {
  return (long long)(ni + 2 * FV_GHOST) * (nj + 2 * FV_GHOST) * (nk + 2 * FV_GHOST);
}

int storage_bytes(int precision) {
  return precision == FV_PREC_FP64 ? 8 : (precision == FV_PREC_DF64 ? 8 : 4);
}

// ---------------------------------------------------------------------------
// metrics: face vectors S = 1/2 (x_c - x_a) x (x_d - x_b), unit normals,
// areas, volumes = 1/3 sum of (face centroid . outward S)
// ---------------------------------------------------------------------------
struct NodeView {
  const double* x;
  int ni, nj;
  __device__ const double* at(int i, int j, int k) const {
    return x + 3 * (((long long)k * (nj + 1) + j) * (ni + 1) + i);
  }
};

__device__ void cross_half(const double* a, const double* b, const double* c, const double* d, double* S) {
  double d1[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  double d2[3] = {d[0] - b[0], d[1] - b[1], d[2] - b[2]};
  S[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
  S[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
  S[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
}

// face (dir, i, j, k): the low face of cell (i,j,k) normal to `dir`, nodes in order a b c d
__device__ void face_nodes(const NodeView& N, int dir, int i, int j, int k, const double* p[4]) {
  if (dir == 0) { p[0] = N.at(i, j, k); p[1] = N.at(i, j + 1, k); p[2] = N.at(i, j + 1, k + 1); p[3] = N.at(i, j, k + 1); }
  else if (dir == 1) { p[0] = N.at(i, j, k); p[1] = N.at(i, j, k + 1); p[2] = N.at(i + 1, j, k + 1); p[3] = N.at(i + 1, j, k); }
  else { p[0] = N.at(i, j, k); p[1] = N.at(i + 1, j, k); p[2] = N.at(i + 1, j + 1, k); p[3] = N.at(i, j + 1, k); }
}

__device__ __forceinline__ void store_metric(double* m, long long idx, double v) { m[idx] = v; }
__device__ __forceinline__ void store_metric(float2* m, long long idx, double v) {
  float h = (float)v;
  m[idx] = make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ void store_metric(float* m, long long idx, double v) { m[idx] = (float)v; }

template <class MT>
__global__ void metrics_faces_kernel(const double* nodes, int ni, int nj, int nk, int dir, MT* out,
                                     long long off, long long mstride) {
  const int ei = ni + (dir == 0), ej = nj + (dir == 1), ek = nk + (dir == 2);
  const long long n = (long long)ei * ej * ek;
  NodeView N{nodes, ni, nj};
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n; f += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(f % ei);
    const int j = (int)((f / ei) % ej);
    const int k = (int)(f / ((long long)ei * ej));
    const double* p[4];
    face_nodes(N, dir, i, j, k, p);
    double S[3];
    cross_half(p[0], p[1], p[2], p[3], S);
    const double A = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    // one record per face: (n_x, n_y, n_z, |S|)
    store_metric(out, 4 * (off + f), S[0] / A);
    store_metric(out, 4 * (off + f) + 1, S[1] / A);
    store_metric(out, 4 * (off + f) + 2, S[2] / A);
    store_metric(out, 4 * (off + f) + 3, A);
  }
}

__global__ void volume_kernel(const double* nodes, int ni, int nj, int nk, double* vol, double* invvol) {
  const long long n = (long long)ni * nj * nk;
  NodeView N{nodes, ni, nj};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % ni), j = (int)((c / ni) % nj), k = (int)(c / ((long long)ni * nj));
    double acc = 0.0;
    for (int dir = 0; dir < 3; ++dir)
      for (int side = 0; side < 2; ++side) {
        const double* p[4];
        face_nodes(N, dir, i + (dir == 0 ? side : 0), j + (dir == 1 ? side : 0), k + (dir == 2 ? side : 0), p);
        double S[3];
        cross_half(p[0], p[1], p[2], p[3], S);
        double m[3];
        for (int x = 0; x < 3; ++x) m[x] = 0.25 * (p[0][x] + p[1][x] + p[2][x] + p[3][x]);
        const double dot = m[0] * S[0] + m[1] * S[1] + m[2] * S[2];
        acc += side ? dot : -dot;
      }
    const double v = acc / 3.0;
    vol[c] = v;
    invvol[c] = 1.0 / v;
  }
}

// one value into device memory, in stream order (a replayed graph's dt)
__global__ void set_scalar_kernel(double* p, double v) { *p = v; }

__global__ void fill_kernel(double* p, long long n, double v) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) p[x] = v;
}

// S * Omega from S per unit volume (interior field layout)
__global__ void source_scale_kernel(const double* s, const double* vol, double* out, long long off5, long long ncell_b,
                                    long long cell_off) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < 5 * ncell_b; x += (long long)gridDim.x * blockDim.x) {
    const long long c = x % ncell_b;
    out[off5 + x] = s[off5 + x] * vol[cell_off + c];
  }
}

// binary64 -> (hi, lo) binary32 pairs
__global__ void split_kernel(const double* in, float2* out, long long n) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const double v = in[x];
    const float h = (float)v;
    out[x] = make_float2(h, (float)(v - (double)h));
  }
}

// ---------------------------------------------------------------------------
// ghost exchange.  A connection's items are (tangential a, b, depth d), a
// fastest; item (a, b, d) takes the ghost cell at depth d of the dst patch
// position (a, b) from the src interior cell at depth d under the signed
// tangential axis map.  XCH_COPY: dst ghost <- src donor, both blocks on
// this device (Section 2, Section 4).  Across devices (Section 7.2 V1,
// pack/unpack) the same items split into halves: XCH_PACK writes the donor
// cells of this device's src blocks into a contiguous slab buffer,
// XCH_UNPACK writes a received slab buffer into this device's dst ghosts.
// Connection c's slab occupies buf[5*item_off, 5*(item_off + n_c)),
// variable-major (n_c = 2 L0 L1 items: the 5 values of item x at x,
// x + n_c, ...).
//
// One CTA per tile of FV_XCH_TA x FV_XCH_TB positions and both depths
// (FvXchTile): it reads the tile's donor cells in the src block's memory
// order into shared memory and writes the ghosts in the dst block's order,
// so both sides run along i: the tangential axis that maps to i (a or b,
// through the axis map), or, on a face normal to i, the depth pair (two
// adjacent cells).  Slab buffers are read and written in item order.
// ---------------------------------------------------------------------------
enum { XCH_COPY = 0, XCH_PACK = 1, XCH_UNPACK = 2 };

// memory-contiguous index of a side: 0 = a, 1 = b, 2 = depth
__device__ __forceinline__ int xch_fast_dst(const FvConnDev& c) { return (c.dst_face >> 1) == 0 ? 2 : 0; }
__device__ __forceinline__ int xch_fast_src(const FvConnDev& c) {
  if ((c.src_face >> 1) == 0) return 2;
  return ((c.t0 < 0 ? -c.t0 : c.t0) == 1) ? 0 : 1;   // the item axis that maps to src tangential axis 0 = i
}

// t -> (a, b, d - 1) of a TA x TB x 2 tile with index `fast` fastest, then
// the others in (a, b, depth) order
__device__ __forceinline__ void xch_order(int t, int fast, int& a, int& b, int& d) {
  constexpr int TA = FV_XCH_TA, TB = FV_XCH_TB;
  if (fast == 0) { a = t % TA; b = (t / TA) % TB; d = t / (TA * TB); }
  else if (fast == 1) { b = t % TB; a = (t / TB) % TA; d = t / (TA * TB); }
  else { d = t & 1; a = (t >> 1) % TA; b = (t >> 1) / TA; }
}

__device__ __forceinline__ long long xch_dst_index(const FvBlockDev& D, const FvConnDev& c, int a, int b, int d) {
  const int da = c.dst_face >> 1;
  const int dext[3] = {D.ni, D.nj, D.nk};
  int dc[3];
  const int dt0 = da == 0 ? 1 : 0, dt1 = da == 2 ? 1 : 2;
  dc[dt0] = c.dlo0 + a;
  dc[dt1] = c.dlo1 + b;
  dc[da] = (c.dst_face & 1) ? dext[da] - 1 + d : -d;
  return D.qoff + (long long)(dc[2] + 2) * D.kstride + (long long)(dc[1] + 2) * D.jstride + (dc[0] + 2);
}

__device__ __forceinline__ long long xch_src_index(const FvBlockDev& S, const FvConnDev& c, int a, int b, int d) {
  const int sa = c.src_face >> 1;
  const int sext[3] = {S.ni, S.nj, S.nk};
  int sc[3];
  const int st0 = sa == 0 ? 1 : 0, st1 = sa == 2 ? 1 : 2;
  int st[2] = {c.slo0, c.slo1};
  const int u0 = (c.t0 < 0 ? -c.t0 : c.t0) - 1, u1 = (c.t1 < 0 ? -c.t1 : c.t1) - 1;
  st[u0] += c.t0 > 0 ? a : -a;
  st[u1] += c.t1 > 0 ? b : -b;
  sc[st0] = st[0];
  sc[st1] = st[1];
  sc[sa] = (c.src_face & 1) ? sext[sa] - d : d - 1;
  return S.qoff + (long long)(sc[2] + 2) * S.kstride + (long long)(sc[1] + 2) * S.jstride + (sc[0] + 2);
}

template <int MODE>
__global__ void __launch_bounds__(256) exchange_kernel(const FvBlockDev* __restrict__ blocks,
                                                       const FvConnDev* __restrict__ conns,
                                                       const FvXchTile* __restrict__ tiles, double* q, double* buf) {
  constexpr int TA = FV_XCH_TA, TB = FV_XCH_TB, N = 2 * TA * TB, P = TB * (TA + 1) * 2;
  // [variable][b][a][depth], a row padded by one position against bank
  // conflicts; all five variables are read before the one barrier, so each
  // thread has its items' five loads in flight together (42 KB)
  __shared__ double tile_v[5 * P];
  const FvXchTile T = tiles[blockIdx.x];
  const FvConnDev c = conns[T.conn];
  const long long nc = 2LL * c.L0 * c.L1;
  const int fs = MODE == XCH_UNPACK ? 0 : xch_fast_src(c);
  const int fd = MODE == XCH_PACK ? 0 : xch_fast_dst(c);
  const FvBlockDev* S = MODE == XCH_UNPACK ? nullptr : &blocks[c.src_block];
  const FvBlockDev* D = MODE == XCH_PACK ? nullptr : &blocks[c.dst_block];
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    int a, b, d;
    xch_order(t, fs, a, b, d);
    const int ga = T.a0 + a, gb = T.b0 + b;
    if (ga >= c.L0 || gb >= c.L1) continue;
    const int o = (b * (TA + 1) + a) * 2 + d;
    if (MODE == XCH_UNPACK) {
      const double* src = buf + 5 * c.item_off + ga + (long long)c.L0 * (gb + (long long)c.L1 * d);
#pragma unroll
      for (int v = 0; v < 5; ++v) tile_v[v * P + o] = src[v * nc];
    } else {
      const double* src = q + xch_src_index(*S, c, ga, gb, d + 1);
      const long long pl = S->plane;
#pragma unroll
      for (int v = 0; v < 5; ++v) tile_v[v * P + o] = src[v * pl];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    int a, b, d;
    xch_order(t, fd, a, b, d);
    const int ga = T.a0 + a, gb = T.b0 + b;
    if (ga >= c.L0 || gb >= c.L1) continue;
    const int o = (b * (TA + 1) + a) * 2 + d;
    if (MODE == XCH_PACK) {
      double* dst = buf + 5 * c.item_off + ga + (long long)c.L0 * (gb + (long long)c.L1 * d);
#pragma unroll
      for (int v = 0; v < 5; ++v) dst[v * nc] = tile_v[v * P + o];
    } else {
      double* dst = q + xch_dst_index(*D, c, ga, gb, d + 1);
      const long long pl = D->plane;
#pragma unroll
      for (int v = 0; v < 5; ++v) dst[v * pl] = tile_v[v * P + o];
    }
  }
}

// the tiles of a connection table, connection by connection
std::vector<FvXchTile> xch_tiles(const std::vector<FvConnDev>& cd) {
  std::vector<FvXchTile> out;
  for (int c = 0; c < (int)cd.size(); ++c)
    for (int b0 = 0; b0 < cd[c].L1; b0 += FV_XCH_TB)
      for (int a0 = 0; a0 < cd[c].L0; a0 += FV_XCH_TA) out.push_back(FvXchTile{c, a0, b0, 0});
  return out;
}

// ---------------------------------------------------------------------------
// physical boundaries: work item = (patch, tangential a, b); both ghost
// layers of that boundary position (Section 2; Section 7.2, V2/V3)
// ---------------------------------------------------------------------------
static_assert(FV_BCK_NOSLIP_WALL == FV_BC_NOSLIP_WALL, "boundary kinds");
static_assert(FV_BCK_SLIP_WALL == FV_BC_SLIP_WALL && FV_BCK_FARFIELD == FV_BC_FARFIELD &&
                  FV_BCK_SUPERSONIC_INFLOW == FV_BC_SUPERSONIC_INFLOW && FV_BCK_EXTRAPOLATE == FV_BC_EXTRAPOLATE,
              "boundary kinds");

__device__ __forceinline__ double metric_d(const double* m, long long i) { return m[i]; }
__device__ __forceinline__ double metric_d(const float2* m, long long i) {
  const float2 v = m[i];
  return (double)v.x + (double)v.y;
}
__device__ __forceinline__ double metric_d(const float* m, long long i) { return (double)m[i]; }

// gas constants of the boundary kernels (one division each, on the host)
struct BcGas {
  double g, gm1, igm1, k2, ig;   // gamma, gamma-1, 1/(gamma-1), 2/(gamma-1), 1/gamma
  int e;                         // 2/(gamma-1) when it is a small integer, else 0
};

__device__ __forceinline__ void bc_prim_to_cons(const double V[5], const BcGas& G, double q[5]) {
  q[0] = V[0];
  q[1] = V[0] * V[1];
  q[2] = V[0] * V[2];
  q[3] = V[0] * V[3];
  q[4] = V[4] * G.igm1 + 0.5 * V[0] * (V[1] * V[1] + V[2] * V[2] + V[3] * V[3]);
}

// Characteristic farfield state (1D Riemann invariants along the outward
// normal n) from the interior primitive state Vi with sound speed ci and the
// free stream Vf with sound speed cf.  FP64 is GB300's slow unit: two
// divisions' worth of work in all (the free-stream sound speed comes from
// the host, 1/(gamma-1) and 2/(gamma-1) are constants).
__device__ __forceinline__ void bc_farfield(const BcGas& G, const double Vi[5], double ci, const double Vf[5], double cf,
                                            const double n[3], double Vb[5]) {
  const double vni = Vi[1] * n[0] + Vi[2] * n[1] + Vi[3] * n[2];
  const double vnf = Vf[1] * n[0] + Vf[2] * n[1] + Vf[3] * n[2];
  if (vni >= ci || vni <= -ci) {
    const double* src = vni >= ci ? Vi : Vf;
    for (int m = 0; m < 5; ++m) Vb[m] = src[m];
    return;
  }
  const double rp = vni + G.k2 * ci, rm = vnf - G.k2 * cf;
  const double vnb = 0.5 * (rp + rm), cb = 0.25 * G.gm1 * (rp - rm);
  const bool out = vnb >= 0.0;
  const double* ref = out ? Vi : Vf;
  // equal entropy p / rho^gamma: rho_b = rho_ref (c_b / c_ref)^(2/(gamma-1)),
  // an integer power for gamma = 1.4 (and 5/3, ...); binary64 pow otherwise
  const double ratio = cb / (out ? ci : cf);
  double scale = ratio;
  if (G.e > 0) {
    for (int x = 1; x < G.e; ++x) scale *= ratio;
  } else {
    scale = pow(ratio, G.k2);
  }
  const double rhob = ref[0] * scale;
  const double vnr = ref[1] * n[0] + ref[2] * n[1] + ref[3] * n[2];
  Vb[0] = rhob;
  for (int m = 0; m < 3; ++m) Vb[1 + m] = ref[1 + m] + (vnb - vnr) * n[m];
  Vb[4] = rhob * cb * cb * G.ig;
}

template <class MT>
__global__ void bc_fill_kernel(const FvBlockDev* __restrict__ blocks, const FvBcDev* __restrict__ bcs, int nbc,
                               long long nitems, const MT* m0, const MT* m1, const MT* m2, BcGas G,
                               double* q) {
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < nitems;
       it += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = nbc - 1;
    while (lo < hi) {               // last patch with item_off <= it
      const int mid = (lo + hi + 1) >> 1;
      if (bcs[mid].item_off <= it) lo = mid; else hi = mid - 1;
    }
    const FvBcDev& P = bcs[lo];
    const long long local = it - P.item_off;
    const int a = (int)(local % P.L0), b = (int)(local / P.L0);
    const FvBlockDev& B = blocks[P.block];
    const int ax = P.face >> 1, side = P.face & 1;
    // tangential cell coordinates (scalars, so that nothing is indexed at run time)
    const int ti = ax == 0 ? 0 : P.lo0 + a;
    const int tj = ax == 0 ? P.lo0 + a : (ax == 1 ? 0 : P.lo1 + b);
    const int tk = ax == 2 ? 0 : P.lo1 + b;
    const int ext = ax == 0 ? B.ni : (ax == 1 ? B.nj : B.nk);
    const long long astride = ax == 0 ? 1 : (ax == 1 ? B.jstride : B.kstride);
    // state index of the cell at coordinate t along the face normal
    const long long base = B.qoff + (long long)(tk + 2) * B.kstride + (long long)(tj + 2) * B.jstride + (ti + 2) -
                           2 * astride;
    auto at = [&](int t) { return base + (long long)(t + 2) * astride; };
    // unit normal of the boundary face (pointing +axis)
    double n0, n1, n2;
    if (B.cartesian) {
      n0 = B.cart_n[ax][0]; n1 = B.cart_n[ax][1]; n2 = B.cart_n[ax][2];
    } else {
      const int tf = side ? ext : 0;
      const long long fi = B.face_off[ax] +
                           (ax == 0 ? ((long long)tk * B.nj + tj) * (B.ni + 1) + tf
                                    : (ax == 1 ? ((long long)tk * (B.nj + 1) + tf) * B.ni + ti
                                               : ((long long)tf * B.nj + tj) * B.ni + ti));
      const MT* m = ax == 0 ? m0 : (ax == 1 ? m1 : m2);
      n0 = metric_d(m, 4 * fi); n1 = metric_d(m, 4 * fi + 1); n2 = metric_d(m, 4 * fi + 2);
    }
    const long long i1 = at(side ? ext - 1 : 0);   // first interior cell
    double qb[5];
    if (P.kind == FV_BCK_SUPERSONIC_INFLOW) {
      for (int v = 0; v < 5; ++v) qb[v] = P.qstate[v];
    } else if (P.kind == FV_BCK_EXTRAPOLATE) {
      for (int v = 0; v < 5; ++v) qb[v] = q[i1 + v * B.plane];
    } else if (P.kind == FV_BCK_FARFIELD) {
      double qi[5], Vi[5], Vb[5];
      for (int v = 0; v < 5; ++v) qi[v] = q[i1 + v * B.plane];
      const double ri = 1.0 / qi[0];
      Vi[0] = qi[0];
      Vi[1] = qi[1] * ri;
      Vi[2] = qi[2] * ri;
      Vi[3] = qi[3] * ri;
      Vi[4] = G.gm1 * (qi[4] - 0.5 * (qi[1] * Vi[1] + qi[2] * Vi[2] + qi[3] * Vi[3]));
      const double ci = sqrt(G.g * Vi[4] * ri);
      const double sg = side ? 1.0 : -1.0;
      const double nout[3] = {sg * n0, sg * n1, sg * n2};
      const double Vf[5] = {P.state[0], P.state[1], P.state[2], P.state[3], P.state[4]};
      bc_farfield(G, Vi, ci, Vf, P.cstate, nout, Vb);
      bc_prim_to_cons(Vb, G, qb);
    }
#pragma unroll
    for (int d = 1; d <= FV_GHOST; ++d) {
      const long long gi = at(side ? ext - 1 + d : -d);
      if (P.kind == FV_BCK_NOSLIP_WALL) {
        // mirror of the interior cell at the same depth, momentum reversed
        const long long mi = at(side ? ext - d : d - 1);
        q[gi] = q[mi];
        q[gi + B.plane] = -q[mi + B.plane];
        q[gi + 2 * B.plane] = -q[mi + 2 * B.plane];
        q[gi + 3 * B.plane] = -q[mi + 3 * B.plane];
        q[gi + 4 * B.plane] = q[mi + 4 * B.plane];
      } else if (P.kind == FV_BCK_SLIP_WALL) {
        // mirror of the interior cell at the same depth, normal momentum reflected
        const long long mi = at(side ? ext - d : d - 1);
        const double mx = q[mi + B.plane], my = q[mi + 2 * B.plane], mz = q[mi + 3 * B.plane];
        const double mn2 = 2.0 * (mx * n0 + my * n1 + mz * n2);
        q[gi] = q[mi];
        q[gi + B.plane] = mx - mn2 * n0;
        q[gi + 2 * B.plane] = my - mn2 * n1;
        q[gi + 3 * B.plane] = mz - mn2 * n2;
        q[gi + 4 * B.plane] = q[mi + 4 * B.plane];
      } else if (P.kind != FV_BCK_FIXED) {
#pragma unroll
        for (int v = 0; v < 5; ++v) q[gi + v * B.plane] = qb[v];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// viscous terms: auxiliary-volume geometry (setup) and edge ghosts (per stage)
// ---------------------------------------------------------------------------

// Omega and the cell-averaged face vectors of every interior cell of a
// curvilinear block, in its padded box
__global__ void geo_cells_kernel(const double* nodes, int ni, int nj, int nk, const double* vol, long long pad_off,
                                 long long P, double* geo) {
  const long long n = (long long)ni * nj * nk;
  NodeView N{nodes, ni, nj};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % ni), j = (int)((c / ni) % nj), k = (int)(c / ((long long)ni * nj));
    const long long pc = pad_off + ((long long)(k + 1) * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1);
    geo[pc] = vol[c];
    for (int dir = 0; dir < 3; ++dir) {
      const double* p[4];
      double lo[3], hi[3];
      face_nodes(N, dir, i, j, k, p);
      cross_half(p[0], p[1], p[2], p[3], lo);
      face_nodes(N, dir, i + (dir == 0), j + (dir == 1), k + (dir == 2), p);
      cross_half(p[0], p[1], p[2], p[3], hi);
      for (int x = 0; x < 3; ++x) geo[(1 + 3 * dir + x) * P + pc] = 0.5 * (lo[x] + hi[x]);
    }
  }
}

// the same for a Cartesian block (every cell alike)
__global__ void geo_cart_kernel(FvBlockDev B, long long P, double* geo) {
  const long long n = (long long)B.ni * B.nj * B.nk;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % B.ni), j = (int)((c / B.ni) % B.nj), k = (int)(c / ((long long)B.ni * B.nj));
    const long long pc = B.pad_off + ((long long)(k + 1) * (B.nj + 2) + (j + 1)) * (B.ni + 2) + (i + 1);
    geo[pc] = 1.0 / B.cart_invvol;
    for (int dir = 0; dir < 3; ++dir)
      for (int x = 0; x < 3; ++x) geo[(1 + 3 * dir + x) * P + pc] = B.cart_n[dir][x] * B.cart_area[dir];
  }
}

// geometry planes [10][P] in binary64 -> per-cell records [P][12] in the
// storage type of a form (the last two entries of a record are padding)
template <class MT>
__global__ void geo_records_kernel(const double* in, MT* out, long long P) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < P; x += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < 10; ++c) store_metric(out, 12 * x + c, in[c * P + x]);
    store_metric(out, 12 * x + 10, 0.0);
    store_metric(out, 12 * x + 11, 0.0);
  }
}

// per-face gradient geometry of one block and direction (binary64 in, the
// storage type out): G_d = (Sbar_d(L) + Sbar_d(R)) / 2 / Omega_f for the
// face's own family a and the tangential families b, c, Omega_f =
// (Omega_L + Omega_R) / 2, then the face's area vector S = n |S|
template <class MT>
__global__ void face_geometry_kernel(FvBlockDev B, int dir, const double* geo, long long P, const MT* metric,
                                     MT* out) {
  const int ei = B.ni + (dir == 0), ej = B.nj + (dir == 1), ek = B.nk + (dir == 2);
  const long long n = (long long)ei * ej * ek;
  const long long pi = B.ni + 2, pij = pi * (B.nj + 2);
  const long long sa = dir == 0 ? 1 : (dir == 1 ? pi : pij);
  const int fam[3] = {dir, dir == 0 ? 1 : 0, dir == 2 ? 1 : 2};
  for (long long loc = blockIdx.x * (long long)blockDim.x + threadIdx.x; loc < n;
       loc += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(loc % ei), j = (int)((loc / ei) % ej), k = (int)(loc / ((long long)ei * ej));
    const long long pR = B.pad_off + (k + 1) * pij + (long long)(j + 1) * pi + (i + 1), pL = pR - sa;
    const long long o = 12 * (B.vface_off[dir] + loc);
    const double om = 0.5 * (geo[pL] + geo[pR]);
    for (int d = 0; d < 3; ++d)
      for (int x = 0; x < 3; ++x) {
        const long long r = (long long)(1 + 3 * fam[d] + x) * P;
        store_metric(out, o + 3 * d + x, 0.5 * (geo[r + pL] + geo[r + pR]) / om);
      }
    for (int x = 0; x < 3; ++x) {
      double S;
      if (B.cartesian) {
        S = B.cart_n[dir][x] * B.cart_area[dir];
      } else {
        const long long m = 4 * (B.face_off[dir] + loc);
        S = metric_d(metric, m + x) * metric_d(metric, m + 3);
      }
      store_metric(out, o + 9 + x, S);
    }
  }
}

// ghost-cell geometry: dst <- src with face family d taken from family
// fam_d of the source, times sign_d (code: fam0 | fam1 << 2 | fam2 << 4,
// negative signs in bits 6, 7, 8)
struct GeoItem { long long dst, src; int code, pad_; };

__global__ void geo_ghost_kernel(const GeoItem* __restrict__ items, long long n, long long P, double* geo) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const GeoItem it = items[x];
    geo[it.dst] = geo[it.src];
    for (int d = 0; d < 3; ++d) {
      const int fam = (it.code >> (2 * d)) & 3;
      const double sg = (it.code >> (6 + d)) & 1 ? -1.0 : 1.0;
      for (int c = 0; c < 3; ++c) geo[(1 + 3 * d + c) * P + it.dst] = sg * geo[(1 + 3 * fam + c) * P + it.src];
    }
  }
}

__global__ void edge_fill_kernel(const fv_ctx::EdgeItem* __restrict__ items, long long n, double* q) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const fv_ctx::EdgeItem it = items[x];
    if (it.s2 < 0) {
      for (int v = 0; v < 5; ++v) q[it.dst + v * it.dplane] = q[it.s1 + v * it.s1plane];
    } else {
      for (int v = 0; v < 5; ++v)
        q[it.dst + v * it.dplane] = 0.5 * (q[it.s1 + v * it.s1plane] + q[it.s2 + v * it.s2plane]);
    }
  }
}

// ---------------------------------------------------------------------------
// residual norms (deterministic two-level reduction)
// ---------------------------------------------------------------------------
int grid_for(long long n, int threads, int nsm) {
  long long g = (n + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(g, (long long)nsm * 16));
}

fv_ctx* H(fv_handle h) { return reinterpret_cast<fv_ctx*>(h); }

// destroy the cached RK-step graphs after the device is idle, so that no
// graph that may still run reads a dt slot being freed
void drop_graphs(fv_ctx* h) {
  if (h->graphs.empty()) return;
  cudaDeviceSynchronize();
  for (auto& g : h->graphs) {
    cudaGraphExecDestroy(g.second.exec);
    cudaFree(g.second.dt_dev);
  }
  h->graphs.clear();
}

// laminar viscous terms of state q: face variables, then the face fluxes of
// every direction (they feed the fused kernel through FvStageArgs::fv)
int do_visc(fv_ctx* h, const double* q, cudaStream_t s) {
  FvViscArgs v;
  std::memset(&v, 0, sizeof(v));
  v.blocks = h->d_blocks;
  v.tiles = h->d_vtiles;
  v.ntiles = h->nvtiles;
  v.q = q;
  for (int d = 0; d < h->cfg.dim; ++d) {
    v.fgeo[d] = h->fgeo[d];
    v.fv[d] = h->fvis[d];
  }
  v.vp.gamma = h->cfg.gamma;
  v.vp.mu = h->cfg.mu;
  v.vp.r_gas = h->cfg.r_gas;
  v.vp.kfac = h->cfg.gamma * h->cfg.r_gas / ((h->cfg.gamma - 1.0) * h->cfg.prandtl);
  v.vp.t_ref = h->cfg.t_ref;
  v.vp.s_suth = h->cfg.s_suth;
  v.vp.sutherland = h->cfg.sutherland;
  v.vp.dim = h->cfg.dim;
  if (fv_visc_faces(v, h->cfg.precision == FV_PREC_FP64 ? 0 : 1, s))
    return cuda_fail(h, cudaGetLastError(), "viscous face fluxes");
  return FV_OK;
}

// the compiled stage kernel variant of the handle's form, scheme, viscous
// terms and boundary overwrites
struct StageVariant {
  int (*launch)(const FvStageArgs&, const FvLaunch&, cudaStream_t);
  int (*occupancy)(const FvLaunch&, size_t*);
};
StageVariant stage_variant(const fv_ctx* h) {
#define FV_VARIANT_ENTRY(NAME) {fv_launch_stage_##NAME, fv_stage_occupancy_##NAME},
  // in FV_STAGE_VARIANTS order: [form][fast][visc][bc]
  static const StageVariant table[] = {FV_STAGE_VARIANTS(FV_VARIANT_ENTRY)};
#undef FV_VARIANT_ENTRY
  const FvLaunch& l = h->launch;
  const int form = h->cfg.precision == FV_PREC_FP64 ? 0 : (h->cfg.precision == FV_PREC_DF64 ? 1 : 2);
  return table[8 * form + (l.fast ? 4 : 0) + (l.visc ? 2 : 0) + (l.bc ? 1 : 0)];
}

int launch_stage(fv_ctx* h, const FvStageArgs& a, cudaStream_t s) {
  int rc;
  const FvLaunch& l = h->launch;
  if (l.visc && h->cfg.precision != FV_PREC_FP32FLUX) {
    // binary64 and double-float: the viscous fluxes by the separate kernel
    rc = do_visc(h, a.qin, s);
    if (rc) return rc;
  }
  rc = stage_variant(h).launch(a, l, s);
  if (rc == -2) return fail(h, FV_ERR_UNSUPPORTED, "tile shape not compiled");
  if (rc != 0) return cuda_fail(h, cudaGetLastError(), "stage kernel launch");
  return FV_OK;
}

FvStageArgs base_args(fv_ctx* h) {
  FvStageArgs a;
  std::memset(&a, 0, sizeof(a));
  a.blocks = h->d_blocks;
  a.tiles = h->d_tiles;
  a.ntiles = h->ntiles;
  a.tile_counter = h->d_tile_counter;
  for (int d = 0; d < 3; ++d) { a.metric[d] = h->metric[d]; a.mstride[d] = h->nfaces[d]; }
  a.invvol = h->invvol;
  a.srcvol = h->srcvol;
  a.srcvol2 = h->srcvol2;
  a.ncell_total = h->ncell;
  a.fp.gamma = h->cfg.gamma;
  a.fp.eps = h->cfg.eps;
  a.fp.kappa = h->cfg.kappa;
  a.fp.harten = h->cfg.harten;
  a.fp.va_delta2 = h->cfg.va_delta2;
  a.fp.limiter = h->cfg.limiter;
  a.fp.fix_all = h->cfg.fix_all;
  a.fp.flux = h->cfg.flux;
  if (h->launch.visc && h->cfg.precision == FV_PREC_FP32FLUX) {
    // binary32: viscous terms fused into the stage kernel
    a.geo = h->geo_t;
    a.vp.gamma = h->cfg.gamma;
    a.vp.mu = h->cfg.mu;
    a.vp.r_gas = h->cfg.r_gas;
    a.vp.kfac = h->cfg.gamma * h->cfg.r_gas / ((h->cfg.gamma - 1.0) * h->cfg.prandtl);
    a.vp.t_ref = h->cfg.t_ref;
    a.vp.s_suth = h->cfg.s_suth;
    a.vp.sutherland = h->cfg.sutherland;
    a.vp.dim = h->cfg.dim;
  } else if (h->cfg.visc) {
    for (int d = 0; d < h->cfg.dim; ++d) a.fv[d] = h->fvis[d];
  }
  return a;
}

int stage_in(const fv_ctx* h, int m) {
  if (m == 1) return 0;
  const int M = h->cfg.n_stages;
  const int prev = m - 1;
  return prev == M ? 0 : ((prev & 1) ? 1 : 2);
}
int stage_out(const fv_ctx* h, int m) {
  return m == h->cfg.n_stages ? 0 : ((m & 1) ? 1 : 2);
}

// connections first, then the physical boundaries
int do_exchange(fv_ctx* h, double* q, cudaStream_t s) {
  const int threads = 256;
  if (h->nxtiles) {
    exchange_kernel<XCH_COPY><<<h->nxtiles, threads, 0, s>>>(h->d_blocks, h->d_conns, h->d_xtiles, q, nullptr);
    CK(h, cudaGetLastError());
  }
  if (h->bc_items) {
    const int grid = grid_for(h->bc_items, threads, h->nsm);
    const long long* ms = h->nfaces;
    BcGas G;
    G.g = h->cfg.gamma;
    G.gm1 = G.g - 1.0;
    G.igm1 = 1.0 / G.gm1;
    G.k2 = 2.0 / G.gm1;
    G.ig = 1.0 / G.g;
    G.e = (G.k2 == std::rint(G.k2) && G.k2 >= 1.0 && G.k2 <= 16.0) ? (int)G.k2 : 0;
    if (h->cfg.precision == FV_PREC_FP64) {
      bc_fill_kernel<double><<<grid, threads, 0, s>>>(h->d_blocks, h->d_bcs, h->nbc, h->bc_items,
                                                      (const double*)h->metric[0], (const double*)h->metric[1],
                                                      (const double*)h->metric[2], G, q);
    } else if (h->cfg.precision == FV_PREC_DF64) {
      bc_fill_kernel<float2><<<grid, threads, 0, s>>>(h->d_blocks, h->d_bcs, h->nbc, h->bc_items,
                                                      (const float2*)h->metric[0], (const float2*)h->metric[1],
                                                      (const float2*)h->metric[2], G, q);
    } else {
      bc_fill_kernel<float><<<grid, threads, 0, s>>>(h->d_blocks, h->d_bcs, h->nbc, h->bc_items,
                                                     (const float*)h->metric[0], (const float*)h->metric[1],
                                                     (const float*)h->metric[2], G, q);
    }
    CK(h, cudaGetLastError());
  }
  if (h->nedges) {
    edge_fill_kernel<<<grid_for(h->nedges, 256, h->nsm), 256, 0, s>>>(h->d_edges, h->nedges, q);
    CK(h, cudaGetLastError());
  }
  return FV_OK;
}

// dt_dev: null, or device memory holding dt (a captured graph reads it at
// replay; alpha_m * dt is then formed by the kernel, the same binary64 product)
int do_stage(fv_ctx* h, int m, double dt, cudaStream_t s, const double* dt_dev = nullptr) {
  const int bi = stage_in(h, m), bo = stage_out(h, m);
  int rc = do_exchange(h, h->buf[bi], s);
  if (rc) return rc;
  FvStageArgs a = base_args(h);
  a.mode = FV_MODE_RK;
  a.qin = h->buf[bi];
  a.q0 = h->buf[0];
  a.qout = h->buf[bo];
  a.alpha_dt = h->cfg.alpha[m - 1] * dt;
  a.alpha = h->cfg.alpha[m - 1];
  a.dt_dev = dt_dev;
  const bool mon = m == 1 && h->monitor;
  if (mon) a.rmon = h->rmon;
  rc = launch_stage(h, a, s);
  if (rc || !mon) return rc;
  if (fv_monitor_reduce(h->rmon, h->cfg.precision == FV_PREC_FP64, h->ncell, h->mon_partials, FV_NORM_PARTS * h->nsm,
                        h->mon_norm, s))
    return cuda_fail(h, cudaGetLastError(), "residual monitor reduction");
  h->mon_ran = true;
  return FV_OK;
}

// copy between the packed ghosted layout and the internal layout (identical
// when pitch == ni+4)
int copy_state(fv_ctx* h, const double* src, double* dst, bool to_internal, cudaStream_t s) {
  // rows of the internal layout are unpadded, so the packed and internal
  // layouts coincide: one flat copy (a pitched copy of ~1 KB rows runs far
  // below the host link's bandwidth when one side is host memory)
  bool flat = h->state_elems == h->ext_state_elems;
  long long off = 0;
  for (const FvBlockDev& b : h->hb) {
    flat = flat && b.pitch == b.ni + 2 * FV_GHOST && b.qoff == off;
    off += 5 * ghosted_cells(b.ni, b.nj, b.nk);
  }
  if (flat) {
    CK(h, cudaMemcpyAsync(dst, src, sizeof(double) * h->ext_state_elems, cudaMemcpyDefault, s));
    return FV_OK;
  }
  long long ext = 0;
  for (const FvBlockDev& b : h->hb) {
    const long long cells = ghosted_cells(b.ni, b.nj, b.nk);
    const size_t wbytes = sizeof(double) * (b.ni + 4);
    const size_t rows = (size_t)(b.nj + 4) * (b.nk + 4);
    for (int v = 0; v < 5; ++v) {
      const double* e = (to_internal ? src : dst) + ext + v * cells;
      double* in = (to_internal ? dst : const_cast<double*>(src)) + b.qoff + v * b.plane;
      if (to_internal)
        CK(h, cudaMemcpy2DAsync(in, sizeof(double) * b.pitch, e, wbytes, wbytes, rows, cudaMemcpyDefault, s));
      else
        CK(h, cudaMemcpy2DAsync(const_cast<double*>(e), wbytes, in, sizeof(double) * b.pitch, wbytes, rows,
                                cudaMemcpyDefault, s));
    }
    ext += 5 * cells;
  }
  return FV_OK;
}

void choose_launch(fv_ctx* h) {
  const fv_config& c = h->cfg;
  FvLaunch l{};
  l.three_d = c.dim == 3;
  int shape = c.tile;
  if (shape <= 0) {
    // automatic: narrow blocks prefer narrow tiles
    int maxni = 0;
    for (auto& b : h->hb) maxni = std::max(maxni, b.ni);
    shape = maxni >= 24 ? 1 : 3;
  }
  shape = std::min(std::max(shape, 1), FV_NUM_SHAPES);
  l.shape = shape;
  l.tx = FV_SHAPE_TABLE[shape - 1][0];
  l.ty = FV_SHAPE_TABLE[shape - 1][1];
  l.threads = FV_SHAPE_TABLE[shape - 1][2];
  l.fast = fv_default_scheme(c.flux, c.limiter, c.eps, c.kappa, c.harten, c.fix_all);
  // viscous kernels: the binary32 form fuses the viscous faces into the
  // stage kernel (its T on the fly costs a MUFU reciprocal); for binary64
  // and double-float a separate kernel measured faster, and their _visc
  // stage kernels subtract its per-face fluxes
  l.visc = c.visc != 0;
  l.bc = 0;
  for (const FvBlockDev& b : h->hb) l.bc |= b.bcmap != nullptr;
  h->launch = l;
}

int query_occupancy(fv_ctx* h, size_t* smem) { return stage_variant(h).occupancy(h->launch, smem); }

int build_tiles(fv_ctx* h) {
  const FvLaunch& l = h->launch;
  size_t smem = 0;
  const int occ = query_occupancy(h, &smem);
  if (occ <= 0) return fail(h, FV_ERR_UNSUPPORTED, "stage kernel cannot be resident with this tile shape");
  const long long slots = (long long)h->nsm * occ;
  long long columns = 0;
  for (auto& b : h->hb) columns += (long long)((b.ni + l.tx - 1) / l.tx) * ((b.nj + l.ty - 1) / l.ty);
  std::vector<FvTile> tiles;
  std::vector<long long> cost;
  for (int bi = 0; bi < (int)h->hb.size(); ++bi) {
    const FvBlockDev& b = h->hb[bi];
    int kc = h->cfg.kchunk;
    if (h->cfg.dim == 2) kc = 1;
    else if (kc == 0) {
      // split k so that the whole problem fills the resident CTA slots a few times
      const long long want = std::max<long long>(1, (3 * slots + columns - 1) / std::max<long long>(columns, 1));
      kc = (int)std::max<long long>(4, (b.nk + want - 1) / want);
    } else if (kc < 0) {
      // -w: about w tiles per resident CTA slot
      const long long want = std::max<long long>(1, (-kc * slots) / std::max<long long>(columns, 1));
      kc = (int)std::max<long long>(2, (b.nk + want - 1) / want);
    }
    kc = std::min(kc, b.nk);
    for (int k0 = 0; k0 < b.nk; k0 += kc)
      for (int j0 = 0; j0 < b.nj; j0 += l.ty)
        for (int i0 = 0; i0 < b.ni; i0 += l.tx) {
          const int k1 = std::min(b.nk, k0 + kc);
          FvTile t{bi, i0, j0, k0 | (k1 << 16)};
          tiles.push_back(t);
          cost.push_back((long long)std::min(l.tx, b.ni - i0) * std::min(l.ty, b.nj - j0) * (k1 - k0 + 2));
        }
  }
  // largest tiles first (static round-robin assignment then balances better)
  std::vector<int> order(tiles.size());
  for (size_t x = 0; x < order.size(); ++x) order[x] = (int)x;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<FvTile> sorted;
  for (int x : order) sorted.push_back(tiles[x]);
  h->ntiles = (int)sorted.size();
  h->launch.grid = (int)std::min<long long>(h->ntiles, slots);
  if (h->d_tiles) { cudaFree(h->d_tiles); h->d_tiles = nullptr; }
  CK(h, cudaMalloc(&h->d_tiles, sizeof(FvTile) * sorted.size()));
  CK(h, cudaMemcpy(h->d_tiles, sorted.data(), sizeof(FvTile) * sorted.size(), cudaMemcpyHostToDevice));
  return FV_OK;
}

// ---------------------------------------------------------------------------
// viscous-term tables (host): ghost geometry items and edge-ghost items
// ---------------------------------------------------------------------------
long long pad_index(const FvBlockDev& B, int i, int j, int k) {
  return B.pad_off + ((long long)(k + 1) * (B.nj + 2) + (j + 1)) * (B.ni + 2) + (i + 1);
}
long long state_index(const FvBlockDev& B, int i, int j, int k) {
  return B.qoff + (long long)(k + 2) * B.kstride + (long long)(j + 2) * B.jstride + (i + 2);
}
// tangential axes of a face normal to axis a, in (i, j, k) order
void tangential(int a, int t[2]) {
  t[0] = a == 0 ? 1 : 0;
  t[1] = a == 2 ? 1 : 2;
}
// donor cell (depth 1) of dst tangential coordinates (u0, u1) of connection c
// (u may lie one cell outside the patch)
void donor_cell(const fv_ctx* h, const fv_connection& c, int u0, int u1, int sc[3]) {
  const FvBlockDev& S = h->hb[c.src_block];
  const int sa = c.src_face / 2;
  int st[2];
  tangential(sa, st);
  int v[2] = {c.src_lo[0], c.src_lo[1]};
  const int a = u0 - c.dst_lo[0], b = u1 - c.dst_lo[1];
  v[std::abs(c.transform[0]) - 1] += c.transform[0] > 0 ? a : -a;
  v[std::abs(c.transform[1]) - 1] += c.transform[1] > 0 ? b : -b;
  const int sext[3] = {S.ni, S.nj, S.nk};
  sc[st[0]] = v[0];
  sc[st[1]] = v[1];
  sc[sa] = (c.src_face & 1) ? sext[sa] - 1 : 0;
}

int build_visc_tables(fv_ctx* h) {
  // ghost geometry: copies of the adjacent interior cell, then the donors
  std::vector<GeoItem> copies, donors;
  const int ident = 0 | (1 << 2) | (2 << 4);
  for (const FvBlockDev& B : h->hb) {
    const int ext[3] = {B.ni, B.nj, B.nk};
    for (int f = 0; f < 6; ++f) {
      const int a = f / 2;
      int t[2];
      tangential(a, t);
      for (int u1 = 0; u1 < ext[t[1]]; ++u1)
        for (int u0 = 0; u0 < ext[t[0]]; ++u0) {
          int g[3], in[3];
          g[t[0]] = in[t[0]] = u0;
          g[t[1]] = in[t[1]] = u1;
          g[a] = (f & 1) ? ext[a] : -1;
          in[a] = (f & 1) ? ext[a] - 1 : 0;
          copies.push_back(GeoItem{pad_index(B, g[0], g[1], g[2]), pad_index(B, in[0], in[1], in[2]), ident, 0});
        }
    }
  }
  for (const fv_connection& c : h->conns) {
    const FvBlockDev& D = h->hb[c.dst_block];
    const FvBlockDev& S = h->hb[c.src_block];
    const int da = c.dst_face / 2, sa = c.src_face / 2;
    int dt[2], st[2];
    tangential(da, dt);
    tangential(sa, st);
    int fam[3], neg[3];
    fam[da] = sa;
    neg[da] = (c.dst_face & 1) == (c.src_face & 1);   // index direction reverses
    for (int x = 0; x < 2; ++x) {
      fam[dt[x]] = st[std::abs(c.transform[x]) - 1];
      neg[dt[x]] = c.transform[x] < 0;
    }
    const int code = fam[0] | (fam[1] << 2) | (fam[2] << 4) | (neg[0] << 6) | (neg[1] << 7) | (neg[2] << 8);
    const int dext[3] = {D.ni, D.nj, D.nk};
    for (int u1 = c.dst_lo[1]; u1 < c.dst_hi[1]; ++u1)
      for (int u0 = c.dst_lo[0]; u0 < c.dst_hi[0]; ++u0) {
        int g[3], sc[3];
        g[dt[0]] = u0;
        g[dt[1]] = u1;
        g[da] = (c.dst_face & 1) ? dext[da] : -1;
        donor_cell(h, c, u0, u1, sc);
        donors.push_back(GeoItem{pad_index(D, g[0], g[1], g[2]), pad_index(S, sc[0], sc[1], sc[2]), code, 0});
      }
  }
  for (const auto* list : {&copies, &donors}) {
    if (list->empty()) continue;
    GeoItem* d = nullptr;
    CK(h, cudaMalloc(&d, sizeof(GeoItem) * list->size()));
    CK(h, cudaMemcpy(d, list->data(), sizeof(GeoItem) * list->size(), cudaMemcpyHostToDevice));
    geo_ghost_kernel<<<grid_for((long long)list->size(), 256, h->nsm), 256>>>(d, (long long)list->size(), h->pad_total,
                                                                          h->geo);
    CK(h, cudaDeviceSynchronize());
    cudaFree(d);
  }
  // depth-1 edge ghosts: a connection of either face extended by one cell
  // along the face (faces of the lower axis first, connections in table
  // order), else the mean of the two face-adjacent ghosts
  std::vector<fv_ctx::EdgeItem> edges;
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  const int npairs = h->cfg.dim == 3 ? 3 : 1;
  for (int bk = 0; bk < h->nblocks; ++bk) {
    const FvBlockDev& B = h->hb[bk];
    const int ext[3] = {B.ni, B.nj, B.nk};
    for (int pr = 0; pr < npairs; ++pr) {
      const int a = pairs[pr][0], b = pairs[pr][1], c3 = 3 - a - b;
      const int nc = h->cfg.dim == 3 ? ext[c3] : 1;
      for (int sa = 0; sa < 2; ++sa)
        for (int sb = 0; sb < 2; ++sb)
          for (int t = 0; t < nc; ++t) {
            int e[3];
            e[a] = sa ? ext[a] : -1;
            e[b] = sb ? ext[b] : -1;
            e[c3] = t;
            fv_ctx::EdgeItem it{state_index(B, e[0], e[1], e[2]), B.plane, 0, 0, -1, 0};
            bool found = false;
            for (int pass = 0; pass < 2 && !found; ++pass) {
              const int fa = pass == 0 ? a : b, other = pass == 0 ? b : a;
              const int face = 2 * fa + (pass == 0 ? sa : sb);
              int tn[2];
              tangential(fa, tn);
              for (const fv_connection& c : h->conns) {
                if (c.dst_block != bk || c.dst_face != face) continue;
                bool inside = true;
                for (int x = 0; x < 2; ++x) {
                  const int lo = c.dst_lo[x] - (tn[x] == other), hi = c.dst_hi[x] + (tn[x] == other);
                  if (e[tn[x]] < lo || e[tn[x]] >= hi) inside = false;
                }
                if (!inside) continue;
                int sc[3];
                donor_cell(h, c, e[tn[0]], e[tn[1]], sc);
                const FvBlockDev& S = h->hb[c.src_block];
                it.s1 = state_index(S, sc[0], sc[1], sc[2]);
                it.s1plane = S.plane;
                found = true;
                break;
              }
            }
            if (!found) {
              int f1[3] = {e[0], e[1], e[2]}, f2[3] = {e[0], e[1], e[2]};
              f1[b] = sb ? ext[b] - 1 : 0;
              f2[a] = sa ? ext[a] - 1 : 0;
              it.s1 = state_index(B, f1[0], f1[1], f1[2]);
              it.s1plane = B.plane;
              it.s2 = state_index(B, f2[0], f2[1], f2[2]);
              it.s2plane = B.plane;
            }
            edges.push_back(it);
          }
    }
  }
  h->nedges = (long long)edges.size();
  if (h->nedges) {
    CK(h, cudaMalloc(&h->d_edges, sizeof(fv_ctx::EdgeItem) * edges.size()));
    CK(h, cudaMemcpy(h->d_edges, edges.data(), sizeof(fv_ctx::EdgeItem) * edges.size(), cudaMemcpyHostToDevice));
  }
  return FV_OK;
}

int validate(const fv_block_desc* blocks, int nblocks, const fv_connection* conns, int nconn, const fv_config* cfg) {
  if (!blocks || nblocks <= 0) return fail(nullptr, FV_ERR_INVALID_ARG, "no blocks");
  if (!cfg) return fail(nullptr, FV_ERR_INVALID_ARG, "no config");
  if (cfg->dim != 2 && cfg->dim != 3) return fail(nullptr, FV_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (cfg->n_stages < 2 || cfg->n_stages > 8) return fail(nullptr, FV_ERR_INVALID_ARG, "n_stages must be 2..8");
  if (cfg->precision < 0 || cfg->precision > 2) return fail(nullptr, FV_ERR_INVALID_ARG, "unknown precision");
  if (cfg->limiter < 0 || cfg->limiter > 2) return fail(nullptr, FV_ERR_INVALID_ARG, "unknown limiter");
  if (cfg->flux < 0 || cfg->flux > 2) return fail(nullptr, FV_ERR_INVALID_ARG, "unknown face flux");
  if (!(cfg->gamma > 1.0)) return fail(nullptr, FV_ERR_INVALID_ARG, "gamma must exceed 1");
  if (cfg->visc != 0 && cfg->visc != 1) return fail(nullptr, FV_ERR_INVALID_ARG, "visc must be 0 or 1");
  if (cfg->visc && !(cfg->mu >= 0.0 && cfg->prandtl > 0.0 && cfg->r_gas > 0.0 &&
                     (!cfg->sutherland || (cfg->t_ref > 0.0 && cfg->s_suth >= 0.0))))
    return fail(nullptr, FV_ERR_INVALID_ARG, "viscous parameters: need mu >= 0, prandtl > 0, r_gas > 0, t_ref > 0, s_suth >= 0");
  for (int b = 0; b < nblocks; ++b) {
    const fv_block_desc& d = blocks[b];
    if (d.ni < 1 || d.nj < 1 || d.nk < 1 || d.ni > 32000 || d.nj > 32000 || d.nk > 16000)
      return fail(nullptr, FV_ERR_INVALID_ARG, "block " + std::to_string(b) + ": extents out of range");
    if (cfg->dim == 2 && d.nk != 1) return fail(nullptr, FV_ERR_INVALID_ARG, "dim 2 needs nk == 1");
    if (!d.nodes && !(d.h[0] > 0 && d.h[1] > 0 && d.h[2] > 0))
      return fail(nullptr, FV_ERR_INVALID_ARG, "block " + std::to_string(b) + ": Cartesian spacing must be positive");
  }
  // ranges and overlap of dst ghost patches
  std::vector<std::vector<std::vector<char>>> used(nblocks, std::vector<std::vector<char>>(6));
  for (int c = 0; c < nconn; ++c) {
    const fv_connection& x = conns[c];
    const std::string tag = "connection " + std::to_string(c) + ": ";
    if (x.dst_block < 0 || x.dst_block >= nblocks || x.src_block < 0 || x.src_block >= nblocks)
      return fail(nullptr, FV_ERR_INVALID_ARG, tag + "block index out of range");
    if (x.dst_face < 0 || x.dst_face > 5 || x.src_face < 0 || x.src_face > 5)
      return fail(nullptr, FV_ERR_INVALID_ARG, tag + "face out of range");
    if (cfg->dim == 2 && (x.dst_face >= 4 || x.src_face >= 4))
      return fail(nullptr, FV_ERR_INVALID_ARG, tag + "k faces do not exist in 2D");
    const fv_block_desc& D = blocks[x.dst_block];
    const fv_block_desc& S = blocks[x.src_block];
    const int dext[3] = {D.ni, D.nj, D.nk}, sext[3] = {S.ni, S.nj, S.nk};
    const int da = x.dst_face / 2, sa = x.src_face / 2;
    int dt[2], st[2], n = 0, m = 0;
    for (int a = 0; a < 3; ++a) { if (a != da) dt[n++] = a; if (a != sa) st[m++] = a; }
    for (int t = 0; t < 2; ++t)
      if (x.dst_lo[t] < 0 || x.dst_hi[t] > dext[dt[t]] || x.dst_lo[t] >= x.dst_hi[t])
        return fail(nullptr, FV_ERR_INVALID_ARG, tag + "dst patch outside the face");
    const int t0 = x.transform[0], t1 = x.transform[1];
    if (!(std::abs(t0) == 1 || std::abs(t0) == 2) || !(std::abs(t1) == 1 || std::abs(t1) == 2) || std::abs(t0) == std::abs(t1))
      return fail(nullptr, FV_ERR_INVALID_ARG, tag + "transform must be a signed permutation of (1,2)");
    if (sext[sa] < FV_GHOST) return fail(nullptr, FV_ERR_INVALID_ARG, tag + "src block thinner than the ghost depth");
    for (int t = 0; t < 2; ++t) {
      const int T = t == 0 ? t0 : t1;
      const int u = std::abs(T) - 1;
      const int L = x.dst_hi[t] - x.dst_lo[t];
      const int first = x.src_lo[u], last = x.src_lo[u] + (T > 0 ? L - 1 : -(L - 1));
      if (std::min(first, last) < 0 || std::max(first, last) >= sext[st[u]])
        return fail(nullptr, FV_ERR_INVALID_ARG, tag + "src patch outside the src face");
    }
    auto& u = used[x.dst_block][x.dst_face];
    if (u.empty()) u.assign((size_t)dext[dt[0]] * dext[dt[1]], 0);
    for (int b = x.dst_lo[1]; b < x.dst_hi[1]; ++b)
      for (int a = x.dst_lo[0]; a < x.dst_hi[0]; ++a) {
        char& f = u[(size_t)b * dext[dt[0]] + a];
        if (f) return fail(nullptr, FV_ERR_INVALID_ARG, tag + "dst ghost cells already filled by another connection");
        f = 1;
      }
  }
  return FV_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void fv_config_default(fv_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->gamma = 1.4;
  c->eps = 1.0;
  c->kappa = -1.0;
  c->harten = 0.1;
  c->va_delta2 = 1e-12;
  c->limiter = FV_LIM_VANLEER;
  c->fix_all = 0;
  c->dim = 3;
  c->n_stages = 4;
  c->alpha[0] = 0.25;
  c->alpha[1] = 1.0 / 3.0;
  c->alpha[2] = 0.5;
  c->alpha[3] = 1.0;
  c->precision = FV_PREC_FP64;
  c->visc = 0;
  c->mu = 0.0;
  c->prandtl = 0.72;
  c->r_gas = 287.0;
  c->sutherland = 0;
  c->t_ref = 273.15;
  c->s_suth = 110.4;
}

const char* fv_last_error(fv_handle h) {
  if (!h) return g_create_error.c_str();
  return H(h)->err.c_str();
}

int fv_create_blocks(const fv_block_desc* blocks, int nblocks, const fv_connection* conns, int nconn,
                     const fv_config* cfg, fv_handle* out) {
  if (!out) return fail(nullptr, FV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nconn < 0 || (nconn > 0 && !conns)) return fail(nullptr, FV_ERR_INVALID_ARG, "bad connection list");
  int rc = validate(blocks, nblocks, conns, nconn, cfg);
  if (rc) return rc;
  std::unique_ptr<fv_ctx> h(new fv_ctx());
  h->cfg = *cfg;
  h->nblocks = nblocks;
  h->nconn = nconn;
  h->conns.assign(conns, conns + nconn);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) return fail(nullptr, FV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
  // ---- layout ----
  long long qoff = 0, cell_off = 0, foff[3] = {0, 0, 0};
  for (int b = 0; b < nblocks; ++b) {
    const fv_block_desc& d = blocks[b];
    FvBlockDev B;
    std::memset(&B, 0, sizeof(B));
    B.ni = d.ni; B.nj = d.nj; B.nk = d.nk;
    B.pitch = d.ni + 2 * FV_GHOST;
    B.jstride = B.pitch;
    B.kstride = (long long)B.pitch * (d.nj + 2 * FV_GHOST);
    B.plane = B.kstride * (d.nk + 2 * FV_GHOST);
    B.qoff = qoff;
    qoff += 5 * B.plane;
    B.cell_off = cell_off;
    cell_off += (long long)d.ni * d.nj * d.nk;
    B.cartesian = d.nodes == nullptr;
    if (B.cartesian) {
      const double hx = d.h[0], hy = d.h[1], hz = d.h[2];
      for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) B.cart_n[x][y] = x == y ? 1.0 : 0.0;
      B.cart_area[0] = hy * hz; B.cart_area[1] = hx * hz; B.cart_area[2] = hx * hy;
      B.cart_invvol = 1.0 / (hx * hy * hz);
    } else {
      B.face_off[0] = foff[0]; foff[0] += (long long)(d.ni + 1) * d.nj * d.nk;
      B.face_off[1] = foff[1]; foff[1] += (long long)d.ni * (d.nj + 1) * d.nk;
      B.face_off[2] = foff[2]; foff[2] += (long long)d.ni * d.nj * (d.nk + 1);
    }
    h->hb.push_back(B);
  }
  if (cfg->visc) {
    long long po = 0, vo[3] = {0, 0, 0};
    for (auto& B : h->hb) {
      B.pad_off = po;
      po += (long long)(B.ni + 2) * (B.nj + 2) * (B.nk + 2);
      for (int d = 0; d < 3; ++d) {
        B.vface_off[d] = vo[d];
        vo[d] += (long long)(B.ni + (d == 0)) * (B.nj + (d == 1)) * (B.nk + (d == 2));
      }
    }
    h->pad_total = po;
    for (int d = 0; d < 3; ++d) h->nvfaces[d] = vo[d];
  }
  h->state_elems = qoff;
  h->ext_state_elems = 0;
  for (auto& B : h->hb) h->ext_state_elems += 5 * ghosted_cells(B.ni, B.nj, B.nk);
  h->ncell = cell_off;
  for (int d = 0; d < 3; ++d) h->nfaces[d] = foff[d];
  fv_ctx* hp = h.get();
  // ---- allocations ----
  for (int x = 0; x < 3; ++x) CK(hp, cudaMalloc(&h->buf[x], sizeof(double) * h->state_elems));
  CK(hp, cudaMalloc(&h->d_blocks, sizeof(FvBlockDev) * nblocks));
  CK(hp, cudaMalloc(&h->d_tile_counter, 2 * sizeof(int)));
  CK(hp, cudaMemset(h->d_tile_counter, 0, 2 * sizeof(int)));
  CK(hp, cudaMalloc(&h->invvol, sizeof(double) * h->ncell));
  CK(hp, cudaMalloc(&h->vol, sizeof(double) * h->ncell));
  const int mb = storage_bytes(cfg->precision);
  for (int d = 0; d < 3; ++d)
    if (h->nfaces[d]) CK(hp, cudaMalloc(&h->metric[d], (size_t)mb * 4 * h->nfaces[d]));
  if (cfg->visc) {
    CK(hp, cudaMalloc(&h->geo, sizeof(double) * 10 * h->pad_total));
    CK(hp, cudaMemset(h->geo, 0, sizeof(double) * 10 * h->pad_total));
    if (cfg->precision != FV_PREC_FP32FLUX) {
      for (int d = 0; d < cfg->dim; ++d) {
        CK(hp, cudaMalloc(&h->fvis[d], (size_t)mb * 4 * h->nvfaces[d]));
        CK(hp, cudaMalloc(&h->fgeo[d], (size_t)mb * 12 * h->nvfaces[d]));
      }
    }
  }
  // ---- metrics ----
  double* d_nodes = nullptr;
  for (int b = 0; b < nblocks; ++b) {
    const FvBlockDev& B = h->hb[b];
    const long long nc = (long long)B.ni * B.nj * B.nk;
    if (B.cartesian) {
      fill_kernel<<<grid_for(nc, 256, h->nsm), 256>>>(h->invvol + B.cell_off, nc, B.cart_invvol);
      fill_kernel<<<grid_for(nc, 256, h->nsm), 256>>>(h->vol + B.cell_off, nc, 1.0 / B.cart_invvol);
      if (cfg->visc) geo_cart_kernel<<<grid_for(nc, 256, h->nsm), 256>>>(B, h->pad_total, h->geo);
      continue;
    }
    const long long nn = 3LL * (B.ni + 1) * (B.nj + 1) * (B.nk + 1);
    if (d_nodes) cudaFree(d_nodes);
    CK(hp, cudaMalloc(&d_nodes, sizeof(double) * nn));
    CK(hp, cudaMemcpy(d_nodes, blocks[b].nodes, sizeof(double) * nn, cudaMemcpyHostToDevice));
    for (int dir = 0; dir < 3; ++dir) {
      const long long nf = (long long)(B.ni + (dir == 0)) * (B.nj + (dir == 1)) * (B.nk + (dir == 2));
      const int g = grid_for(nf, 256, h->nsm);
      if (cfg->precision == FV_PREC_FP64)
        metrics_faces_kernel<<<g, 256>>>(d_nodes, B.ni, B.nj, B.nk, dir, (double*)h->metric[dir], B.face_off[dir], h->nfaces[dir]);
      else if (cfg->precision == FV_PREC_DF64)
        metrics_faces_kernel<<<g, 256>>>(d_nodes, B.ni, B.nj, B.nk, dir, (float2*)h->metric[dir], B.face_off[dir], h->nfaces[dir]);
      else
        metrics_faces_kernel<<<g, 256>>>(d_nodes, B.ni, B.nj, B.nk, dir, (float*)h->metric[dir], B.face_off[dir], h->nfaces[dir]);
    }
    volume_kernel<<<grid_for(nc, 256, h->nsm), 256>>>(d_nodes, B.ni, B.nj, B.nk, h->vol + B.cell_off, h->invvol + B.cell_off);
    if (cfg->visc)
      geo_cells_kernel<<<grid_for(nc, 256, h->nsm), 256>>>(d_nodes, B.ni, B.nj, B.nk, h->vol + B.cell_off, B.pad_off,
                                                           h->pad_total, h->geo);
    CK(hp, cudaDeviceSynchronize());
  }
  if (d_nodes) cudaFree(d_nodes);
  CK(hp, cudaGetLastError());
  CK(hp, cudaMemcpy(h->d_blocks, h->hb.data(), sizeof(FvBlockDev) * nblocks, cudaMemcpyHostToDevice));
  // ---- connections ----
  if (nconn) {
    std::vector<FvConnDev> cd(nconn);
    long long items = 0;
    for (int c = 0; c < nconn; ++c) {
      const fv_connection& x = conns[c];
      FvConnDev& y = cd[c];
      y.dst_block = x.dst_block; y.dst_face = x.dst_face;
      y.dlo0 = x.dst_lo[0]; y.dlo1 = x.dst_lo[1];
      y.L0 = x.dst_hi[0] - x.dst_lo[0]; y.L1 = x.dst_hi[1] - x.dst_lo[1];
      y.src_block = x.src_block; y.src_face = x.src_face;
      y.slo0 = x.src_lo[0]; y.slo1 = x.src_lo[1];
      y.t0 = x.transform[0]; y.t1 = x.transform[1];
      y.item_off = items;
      items += 2LL * y.L0 * y.L1;
    }
    h->conn_items = items;
    h->hconns = cd;
    CK(hp, cudaMalloc(&h->d_conns, sizeof(FvConnDev) * nconn));
    CK(hp, cudaMemcpy(h->d_conns, cd.data(), sizeof(FvConnDev) * nconn, cudaMemcpyHostToDevice));
    const std::vector<FvXchTile> xt = xch_tiles(cd);
    h->nxtiles = (int)xt.size();
    CK(hp, cudaMalloc(&h->d_xtiles, sizeof(FvXchTile) * xt.size()));
    CK(hp, cudaMemcpy(h->d_xtiles, xt.data(), sizeof(FvXchTile) * xt.size(), cudaMemcpyHostToDevice));
  }
  // ---- viscous-term tables ----
  if (cfg->visc) {
    CK(hp, cudaDeviceSynchronize());
    rc = build_visc_tables(hp);
    if (rc) { g_create_error = h->err; fv_destroy(reinterpret_cast<fv_handle>(h.release())); return rc; }
    {
      const long long P = h->pad_total;
      if (cfg->precision == FV_PREC_FP32FLUX) {
        CK(hp, cudaMalloc(&h->geo_t, (size_t)mb * 12 * P));
        geo_records_kernel<<<grid_for(P, 256, h->nsm), 256>>>(h->geo, (float*)h->geo_t, P);
      } else {
        for (int d = 0; d < cfg->dim; ++d)
          for (const FvBlockDev& B : h->hb) {
            const long long nf = (long long)(B.ni + (d == 0)) * (B.nj + (d == 1)) * (B.nk + (d == 2));
            const int g = grid_for(nf, 256, h->nsm);
            if (cfg->precision == FV_PREC_FP64)
              face_geometry_kernel<<<g, 256>>>(B, d, h->geo, P, (const double*)h->metric[d], (double*)h->fgeo[d]);
            else
              face_geometry_kernel<<<g, 256>>>(B, d, h->geo, P, (const float2*)h->metric[d], (float2*)h->fgeo[d]);
          }
        // the viscous face kernel's work units: 32 x 8 face positions
        // (i = 0..ni, j = 0..nj) of a block, FV_VISC_KC positions along k
        // (k = 0..nk; one plane in 2D)
        std::vector<FvViscTile> vt;
        for (int b = 0; b < nblocks; ++b) {
          const FvBlockDev& B = h->hb[b];
          const int kpos = cfg->dim == 3 ? B.nk + 1 : 1;
          for (int k0 = 0; k0 < kpos; k0 += FV_VISC_KC)
            for (int j0 = 0; j0 <= B.nj; j0 += FV_VISC_TY)
              for (int i0 = 0; i0 <= B.ni; i0 += FV_VISC_TX) vt.push_back(FvViscTile{b, i0, j0, k0});
        }
        h->nvtiles = (int)vt.size();
        CK(hp, cudaMalloc(&h->d_vtiles, sizeof(FvViscTile) * vt.size()));
        CK(hp, cudaMemcpy(h->d_vtiles, vt.data(), sizeof(FvViscTile) * vt.size(), cudaMemcpyHostToDevice));
      }
      CK(hp, cudaDeviceSynchronize());
      cudaFree(h->geo);
      h->geo = nullptr;
    }
  }
  // ---- tiles ----
  choose_launch(hp);
  rc = build_tiles(hp);
  if (rc) { g_create_error = h->err; fv_destroy(reinterpret_cast<fv_handle>(h.release())); return rc; }
  CK(hp, cudaDeviceSynchronize());
  *out = reinterpret_cast<fv_handle>(h.release());
  return FV_OK;
}

int fv_destroy(fv_handle hh) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  cudaDeviceSynchronize();
  drop_graphs(h);
  for (int x = 0; x < 3; ++x) cudaFree(h->buf[x]);
  for (int d = 0; d < 3; ++d) cudaFree(h->metric[d]);
  cudaFree(h->d_blocks); cudaFree(h->d_tiles); cudaFree(h->d_conns); cudaFree(h->d_tile_counter);
  cudaFree(h->invvol); cudaFree(h->vol); cudaFree(h->srcvol); cudaFree(h->srcvol2);
  cudaFree(h->scratch_r); cudaFree(h->partials); cudaFree(h->d_norm); cudaFree(h->stage_buf);
  cudaFree(h->adj_contrib); cudaFree(h->adj_lamg); cudaFree(h->adj_qx);
  cudaFree(h->d_bcs); cudaFree(h->d_bcmap);
  cudaFree(h->d_hsend); cudaFree(h->d_hrecv); cudaFree(h->d_hstiles); cudaFree(h->d_hrtiles); cudaFree(h->d_xtiles);
  cudaFree(h->geo_t);
  cudaFree(h->geo); cudaFree(h->d_vtiles); cudaFree(h->d_edges);
  cudaFree(h->rmon); cudaFree(h->mon_partials); cudaFree(h->mon_norm);
  for (int d = 0; d < 3; ++d) { cudaFree(h->fvis[d]); cudaFree(h->fgeo[d]); }
  delete h;
  return FV_OK;
}

int64_t fv_state_size(fv_handle h) { return h ? H(h)->ext_state_elems : -1; }
int64_t fv_field_size(fv_handle h) { return h ? 5 * H(h)->ncell : -1; }
int64_t fv_cell_count(fv_handle h) { return h ? H(h)->ncell : -1; }

int fv_set_state(fv_handle hh, const double* q, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (!q) return fail(h, FV_ERR_INVALID_ARG, "q is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = copy_state(h, q, h->buf[0], true, s);
  if (rc) return rc;
  for (int x = 1; x < 3; ++x)
    CK(h, cudaMemcpyAsync(h->buf[x], h->buf[0], sizeof(double) * h->state_elems, cudaMemcpyDeviceToDevice, s));
  return FV_OK;
}

int fv_stage_state(fv_handle hh, const double* q, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (!q) return fail(h, FV_ERR_INVALID_ARG, "q is NULL");
  if (!h->stage_buf) CK(h, cudaMalloc(&h->stage_buf, sizeof(double) * h->ext_state_elems));
  CK(h, cudaMemcpyAsync(h->stage_buf, q, sizeof(double) * h->ext_state_elems, cudaMemcpyDefault,
                        (cudaStream_t)stream));
  h->staged = true;
  return FV_OK;
}

int fv_set_state_staged(fv_handle hh, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (!h->staged) return fail(h, FV_ERR_INVALID_ARG, "no state has been staged");
  return fv_set_state(hh, h->stage_buf, stream);
}

int fv_set_buffer(fv_handle hh, int buffer, const double* q, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (!q) return fail(h, FV_ERR_INVALID_ARG, "q is NULL");
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  return copy_state(h, q, h->buf[buffer], true, (cudaStream_t)stream);
}

int fv_get_state(fv_handle hh, int buffer, double* q, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (!q) return fail(h, FV_ERR_INVALID_ARG, "q is NULL");
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = copy_state(h, h->buf[buffer], q, false, s);
  if (rc) return rc;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, q) == cudaSuccess && at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    CK(h, cudaStreamSynchronize(s));
  return FV_OK;
}

int fv_set_source(fv_handle hh, const double* src, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  cudaStream_t s = (cudaStream_t)stream;
  drop_graphs(h);
  if (!src) {
    if (h->srcvol || h->srcvol2) {
      CK(h, cudaStreamSynchronize(s));
      cudaFree(h->srcvol); h->srcvol = nullptr;
      cudaFree(h->srcvol2); h->srcvol2 = nullptr;
    }
    return FV_OK;
  }
  if (!h->srcvol) CK(h, cudaMalloc(&h->srcvol, sizeof(double) * 5 * h->ncell));
  CK(h, cudaMemcpyAsync(h->srcvol, src, sizeof(double) * 5 * h->ncell, cudaMemcpyDefault, s));
  for (auto& B : h->hb) {
    const long long nc = (long long)B.ni * B.nj * B.nk;
    source_scale_kernel<<<grid_for(5 * nc, 256, h->nsm), 256, 0, s>>>(h->srcvol, h->vol, h->srcvol, 5 * B.cell_off, nc,
                                                                    B.cell_off);
  }
  if (h->cfg.precision != FV_PREC_FP64) {
    if (!h->srcvol2) CK(h, cudaMalloc(&h->srcvol2, sizeof(float2) * 5 * h->ncell));
    split_kernel<<<grid_for(5 * h->ncell, 256, h->nsm), 256, 0, s>>>(h->srcvol, h->srcvol2, 5 * h->ncell);
  }
  CK(h, cudaGetLastError());
  return FV_OK;
}

int fv_set_boundaries(fv_handle hh, const fv_bc_patch* patches, int n) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (n < 0 || (n > 0 && !patches)) return fail(h, FV_ERR_INVALID_ARG, "bad boundary patch list");
  std::vector<FvBcDev> dev(n);
  std::vector<long long> map_off(h->hb.size(), -1);
  long long map_total = 0, items = 0;
  for (int p = 0; p < n; ++p) {
    const fv_bc_patch& P = patches[p];
    char msg[160];
    if (P.block < 0 || P.block >= h->nblocks) {
      std::snprintf(msg, sizeof(msg), "boundary patch %d: block %d out of range", p, P.block);
      return fail(h, FV_ERR_INVALID_ARG, msg);
    }
    const FvBlockDev& B = h->hb[P.block];
    if (P.face < 0 || P.face > 5 || (h->cfg.dim == 2 && P.face > 3)) {
      std::snprintf(msg, sizeof(msg), "boundary patch %d: face %d not valid for dim %d", p, P.face, h->cfg.dim);
      return fail(h, FV_ERR_INVALID_ARG, msg);
    }
    const int ax = P.face / 2;
    const int ext[3] = {B.ni, B.nj, B.nk};
    const int e0 = ext[ax == 0 ? 1 : 0], e1 = ext[ax == 2 ? 1 : 2];
    if (P.lo[0] < 0 || P.lo[1] < 0 || P.hi[0] > e0 || P.hi[1] > e1 || P.lo[0] >= P.hi[0] || P.lo[1] >= P.hi[1]) {
      std::snprintf(msg, sizeof(msg), "boundary patch %d: range [%d,%d)x[%d,%d) outside the %dx%d face", p, P.lo[0],
                    P.hi[0], P.lo[1], P.hi[1], e0, e1);
      return fail(h, FV_ERR_INVALID_ARG, msg);
    }
    if (P.kind < FV_BC_FIXED || P.kind > FV_BC_NOSLIP_WALL) {
      std::snprintf(msg, sizeof(msg), "boundary patch %d: unknown kind %d", p, P.kind);
      return fail(h, FV_ERR_INVALID_ARG, msg);
    }
    if (P.kind == FV_BC_SUPERSONIC_INFLOW || P.kind == FV_BC_FARFIELD) {
      bool ok = P.state[0] > 0.0 && P.state[4] > 0.0;
      for (int v = 0; v < 5; ++v) ok = ok && std::isfinite(P.state[v]);
      if (!ok) {
        std::snprintf(msg, sizeof(msg), "boundary patch %d: state needs finite values, rho > 0 and p > 0", p);
        return fail(h, FV_ERR_INVALID_ARG, msg);
      }
    }
    if ((P.kind == FV_BC_SLIP_WALL || P.kind == FV_BC_NOSLIP_WALL) && ext[ax] < 2) {
      std::snprintf(msg, sizeof(msg), "boundary patch %d: a slip wall needs two cells along the face normal", p);
      return fail(h, FV_ERR_INVALID_ARG, msg);
    }
    FvBcDev& D = dev[p];
    std::memset(&D, 0, sizeof(D));
    D.block = P.block; D.face = P.face; D.lo0 = P.lo[0]; D.lo1 = P.lo[1];
    D.L0 = P.hi[0] - P.lo[0]; D.L1 = P.hi[1] - P.lo[1]; D.kind = P.kind;
    D.item_off = items;
    for (int v = 0; v < 5; ++v) D.state[v] = P.state[v];
    if (P.kind == FV_BC_SUPERSONIC_INFLOW || P.kind == FV_BC_FARFIELD) {
      const double g = h->cfg.gamma, r = P.state[0];
      D.qstate[0] = r;
      for (int v = 1; v < 4; ++v) D.qstate[v] = r * P.state[v];
      D.qstate[4] = P.state[4] / (g - 1.0) +
                    0.5 * r * (P.state[1] * P.state[1] + P.state[2] * P.state[2] + P.state[3] * P.state[3]);
      D.cstate = std::sqrt(g * P.state[4] / r);
    }
    items += (long long)D.L0 * D.L1;
    if ((P.kind == FV_BC_SLIP_WALL || P.kind == FV_BC_FARFIELD || P.kind == FV_BC_NOSLIP_WALL) &&
        map_off[P.block] < 0) {
      map_off[P.block] = map_total;
      map_total += 2LL * ((long long)B.nj * B.nk + (long long)B.ni * B.nk + (long long)B.ni * B.nj);
    }
  }
  // face maps: every patch writes its kind over its range, in order
  std::vector<signed char> maps(map_total, 0);
  for (int p = 0; p < n; ++p) {
    const fv_bc_patch& P = patches[p];
    if (map_off[P.block] < 0) continue;
    const FvBlockDev& B = h->hb[P.block];
    const long long sz[6] = {(long long)B.nj * B.nk, (long long)B.nj * B.nk, (long long)B.ni * B.nk,
                             (long long)B.ni * B.nk, (long long)B.ni * B.nj, (long long)B.ni * B.nj};
    long long base = map_off[P.block];
    for (int f = 0; f < P.face; ++f) base += sz[f];
    const int ext0 = P.face < 2 ? B.nj : B.ni;
    const signed char code =
        (P.kind == FV_BC_SLIP_WALL || P.kind == FV_BC_FARFIELD || P.kind == FV_BC_NOSLIP_WALL) ? (signed char)P.kind : 0;
    for (int t1 = P.lo[1]; t1 < P.hi[1]; ++t1)
      for (int t0 = P.lo[0]; t0 < P.hi[0]; ++t0) maps[base + (long long)t1 * ext0 + t0] = code;
  }
  CK(h, cudaDeviceSynchronize());
  // drop the old set first (a failed allocation below leaves no boundaries)
  drop_graphs(h);
  h->nbc = 0;
  h->bc_items = 0;
  h->bcs.clear();
  for (auto& B : h->hb) B.bcmap = nullptr;
  CK(h, cudaMemcpy(h->d_blocks, h->hb.data(), sizeof(FvBlockDev) * h->hb.size(), cudaMemcpyHostToDevice));
  cudaFree(h->d_bcs); h->d_bcs = nullptr;
  cudaFree(h->d_bcmap); h->d_bcmap = nullptr;
  if (n) {
    CK(h, cudaMalloc(&h->d_bcs, sizeof(FvBcDev) * n));
    CK(h, cudaMemcpy(h->d_bcs, dev.data(), sizeof(FvBcDev) * n, cudaMemcpyHostToDevice));
  }
  if (map_total) {
    CK(h, cudaMalloc(&h->d_bcmap, map_total));
    CK(h, cudaMemcpy(h->d_bcmap, maps.data(), map_total, cudaMemcpyHostToDevice));
  }
  for (size_t b = 0; b < h->hb.size(); ++b) h->hb[b].bcmap = map_off[b] < 0 ? nullptr : h->d_bcmap + map_off[b];
  CK(h, cudaMemcpy(h->d_blocks, h->hb.data(), sizeof(FvBlockDev) * h->hb.size(), cudaMemcpyHostToDevice));
  h->bcs.assign(patches, patches + n);
  h->nbc = n;
  h->bc_items = items;
  // the stage kernel variant with (or without) the boundary overwrites, and
  // its occupancy and tile table
  choose_launch(h);
  return build_tiles(h);
}

int fv_exchange_ghosts(fv_handle hh, int buffer, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  return do_exchange(h, h->buf[buffer], (cudaStream_t)stream);
}

int fv_residual(fv_handle hh, int buffer, double* r_dev, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  if (!r_dev) return fail(h, FV_ERR_INVALID_ARG, "r_dev is NULL");
  FvStageArgs a = base_args(h);
  a.mode = FV_MODE_RESIDUAL;
  a.qin = h->buf[buffer];
  a.rout = r_dev;
  a.rout_varmajor = 0;
  return launch_stage(h, a, (cudaStream_t)stream);
}

int fv_rk_stage(fv_handle hh, int stage, double dt, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (stage < 1 || stage > h->cfg.n_stages) return fail(h, FV_ERR_INVALID_ARG, "stage out of range");
  return do_stage(h, stage, dt, (cudaStream_t)stream);
}

int fv_rk_step(fv_handle hh, double dt, int use_graph, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) {
    for (int m = 1; m <= h->cfg.n_stages; ++m) {
      int rc = do_stage(h, m, dt, s);
      if (rc) return rc;
    }
    return FV_OK;
  }
  auto it = h->graphs.find(s);
  if (it == h->graphs.end()) {
    if ((int)h->graphs.size() >= FV_MAX_GRAPHS) {
      // evict the least recently used stream's graph; the device is idle
      // first, so neither it nor its dt slot is in use
      auto lru = h->graphs.begin();
      for (auto g = h->graphs.begin(); g != h->graphs.end(); ++g)
        if (g->second.used < lru->second.used) lru = g;
      CK(h, cudaDeviceSynchronize());
      cudaGraphExecDestroy(lru->second.exec);
      cudaFree(lru->second.dt_dev);
      h->graphs.erase(lru);
    }
    fv_ctx::StepGraph sg;
    CK(h, cudaMalloc(&sg.dt_dev, sizeof(double)));
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaFree(sg.dt_dev); return cuda_fail(h, e, "cudaStreamCreateWithFlags"); }
    cudaGraph_t g;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); cudaFree(sg.dt_dev); return cuda_fail(h, e, "cudaStreamBeginCapture"); }
    int rc = FV_OK;
    for (int m = 1; m <= h->cfg.n_stages && rc == FV_OK; ++m) rc = do_stage(h, m, dt, cs, sg.dt_dev);
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc || e != cudaSuccess) {
      cudaFree(sg.dt_dev);
      return rc ? rc : cuda_fail(h, e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&sg.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { cudaFree(sg.dt_dev); return cuda_fail(h, e, "cudaGraphInstantiate"); }
    // dt differs from any value the slot holds: written below
    sg.dt = std::nan("");
    it = h->graphs.emplace(s, sg).first;
  }
  fv_ctx::StepGraph& sg = it->second;
  if (!(sg.dt == dt)) {
    set_scalar_kernel<<<1, 1, 0, s>>>(sg.dt_dev, dt);
    CK(h, cudaGetLastError());
    sg.dt = dt;
  }
  sg.used = ++h->graph_clock;
  CK(h, cudaGraphLaunch(sg.exec, s));
  return FV_OK;
}

int fv_residual_norms(fv_handle hh, int buffer, double* out_host, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  if (!out_host) return fail(h, FV_ERR_INVALID_ARG, "out_host is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int nparts = FV_NORM_PARTS * h->nsm;
  if (!h->scratch_r) CK(h, cudaMalloc(&h->scratch_r, sizeof(double) * 5 * h->ncell));
  if (!h->partials) CK(h, cudaMalloc(&h->partials, sizeof(double) * 15 * nparts));
  if (!h->d_norm) CK(h, cudaMalloc(&h->d_norm, sizeof(double) * 16));
  int rc = do_exchange(h, h->buf[buffer], s);
  if (rc) return rc;
  FvStageArgs a = base_args(h);
  a.mode = FV_MODE_RESIDUAL;
  a.qin = h->buf[buffer];
  a.rout = h->scratch_r;
  a.rout_varmajor = 1;
  rc = launch_stage(h, a, s);
  if (rc) return rc;
  if (fv_monitor_reduce(h->scratch_r, 1, h->ncell, h->partials, nparts, h->d_norm, s))
    return cuda_fail(h, cudaGetLastError(), "residual norm reduction");
  double tmp[15];
  CK(h, cudaMemcpyAsync(tmp, h->d_norm, sizeof(double) * 15, cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  std::memcpy(out_host, tmp, sizeof(double) * 10);
  for (int v = 0; v < 5; ++v)
    if (tmp[10 + v] != 0.0) return fail(h, FV_ERR_NONFINITE, "residual has non-finite entries");
  return FV_OK;
}

int fv_set_monitor(fv_handle hh, int on) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  CK(h, cudaDeviceSynchronize());
  if (on && !h->rmon) {
    const size_t eb = h->cfg.precision == FV_PREC_FP64 ? sizeof(double) : sizeof(float2);
    CK(h, cudaMalloc(&h->rmon, eb * 5 * h->ncell));
    CK(h, cudaMalloc(&h->mon_partials, sizeof(double) * 15 * FV_NORM_PARTS * h->nsm));
    CK(h, cudaMalloc(&h->mon_norm, sizeof(double) * 16));
  }
  h->monitor = on ? 1 : 0;
  h->mon_ran = false;
  drop_graphs(h);
  return FV_OK;
}

int fv_monitor_norms(fv_handle hh, double* out_host, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (!out_host) return fail(h, FV_ERR_INVALID_ARG, "out_host is NULL");
  if (!h->monitor || !h->mon_ran) return fail(h, FV_ERR_INVALID_ARG, "no monitored RK stage 1 has run");
  cudaStream_t s = (cudaStream_t)stream;
  double tmp[15];
  CK(h, cudaMemcpyAsync(tmp, h->mon_norm, sizeof(double) * 15, cudaMemcpyDeviceToHost, s));
  CK(h, cudaStreamSynchronize(s));
  std::memcpy(out_host, tmp, sizeof(double) * 10);
  for (int v = 0; v < 5; ++v)
    if (tmp[10 + v] != 0.0) return fail(h, FV_ERR_NONFINITE, "residual has non-finite entries");
  return FV_OK;
}

int fv_autotune(fv_handle hh, double dt, int reps, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  cudaStream_t s = (cudaStream_t)stream;
  if (reps <= 0) reps = 3;
  CK(h, cudaStreamSynchronize(s));
  cudaEvent_t e0, e1;
  CK(h, cudaEventCreate(&e0));
  CK(h, cudaEventCreate(&e1));
  const int kcs[] = {0, -1, -2, 4, 8, 16, 32};
  float best = 1e30f;
  int best_tile = 1, best_kc = 0;
  const fv_config saved = h->cfg;
  for (int tile = 1; tile <= FV_NUM_SHAPES; ++tile) {
    for (int kc : kcs) {
      if (h->cfg.dim == 2 && kc != 0) continue;
      h->cfg.tile = tile;
      h->cfg.kchunk = kc;
      choose_launch(h);
      if (build_tiles(h) != FV_OK) continue;
      int rc = do_stage(h, 1, dt, s);
      if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); h->cfg = saved; return rc; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) do_stage(h, 1, dt, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_tile = tile; best_kc = kc; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->cfg.tile = best_tile;
  h->cfg.kchunk = best_kc;
  choose_launch(h);
  int rc = build_tiles(h);
  drop_graphs(h);
  CK(h, cudaGetLastError());
  return rc;
}

int fv_set_halo(fv_handle hh, const fv_connection* send, int nsend, const fv_connection* recv, int nrecv) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (nsend < 0 || nrecv < 0 || (nsend && !send) || (nrecv && !recv))
    return fail(h, FV_ERR_INVALID_ARG, "halo: negative count or NULL table");
  const int nb = (int)h->hb.size();
  auto ext = [&](int blk, int axis) { const FvBlockDev& B = h->hb[blk]; return axis == 0 ? B.ni : (axis == 1 ? B.nj : B.nk); };
  // ghost cells already written by this device's own connections
  std::vector<std::vector<std::vector<char>>> used(nb, std::vector<std::vector<char>>(6));
  auto mark = [&](const fv_connection& x, const std::string& tag) -> int {
    const int da = x.dst_face / 2;
    const int t0 = da == 0 ? 1 : 0, t1 = da == 2 ? 1 : 2;
    auto& u = used[x.dst_block][x.dst_face];
    if (u.empty()) u.assign((size_t)ext(x.dst_block, t0) * ext(x.dst_block, t1), 0);
    for (int b = x.dst_lo[1]; b < x.dst_hi[1]; ++b)
      for (int a = x.dst_lo[0]; a < x.dst_hi[0]; ++a) {
        char& f = u[(size_t)b * ext(x.dst_block, t0) + a];
        if (f) return fail(h, FV_ERR_INVALID_ARG, tag + "dst ghost cells already filled by another connection");
        f = 1;
      }
    return FV_OK;
  };
  for (const fv_connection& x : h->conns) mark(x, "");
  const int maxface = h->cfg.dim == 2 ? 3 : 5;
  for (int side = 0; side < 2; ++side) {
    const fv_connection* tab = side ? recv : send;
    const int n = side ? nrecv : nsend;
    for (int c = 0; c < n; ++c) {
      const fv_connection& x = tab[c];
      const std::string tag = std::string(side ? "halo recv " : "halo send ") + std::to_string(c) + ": ";
      const int L0 = x.dst_hi[0] - x.dst_lo[0], L1 = x.dst_hi[1] - x.dst_lo[1];
      if (L0 <= 0 || L1 <= 0) return fail(h, FV_ERR_INVALID_ARG, tag + "empty patch");
      if (side) {
        if (x.dst_block < 0 || x.dst_block >= nb || x.dst_face < 0 || x.dst_face > maxface)
          return fail(h, FV_ERR_INVALID_ARG, tag + "dst block or face out of range");
        const int da = x.dst_face / 2;
        const int t0 = da == 0 ? 1 : 0, t1 = da == 2 ? 1 : 2;
        if (x.dst_lo[0] < 0 || x.dst_lo[1] < 0 || x.dst_hi[0] > ext(x.dst_block, t0) || x.dst_hi[1] > ext(x.dst_block, t1))
          return fail(h, FV_ERR_INVALID_ARG, tag + "dst patch outside the face");
        int rc = mark(x, tag);
        if (rc) return rc;
      } else {
        if (x.src_block < 0 || x.src_block >= nb || x.src_face < 0 || x.src_face > maxface)
          return fail(h, FV_ERR_INVALID_ARG, tag + "src block or face out of range");
        const int t0 = x.transform[0], t1 = x.transform[1];
        if (!(std::abs(t0) == 1 || std::abs(t0) == 2) || !(std::abs(t1) == 1 || std::abs(t1) == 2) ||
            std::abs(t0) == std::abs(t1))
          return fail(h, FV_ERR_INVALID_ARG, tag + "transform must be a signed permutation of (1,2)");
        const int sa = x.src_face / 2;
        if (ext(x.src_block, sa) < FV_GHOST) return fail(h, FV_ERR_INVALID_ARG, tag + "src block thinner than the ghost depth");
        const int st[2] = {sa == 0 ? 1 : 0, sa == 2 ? 1 : 2};
        for (int t = 0; t < 2; ++t) {
          const int T = t == 0 ? t0 : t1;
          const int u = std::abs(T) - 1;
          const int L = t == 0 ? L0 : L1;
          const int first = x.src_lo[u], last = x.src_lo[u] + (T > 0 ? L - 1 : -(L - 1));
          if (std::min(first, last) < 0 || std::max(first, last) >= ext(x.src_block, st[u]))
            return fail(h, FV_ERR_INVALID_ARG, tag + "src patch outside the src face");
        }
      }
    }
  }
  CK(h, cudaDeviceSynchronize());
  cudaFree(h->d_hsend); cudaFree(h->d_hrecv); cudaFree(h->d_hstiles); cudaFree(h->d_hrtiles);
  h->d_hsend = h->d_hrecv = nullptr;
  h->d_hstiles = h->d_hrtiles = nullptr;
  h->nhsend = h->nhrecv = h->nhstiles = h->nhrtiles = 0;
  h->hsend_items = h->hrecv_items = 0;
  for (int side = 0; side < 2; ++side) {
    const fv_connection* tab = side ? recv : send;
    const int n = side ? nrecv : nsend;
    if (!n) continue;
    std::vector<FvConnDev> cd(n);
    long long items = 0;
    for (int c = 0; c < n; ++c) {
      const fv_connection& x = tab[c];
      FvConnDev& y = cd[c];
      y.dst_block = side ? x.dst_block : -1; y.dst_face = x.dst_face;
      y.dlo0 = x.dst_lo[0]; y.dlo1 = x.dst_lo[1];
      y.L0 = x.dst_hi[0] - x.dst_lo[0]; y.L1 = x.dst_hi[1] - x.dst_lo[1];
      y.src_block = side ? -1 : x.src_block; y.src_face = x.src_face;
      y.slo0 = x.src_lo[0]; y.slo1 = x.src_lo[1];
      y.t0 = x.transform[0]; y.t1 = x.transform[1];
      y.item_off = items;
      items += 2LL * y.L0 * y.L1;
    }
    FvConnDev** dst = side ? &h->d_hrecv : &h->d_hsend;
    CK(h, cudaMalloc(dst, sizeof(FvConnDev) * n));
    CK(h, cudaMemcpy(*dst, cd.data(), sizeof(FvConnDev) * n, cudaMemcpyHostToDevice));
    (side ? h->nhrecv : h->nhsend) = n;
    (side ? h->hrecv_items : h->hsend_items) = items;
    const std::vector<FvXchTile> xt = xch_tiles(cd);
    FvXchTile** tdst = side ? &h->d_hrtiles : &h->d_hstiles;
    CK(h, cudaMalloc(tdst, sizeof(FvXchTile) * xt.size()));
    CK(h, cudaMemcpy(*tdst, xt.data(), sizeof(FvXchTile) * xt.size(), cudaMemcpyHostToDevice));
    (side ? h->nhrtiles : h->nhstiles) = (int)xt.size();
  }
  return FV_OK;
}

int64_t fv_halo_size(fv_handle hh, int recv) {
  if (!hh) return -1;
  const fv_ctx* h = H(hh);
  return 5 * (recv ? h->hrecv_items : h->hsend_items);
}

int fv_halo_pack(fv_handle hh, int buffer, double* send_dev, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  if (!h->hsend_items) return FV_OK;
  if (!send_dev) return fail(h, FV_ERR_INVALID_ARG, "send_dev is NULL");
  exchange_kernel<XCH_PACK><<<h->nhstiles, 256, 0, (cudaStream_t)stream>>>(h->d_blocks, h->d_hsend, h->d_hstiles,
                                                                             h->buf[buffer], send_dev);
  CK(h, cudaGetLastError());
  return FV_OK;
}

int fv_halo_unpack(fv_handle hh, int buffer, const double* recv_dev, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (buffer < 0 || buffer > 2) return fail(h, FV_ERR_INVALID_ARG, "buffer must be 0, 1 or 2");
  if (!h->hrecv_items) return FV_OK;
  if (!recv_dev) return fail(h, FV_ERR_INVALID_ARG, "recv_dev is NULL");
  exchange_kernel<XCH_UNPACK><<<h->nhrtiles, 256, 0, (cudaStream_t)stream>>>(
      h->d_blocks, h->d_hrecv, h->d_hrtiles, h->buf[buffer], const_cast<double*>(recv_dev));
  CK(h, cudaGetLastError());
  return FV_OK;
}

int fv_graph_count(fv_handle hh) {
  if (!hh) return -1;
  return (int)H(hh)->graphs.size();
}

int fv_get_launch(fv_handle hh, int* out4) {
  if (!hh || !out4) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  out4[0] = h->cfg.tile <= 0 ? 0 : h->cfg.tile;
  out4[1] = h->cfg.kchunk;
  out4[2] = h->ntiles;
  out4[3] = h->launch.grid;
  return FV_OK;
}

int fv_set_adjoint_arith(fv_handle hh, int precision) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (precision != FV_PREC_FP64 && precision != FV_PREC_DF64)
    return fail(h, FV_ERR_INVALID_ARG, "adjoint arithmetic must be FV_PREC_FP64 or FV_PREC_DF64");
  h->adj_df64 = precision == FV_PREC_DF64;
  return FV_OK;
}

int fv_adjoint_vjp(fv_handle hh, int stage, double dt, const double* qin_dev, const double* lam_out_dev,
                   double* lam_in_dev, double* lam_q0_dev, void* stream) {
  if (!hh) return FV_ERR_INVALID_ARG;
  fv_ctx* h = H(hh);
  if (stage < 1 || stage > h->cfg.n_stages) return fail(h, FV_ERR_INVALID_ARG, "stage out of range");
  if (!qin_dev || !lam_out_dev || !lam_in_dev || !lam_q0_dev) return fail(h, FV_ERR_INVALID_ARG, "NULL pointer");
  if (h->cfg.precision != FV_PREC_FP64)
    return fail(h, FV_ERR_UNSUPPORTED, "the adjoint runs in binary64: create the handle with FV_PREC_FP64");
  if (h->cfg.flux != FV_FLUX_ROE) return fail(h, FV_ERR_UNSUPPORTED, "the adjoint is built for the Roe flux");
  if (h->nbc) return fail(h, FV_ERR_UNSUPPORTED, "the adjoint does not linearise physical boundary patches");
  if (h->cfg.visc) return fail(h, FV_ERR_UNSUPPORTED, "the adjoint is built for the inviscid residual");
  cudaStream_t s = (cudaStream_t)stream;
  const int nd = h->cfg.dim;
  // per-direction offsets of each block's faces in the contribution scratch
  std::vector<long long> coff(3 * h->hb.size());
  long long tot[3] = {0, 0, 0};
  for (size_t b = 0; b < h->hb.size(); ++b) {
    const FvBlockDev& B = h->hb[b];
    for (int d = 0; d < 3; ++d) {
      coff[3 * b + d] = tot[d];
      if (d < nd) tot[d] += (long long)(B.ni + (d == 0)) * (B.nj + (d == 1)) * (B.nk + (d == 2));
    }
  }
  const long long nfaces_all = tot[0] + tot[1] + tot[2];
  if (!h->adj_contrib) CK(h, cudaMalloc(&h->adj_contrib, sizeof(double) * 20 * nfaces_all));
  if (!h->adj_lamg) CK(h, cudaMalloc(&h->adj_lamg, sizeof(double) * h->state_elems));
  double* cdir[3] = {h->adj_contrib, h->adj_contrib + 20 * tot[0], h->adj_contrib + 20 * (tot[0] + tot[1])};
  // linearise around the state the forward stage saw: X(Q^(m-1)), ghosts exchanged
  const double* qx = qin_dev;
  if (h->conn_items || h->bc_items) {
    if (!h->adj_qx) CK(h, cudaMalloc(&h->adj_qx, sizeof(double) * h->state_elems));
    int rc = copy_state(h, qin_dev, h->adj_qx, true, s);
    if (rc) return rc;
    rc = do_exchange(h, h->adj_qx, s);
    if (rc) return rc;
    qx = h->adj_qx;
  }
  const double alpha_dt = h->cfg.alpha[stage - 1] * dt;
  const FvStageArgs a = base_args(h);
  for (size_t b = 0; b < h->hb.size(); ++b) {
    const FvBlockDev& B = h->hb[b];
    for (int d = 0; d < nd; ++d)
      if (fv_adjoint_faces(B, d, qx, lam_out_dev, h->invvol, alpha_dt, (const double*)h->metric[d], h->nfaces[d],
                           a.fp, h->adj_df64, cdir[d] + 20 * coff[3 * b + d], s))
        return cuda_fail(h, cudaGetLastError(), "adjoint face kernel");
  }
  for (size_t b = 0; b < h->hb.size(); ++b) {
    const FvBlockDev& B = h->hb[b];
    if (fv_adjoint_gather(B, cdir[0] + 20 * coff[3 * b], cdir[1] + 20 * coff[3 * b + 1],
                          nd == 3 ? cdir[2] + 20 * coff[3 * b + 2] : nullptr, nd == 3, h->adj_lamg, s))
      return cuda_fail(h, cudaGetLastError(), "adjoint gather kernel");
  }
  for (const FvConnDev& c : h->hconns)
    if (fv_adjoint_transpose(h->d_blocks, c, h->adj_lamg, s)) return cuda_fail(h, cudaGetLastError(), "adjoint transpose");
  for (const FvBlockDev& B : h->hb)
    if (fv_adjoint_finish(B, h->adj_lamg, lam_out_dev, lam_in_dev, lam_q0_dev, s))
      return cuda_fail(h, cudaGetLastError(), "adjoint finish kernel");
  return FV_OK;
}

}  // extern "C"
