"""CPU oracle for the multi-block Euler residual and RK stage.

TEST INFRASTRUCTURE ONLY: the plain, slow restatement of the method that the
CUDA library is checked against.  Only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does.

The arithmetic lives in ``fv_oracle.cpp`` (plain loops, double / dual-number /
op-counting instantiations, built with ``-ffp-contract=off``); this module
builds it, computes metrics through it and sequences the Runge-Kutta stages.
Citations per routine are in the C++ file (paper Section 2 and Eq. (flux)).

Parity pins (see tests/test_oracle_*.py): flux consistency, supersonic
upwinding (which fixes the Roe decomposition), stationary contact, mirror
symmetry, limiter identities, MUSCL reductions, free-stream preservation on a
perturbed grid, discrete conservation on periodic domains, RK amplification
polynomial, second-order truncation error under a manufactured solution,
split-vs-unsplit multi-block equivalence and dual-number JVP vs central
differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Callable, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_metrics.argtypes = [ctypes.c_int] * 3 + [_dp] * 6
        L.oracle_exchange.argtypes = [ctypes.c_int, _ip, _ip, _lp, _dp]
        L.oracle_residual.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [_dp] * 7
        L.oracle_residual_jvp.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [_dp] * 9
        L.oracle_rk_update.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] + [_dp] * 4
        L.oracle_roe_flux.argtypes = [_dp] * 5
        L.oracle_face_flux.argtypes = [_dp] * 5
        L.oracle_muscl.argtypes = [_dp] * 3
        L.oracle_limited.argtypes = [_dp, ctypes.c_double, ctypes.c_double]
        L.oracle_limited.restype = ctypes.c_double
        L.oracle_cons_to_prim.argtypes = [ctypes.c_double, _dp, _dp]
        L.oracle_face_opcount.argtypes = [_dp, _dp, _dp, _lp]
        L.oracle_residual_bc.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [_dp] * 6 + [
            ctypes.c_char_p, _dp]
        L.oracle_bc_fill.argtypes = [_dp] + [ctypes.c_int] * 3 + [_dp] * 3 + [ctypes.c_int] * 6 + [_dp, _dp]
        L.oracle_farfield_state.argtypes = [ctypes.c_double] + [_dp] * 4
        L.oracle_wall_flux.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.oracle_edge_fill.argtypes = [ctypes.c_int, _ip, _ip, _lp, ctypes.c_int, ctypes.c_int, _dp]
        L.oracle_residual_ns.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [_dp] * 7 + [
            ctypes.c_char_p, _dp]
        L.oracle_viscous_face.argtypes = [_dp, _dp, _dp, ctypes.c_int, _dp, _dp]
        L.oracle_viscous_opcount.argtypes = [_dp, _lp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_ip)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_lp)
    raise TypeError(a.dtype)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def params_array(params: dict, dim: int) -> np.ndarray:
    return np.array([params["gamma"], params["eps"], params["kappa"], params["limiter"],
                     params["harten"], params["fix_all"], params["va_delta2"], dim,
                     params.get("flux", 0), params.get("visc", 0), params.get("mu", 0.0),
                     params.get("prandtl", 0.72), params.get("r_gas", 1.0), params.get("sutherland", 0),
                     params.get("t_ref", 273.15), params.get("s_suth", 110.4)], dtype=np.float64)


# ---------------------------------------------------------------------------
# pieces (for the closed-form checks)
# ---------------------------------------------------------------------------

def roe_flux(params: dict, VL, VR, S, dim: int = 3) -> np.ndarray:
    """Roe face flux F^(V_L, V_R, S/|S|) * |S| (primitive inputs)."""
    out = np.zeros(5)
    pa = params_array(params, dim)
    lib().oracle_roe_flux(_p(pa), _p(np.ascontiguousarray(VL, dtype=np.float64)),
                          _p(np.ascontiguousarray(VR, dtype=np.float64)),
                          _p(np.ascontiguousarray(S, dtype=np.float64)), _p(out))
    return out


def face_flux(params: dict, VL, VR, S, dim: int = 3) -> np.ndarray:
    """Face flux of the configured function (params["flux"]: 0 Roe, 1 van Leer
    flux-vector splitting, 2 Steger-Warming) times |S|."""
    out = np.zeros(5)
    pa = params_array(params, dim)
    lib().oracle_face_flux(_p(pa), _p(np.ascontiguousarray(VL, dtype=np.float64)),
                           _p(np.ascontiguousarray(VR, dtype=np.float64)),
                           _p(np.ascontiguousarray(S, dtype=np.float64)), _p(out))
    return out


def muscl(params: dict, v4) -> np.ndarray:
    """Eq. (flux) for one component: returns (V^L_{i+1/2}, V^R_{i+1/2})."""
    out = np.zeros(2)
    pa = params_array(params, 3)
    lib().oracle_muscl(_p(pa), _p(np.ascontiguousarray(v4, dtype=np.float64)), _p(out))
    return out


def limited(params: dict, a: float, b: float) -> float:
    """Psi(a/b) * b for the configured limiter."""
    pa = params_array(params, 3)
    return lib().oracle_limited(_p(pa), float(a), float(b))


def cons_to_prim(q, gamma: float = 1.4) -> np.ndarray:
    out = np.zeros(5)
    lib().oracle_cons_to_prim(gamma, _p(np.ascontiguousarray(q, dtype=np.float64)), _p(out))
    return out


def farfield_state(Vi, Vinf, n_out, gamma: float = 1.4) -> np.ndarray:
    """Characteristic farfield boundary state (primitive) from the interior
    state, the free stream and the outward unit normal."""
    out = np.zeros(5)
    lib().oracle_farfield_state(gamma, _p(np.ascontiguousarray(Vi, dtype=np.float64)),
                                _p(np.ascontiguousarray(Vinf, dtype=np.float64)),
                                _p(np.ascontiguousarray(n_out, dtype=np.float64)), _p(out))
    return out


def wall_flux(p1: float, p2: float, S) -> np.ndarray:
    """Overwritten slip-wall face flux from the two nearest interior pressures."""
    out = np.zeros(5)
    lib().oracle_wall_flux(float(p1), float(p2), _p(np.ascontiguousarray(S, dtype=np.float64)), _p(out))
    return out


def viscous_face(params: dict, V10, geo2, axis: int, S, dim: int = 3) -> np.ndarray:
    """Viscous flux times area of one face from its stencil: V10 = primitives
    (10 x 5) of L, R, L-b, L+b, R-b, R+b, L-c, L+c, R-c, R+c; geo2 = (Omega,
    Sbar_xi, Sbar_eta, Sbar_zeta) of L and R (2 x 10)."""
    out = np.zeros(5)
    pa = params_array(params, dim)
    lib().oracle_viscous_face(_p(pa), _p(np.ascontiguousarray(V10, dtype=np.float64)),
                              _p(np.ascontiguousarray(geo2, dtype=np.float64)), int(axis),
                              _p(np.ascontiguousarray(S, dtype=np.float64)), _p(out))
    return out


def viscous_opcount(params: dict) -> dict:
    """Operation counts of one viscous face (gradients, stresses, flux)."""
    out = np.zeros(6, dtype=np.int64)
    lib().oracle_viscous_opcount(_p(params_array(params, 3)), _p(out))
    return dict(zip(("add", "mul", "div", "sqrt", "abs", "cmp"), map(int, out)))


def face_opcount(params: dict) -> dict:
    """Operation counts of one face (5 reconstructed components + Roe flux)."""
    rng = np.random.default_rng(0)
    V = np.empty((5, 4))
    base = np.array([1.0, 0.3, 0.2, 0.1, 0.8])
    for n in range(5):
        V[n] = base[n] + 0.01 * rng.standard_normal(4)
    out = np.zeros(6, dtype=np.int64)
    pa = params_array(params, 3)
    lib().oracle_face_opcount(_p(pa), _p(np.ascontiguousarray(V)), _p(np.array([0.8, 0.1, 0.05])), _p(out))
    return dict(zip(("add", "mul", "div", "sqrt", "abs", "cmp"), map(int, out)))


# ---------------------------------------------------------------------------
# whole-problem driver
# ---------------------------------------------------------------------------

class Oracle:
    """Oracle solver bound to one ``cases.Problem`` (geometry, connections,
    parameters).  States are packed ghosted float64 arrays; residuals are
    packed interior arrays (5, nk, nj, ni) per block, in block order."""

    def __init__(self, problem, threads: Optional[int] = None):
        import cases  # generators only
        self.pb = problem
        self.blocks = problem.blocks
        self.dim = problem.dim
        self.params = dict(problem.params)
        self.pa = params_array(self.params, self.dim)
        self.alpha = tuple(self.params["alpha"])
        self.M = len(self.alpha)
        if threads is not None:
            set_threads(threads)
        L = lib()
        self.metrics = []
        for b in self.blocks:
            ni, nj, nk = b.ni, b.nj, b.nk
            Sxi = np.zeros((3, nk, nj, ni + 1))
            Seta = np.zeros((3, nk, nj + 1, ni))
            Szeta = np.zeros((3, nk + 1, nj, ni))
            vol = np.zeros((nk, nj, ni))
            nodes = None if b.nodes is None else np.ascontiguousarray(b.nodes, dtype=np.float64)
            h = np.array(b.h, dtype=np.float64)
            L.oracle_metrics(ni, nj, nk, _p(nodes), _p(h), _p(Sxi), _p(Seta), _p(Szeta), _p(vol))
            self.metrics.append((Sxi, Seta, Szeta, vol))
        self.dims = np.array([[b.ni, b.nj, b.nk] for b in self.blocks], dtype=np.int32)
        self.offs = np.array(cases.core.block_offsets(self.blocks), dtype=np.int64)
        self.conns = cases.conn_array(problem.conns)
        self.src = problem.source
        self.ncell = [b.ni * b.nj * b.nk for b in self.blocks]
        self.roffs = np.concatenate([[0], np.cumsum([5 * n for n in self.ncell])]).astype(np.int64)
        # physical boundaries: patches and, per block, the six face maps of
        # overwritten-flux codes (None when the block has no such face)
        self.bcs = list(getattr(problem, "bcs", []) or [])
        self.codes = []
        for n, b in enumerate(self.blocks):
            sizes = [b.nj * b.nk, b.nj * b.nk, b.ni * b.nk, b.ni * b.nk, b.ni * b.nj, b.ni * b.nj]
            maps = [np.zeros(sz, dtype=np.int8) for sz in sizes]
            any_code = False
            for pt in self.bcs:
                if pt.block != n or pt.kind not in (cases.BC_SLIP_WALL, cases.BC_FARFIELD, cases.BC_NOSLIP_WALL):
                    continue
                ext0 = b.nj if pt.face < 2 else b.ni
                m = maps[pt.face]
                for t1 in range(pt.lo[1], pt.hi[1]):
                    m[t1 * ext0 + pt.lo[0]:t1 * ext0 + pt.hi[0]] = pt.kind
                any_code = True
            self.codes.append(np.ascontiguousarray(np.concatenate(maps)) if any_code else None)
        self.visc = bool(self.params.get("visc", 0))
        self.geo = self._aux_geometry() if self.visc else None

    # -- viscous geometry -----------------------------------------------------
    def _aux_geometry(self) -> List[np.ndarray]:
        """Per block, the auxiliary-volume geometry of every cell of the block
        padded by one layer: (10, nk+2, nj+2, ni+2) = Omega, Sbar_xi,
        Sbar_eta, Sbar_zeta (cell-averaged face vectors).  Ghost cells of a
        connected face take the donor cell's geometry with its face families
        mapped to this block's axes (sign flipped where an index direction
        reverses); other ghost cells copy the adjacent interior cell."""
        geos = []
        for n, b in enumerate(self.blocks):
            Sxi, Seta, Szeta, vol = self.metrics[n]
            G = np.zeros((10, b.nk + 2, b.nj + 2, b.ni + 2))
            I = (slice(1, b.nk + 1), slice(1, b.nj + 1), slice(1, b.ni + 1))
            G[(0,) + I] = vol
            G[(slice(1, 4),) + I] = 0.5 * (Sxi[..., :-1] + Sxi[..., 1:])
            G[(slice(4, 7),) + I] = 0.5 * (Seta[:, :, :-1, :] + Seta[:, :, 1:, :])
            G[(slice(7, 10),) + I] = 0.5 * (Szeta[:, :-1] + Szeta[:, 1:])
            # face ghosts: copies of the adjacent interior cell
            G[:, 1:-1, 1:-1, 0] = G[:, 1:-1, 1:-1, 1]
            G[:, 1:-1, 1:-1, -1] = G[:, 1:-1, 1:-1, -2]
            G[:, 1:-1, 0, 1:-1] = G[:, 1:-1, 1, 1:-1]
            G[:, 1:-1, -1, 1:-1] = G[:, 1:-1, -2, 1:-1]
            G[:, 0, 1:-1, 1:-1] = G[:, 1, 1:-1, 1:-1]
            G[:, -1, 1:-1, 1:-1] = G[:, -2, 1:-1, 1:-1]
            geos.append(G)
        for c in self.pb.conns:
            db, sbk = self.blocks[c.dst_block], self.blocks[c.src_block]
            da, sa = c.dst_face // 2, c.src_face // 2
            dext, sext = (db.ni, db.nj, db.nk), (sbk.ni, sbk.nj, sbk.nk)
            dtan = [x for x in range(3) if x != da]
            stan = [x for x in range(3) if x != sa]
            # family of the donor and sign for each of this block's axes
            fam, sgn = [0, 0, 0], [1.0, 1.0, 1.0]
            fam[da] = sa
            sgn[da] = 1.0 if (c.dst_face % 2) != (c.src_face % 2) else -1.0
            for t in range(2):
                fam[dtan[t]] = stan[abs(c.transform[t]) - 1]
                sgn[dtan[t]] = 1.0 if c.transform[t] > 0 else -1.0
            Gd, Gs = geos[c.dst_block], geos[c.src_block]
            for bb in range(c.dst_hi[1] - c.dst_lo[1]):
                for aa in range(c.dst_hi[0] - c.dst_lo[0]):
                    dc = [0, 0, 0]
                    dc[dtan[0]], dc[dtan[1]] = c.dst_lo[0] + aa, c.dst_lo[1] + bb
                    dc[da] = -1 if c.dst_face % 2 == 0 else dext[da]
                    st = [c.src_lo[0], c.src_lo[1]]
                    st[abs(c.transform[0]) - 1] += aa if c.transform[0] > 0 else -aa
                    st[abs(c.transform[1]) - 1] += bb if c.transform[1] > 0 else -bb
                    sc = [0, 0, 0]
                    sc[stan[0]], sc[stan[1]] = st[0], st[1]
                    sc[sa] = 0 if c.src_face % 2 == 0 else sext[sa] - 1
                    src = Gs[:, sc[2] + 1, sc[1] + 1, sc[0] + 1]
                    dst = Gd[:, dc[2] + 1, dc[1] + 1, dc[0] + 1]
                    dst[0] = src[0]
                    for d in range(3):
                        dst[1 + 3 * d:4 + 3 * d] = sgn[d] * src[1 + 3 * fam[d]:4 + 3 * fam[d]]
        return [np.ascontiguousarray(G) for G in geos]

    def edge_fill(self, q: np.ndarray) -> np.ndarray:
        """Depth-1 edge ghosts (connection extensions, else the mean of the two
        face-adjacent ghosts), in place."""
        lib().oracle_edge_fill(len(self.conns), _p(self.conns) if len(self.conns) else None, _p(self.dims),
                               _p(self.offs), self.dim, len(self.blocks), _p(q))
        return q

    # -- pieces ---------------------------------------------------------------
    def block_view(self, q: np.ndarray, n: int) -> np.ndarray:
        import cases
        b = self.blocks[n]
        return q[self.offs[n]:self.offs[n] + 5 * cases.core.ghosted_cells(b)]

    def exchange(self, q: np.ndarray) -> np.ndarray:
        """Connected-boundary ghost fill, in place (Section 2 / Section 4)."""
        if len(self.conns):
            lib().oracle_exchange(len(self.conns), _p(self.conns), _p(self.dims), _p(self.offs), _p(q))
        return q

    def apply_bcs(self, q: np.ndarray) -> np.ndarray:
        """Physical-boundary ghost fill of every patch, in place (Section 2;
        Section 7.2, V2/V3)."""
        for pt in self.bcs:
            b = self.blocks[pt.block]
            Sxi, Seta, Szeta, _ = self.metrics[pt.block]
            qb = self.block_view(q, pt.block)
            assert qb.flags["C_CONTIGUOUS"]
            st = np.ascontiguousarray(pt.state, dtype=np.float64)
            lib().oracle_bc_fill(_p(self.pa), b.ni, b.nj, b.nk, _p(Sxi), _p(Seta), _p(Szeta), int(pt.face),
                                 int(pt.lo[0]), int(pt.lo[1]), int(pt.hi[0]), int(pt.hi[1]), int(pt.kind),
                                 _p(st), qb.ctypes.data_as(_dp))
        return q

    def fill_ghosts(self, q: np.ndarray) -> np.ndarray:
        """Connected-boundary exchange, then the physical boundaries, then
        (laminar terms on) the edge ghosts."""
        q = self.apply_bcs(self.exchange(q))
        return self.edge_fill(q) if self.visc else q

    def residual(self, q: np.ndarray) -> np.ndarray:
        """Residual of every block of the packed state ``q`` as it stands
        (wall and farfield faces overwritten, Section 7.2 V7)."""
        R = np.zeros(int(self.roffs[-1]))
        for n, b in enumerate(self.blocks):
            Sxi, Seta, Szeta, vol = self.metrics[n]
            qb = np.ascontiguousarray(self.block_view(q, n))
            src = None if self.src is None else np.ascontiguousarray(self.src[n], dtype=np.float64)
            Rb = np.zeros(5 * self.ncell[n])
            if self.visc:
                codes = None if self.codes[n] is None else self.codes[n].ctypes.data_as(ctypes.c_char_p)
                lib().oracle_residual_ns(_p(self.pa), b.ni, b.nj, b.nk, _p(Sxi), _p(Seta), _p(Szeta), _p(vol),
                                         _p(self.geo[n]), _p(qb), _p(src), codes, _p(Rb))
            elif self.codes[n] is not None:
                lib().oracle_residual_bc(_p(self.pa), b.ni, b.nj, b.nk, _p(Sxi), _p(Seta), _p(Szeta), _p(vol),
                                         _p(qb), _p(src), self.codes[n].ctypes.data_as(ctypes.c_char_p), _p(Rb))
            else:
                lib().oracle_residual(_p(self.pa), b.ni, b.nj, b.nk, _p(Sxi), _p(Seta), _p(Szeta), _p(vol),
                                      _p(qb), _p(src), _p(Rb))
            R[self.roffs[n]:self.roffs[n + 1]] = Rb
        return R

    def residual_jvp(self, q: np.ndarray, dq: np.ndarray):
        """(R, dR) with dR = dR/dq . dq by dual numbers (ghosts as they stand;
        no overwritten boundary faces)."""
        if any(c is not None for c in self.codes) or self.visc:
            raise NotImplementedError("residual_jvp: boundary overwrites and viscous terms are not linearised")
        R = np.zeros(int(self.roffs[-1]))
        dR = np.zeros_like(R)
        for n, b in enumerate(self.blocks):
            Sxi, Seta, Szeta, vol = self.metrics[n]
            qb = np.ascontiguousarray(self.block_view(q, n))
            dqb = np.ascontiguousarray(self.block_view(dq, n))
            src = None if self.src is None else np.ascontiguousarray(self.src[n], dtype=np.float64)
            Rb = np.zeros(5 * self.ncell[n])
            dRb = np.zeros_like(Rb)
            lib().oracle_residual_jvp(_p(self.pa), b.ni, b.nj, b.nk, _p(Sxi), _p(Seta), _p(Szeta),
                                      _p(vol), _p(qb), _p(dqb), _p(src), _p(Rb), _p(dRb))
            R[self.roffs[n]:self.roffs[n + 1]] = Rb
            dR[self.roffs[n]:self.roffs[n + 1]] = dRb
        return R, dR

    def update(self, q0: np.ndarray, R: np.ndarray, alpha_dt: float) -> np.ndarray:
        """Q^(m) = Q^(0) - alpha_m dt / Omega R on every block's interior."""
        out = np.empty_like(q0)
        for n, b in enumerate(self.blocks):
            vol = self.metrics[n][3]
            q0b = np.ascontiguousarray(self.block_view(q0, n))
            Rb = np.ascontiguousarray(R[self.roffs[n]:self.roffs[n + 1]])
            ob = np.empty_like(q0b)
            lib().oracle_rk_update(b.ni, b.nj, b.nk, float(alpha_dt), _p(vol), _p(q0b), _p(Rb), _p(ob))
            out[self.offs[n]:self.offs[n] + q0b.size] = ob
        return out

    # -- Runge-Kutta ------------------------------------------------------------
    def rk_stage(self, q0: np.ndarray, qin: np.ndarray, m: int, dt: float) -> np.ndarray:
        """Stage m (1..M): fill the ghosts of Q^(m-1) (connections, then
        physical boundaries), R(Q^(m-1)), update."""
        qin = self.fill_ghosts(qin.copy())
        R = self.residual(qin)
        return self.update(q0, R, self.alpha[m - 1] * dt)

    def run(self, q: np.ndarray, dt: float, nstages: int,
            residual_fn: Optional[Callable[[np.ndarray], np.ndarray]] = None) -> np.ndarray:
        """Advance ``nstages`` RK stages (whole steps of M stages, the last one
        possibly partial) from state ``q``.  ``residual_fn`` replaces the Euler
        residual (used to check the stage sequencing on a linear problem)."""
        q0 = q.copy()
        cur = q0
        for s in range(nstages):
            m = s % self.M + 1
            if m == 1:
                q0 = cur
            if residual_fn is None:
                cur = self.rk_stage(q0, cur, m, dt)
            else:
                cur = self.update(q0, residual_fn(cur), self.alpha[m - 1] * dt)
        return cur

    def norms(self, R: np.ndarray):
        """Per-variable L2 (root mean square over all cells) and Linf of R."""
        parts = [R[self.roffs[n]:self.roffs[n + 1]].reshape(5, -1) for n in range(len(self.blocks))]
        allR = np.concatenate(parts, axis=1)
        return np.sqrt(np.mean(allR * allR, axis=1)), np.max(np.abs(allR), axis=1)

    def interior(self, q: np.ndarray) -> List[np.ndarray]:
        import cases
        out = []
        for n, b in enumerate(self.blocks):
            qb = self.block_view(q, n).reshape(cases.ghosted_shape(b))
            out.append(cases.interior_view(b, qb))
        return out
