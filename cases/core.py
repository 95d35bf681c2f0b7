"""Problem containers, layout helpers and connection tables (no method arithmetic)."""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

GAMMA = 1.4
GHOST = 2

FACE_IMIN, FACE_IMAX, FACE_JMIN, FACE_JMAX, FACE_KMIN, FACE_KMAX = range(6)

# Jameson-Schmidt-Turkel low-storage coefficients (Section 2 cites the
# explicit M-step Runge-Kutta scheme of Jameson, Schmidt and Turkel 1981).
RK_ALPHA = {2: (0.5, 1.0), 3: (1.0 / 3.0, 0.5, 1.0),
            4: (0.25, 1.0 / 3.0, 0.5, 1.0)}


@dataclass
class BlockDesc:
    """One structured block: interior extents and its geometry.

    ``nodes`` (shape ``(nk+1, nj+1, ni+1, 3)``) gives a curvilinear grid; when
    it is ``None`` the block is Cartesian with origin ``x0`` and spacing ``h``.
    """
    ni: int
    nj: int
    nk: int
    nodes: Optional[np.ndarray] = None
    x0: Sequence[float] = (0.0, 0.0, 0.0)
    h: Sequence[float] = (1.0, 1.0, 1.0)

    @property
    def ncells(self) -> int:
        return self.ni * self.nj * self.nk


@dataclass
class Connection:
    """Ghost layers of ``dst_face`` of ``dst_block`` filled from ``src_block``.

    Faces are numbered imin, imax, jmin, jmax, kmin, kmax = 0..5.  The patch
    covers dst tangential cell indices ``[dst_lo[0], dst_hi[0])`` x
    ``[dst_lo[1], dst_hi[1])`` (tangential axes in (i,j,k) order with the face
    normal removed).  ``src_lo`` are the src tangential indices of the dst
    corner cell ``dst_lo``; ``transform[t]`` = +-(1 or 2) names the src
    tangential axis (1-based, signed) along which a step of dst tangential
    axis ``t`` moves.  Ghost depth d (1 or 2) takes the src interior cell at
    depth d from ``src_face``.
    """
    dst_block: int
    dst_face: int
    dst_lo: Sequence[int]
    dst_hi: Sequence[int]
    src_block: int
    src_face: int
    src_lo: Sequence[int]
    transform: Sequence[int] = (1, 2)


# Physical boundary kinds of a BCPatch.
BC_FIXED, BC_SUPERSONIC_INFLOW, BC_EXTRAPOLATE, BC_SLIP_WALL, BC_FARFIELD, BC_NOSLIP_WALL = range(6)
BC_NAMES = {BC_FIXED: "fixed", BC_SUPERSONIC_INFLOW: "supersonic_inflow", BC_EXTRAPOLATE: "extrapolate",
            BC_SLIP_WALL: "slip_wall", BC_FARFIELD: "farfield", BC_NOSLIP_WALL: "noslip_wall"}


@dataclass
class BCPatch:
    """Physical boundary on face ``face`` of block ``block`` over tangential
    cells ``[lo[0], hi[0]) x [lo[1], hi[1])`` (tangential axes in (i,j,k)
    order with the face normal removed).  ``state`` is the primitive
    (rho, u, v, w, p) of a supersonic inflow or the farfield free stream."""
    block: int
    face: int
    lo: Sequence[int]
    hi: Sequence[int]
    kind: int
    state: Sequence[float] = (0.0, 0.0, 0.0, 0.0, 0.0)


@dataclass
class Problem:
    blocks: List[BlockDesc]
    conns: List[Connection]
    dim: int                      # 2 or 3
    q: np.ndarray                 # packed ghosted conserved state (float64)
    source: Optional[List[np.ndarray]] = None   # per block (5,nk,nj,ni): S per unit volume at centroids
    dt: float = 0.0
    params: dict = field(default_factory=dict)
    name: str = ""
    bcs: List[BCPatch] = field(default_factory=list)

    @property
    def ncells(self) -> int:
        return sum(b.ncells for b in self.blocks)


def default_params(**over) -> dict:
    """Method parameters.  visc = 1 adds the laminar viscous flux (Section 2):
    constant viscosity ``mu`` (sutherland = 0) or Sutherland's law with
    mu(t_ref) = mu (sutherland = 1, constant s_suth); Prandtl number
    ``prandtl``; gas constant ``r_gas`` (T = p / (rho r_gas))."""
    p = dict(gamma=GAMMA, eps=1.0, kappa=-1.0, limiter=1, harten=0.1,
             fix_all=0, va_delta2=1e-12, n_stages=4, flux=0,
             visc=0, mu=0.0, prandtl=0.72, r_gas=1.0, sutherland=0, t_ref=273.15, s_suth=110.4)
    p.update(over)
    p["alpha"] = RK_ALPHA[p["n_stages"]]
    return p


def ghosted_shape(b: BlockDesc):
    return (5, b.nk + 2 * GHOST, b.nj + 2 * GHOST, b.ni + 2 * GHOST)


def ghosted_cells(b: BlockDesc) -> int:
    return (b.nk + 2 * GHOST) * (b.nj + 2 * GHOST) * (b.ni + 2 * GHOST)


def packed_size(blocks: Sequence[BlockDesc]) -> int:
    return sum(5 * ghosted_cells(b) for b in blocks)


def block_offsets(blocks: Sequence[BlockDesc]) -> List[int]:
    offs, o = [], 0
    for b in blocks:
        offs.append(o)
        o += 5 * ghosted_cells(b)
    return offs


def pack_state(blocks: Sequence[BlockDesc], arrays: Sequence[np.ndarray]) -> np.ndarray:
    return np.concatenate([np.ascontiguousarray(a, dtype=np.float64).ravel() for a in arrays])


def unpack_state(blocks: Sequence[BlockDesc], q: np.ndarray) -> List[np.ndarray]:
    out = []
    for b, o in zip(blocks, block_offsets(blocks)):
        out.append(q[o:o + 5 * ghosted_cells(b)].reshape(ghosted_shape(b)))
    return out


def interior_view(b: BlockDesc, a: np.ndarray) -> np.ndarray:
    g = GHOST
    return a[:, g:g + b.nk, g:g + b.nj, g:g + b.ni]


def prim_to_cons(prim: np.ndarray, gamma: float = GAMMA) -> np.ndarray:
    """(rho,u,v,w,p) -> (rho, rho u, rho v, rho w, rho E) with the ideal-gas
    total energy rho E = p/(gamma-1) + rho |u|^2 / 2 (Section 2, vector Q)."""
    rho, u, v, w, p = prim
    q = np.empty_like(prim)
    q[0] = rho
    q[1] = rho * u
    q[2] = rho * v
    q[3] = rho * w
    q[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return q


def nominal_dt(prims: Sequence[np.ndarray], hs: Sequence[Sequence[float]], cfl: float,
               dim: int, gamma: float = GAMMA) -> float:
    """Fixed global time step from the initial primitive field and the nominal
    spacing of every block: dt = CFL / max_c sum_d (|u_d| + c) / h_d."""
    worst = 0.0
    for prim, h in zip(prims, hs):
        rho, u, v, w, p = prim
        c = np.sqrt(gamma * p / rho)
        s = (np.abs(u) + c) / h[0] + (np.abs(v) + c) / h[1]
        if dim == 3:
            s = s + (np.abs(w) + c) / h[2]
        worst = max(worst, float(s.max()))
    return cfl / worst


def periodic_connections(bidx: int, b: BlockDesc, axes=(0, 1, 2)) -> List[Connection]:
    """Self-connections making block ``bidx`` periodic along ``axes``."""
    ext = (b.ni, b.nj, b.nk)
    out = []
    for a in axes:
        t = [x for x in range(3) if x != a]
        hi = (ext[t[0]], ext[t[1]])
        out.append(Connection(bidx, 2 * a, (0, 0), hi, bidx, 2 * a + 1, (0, 0), (1, 2)))
        out.append(Connection(bidx, 2 * a + 1, (0, 0), hi, bidx, 2 * a, (0, 0), (1, 2)))
    return out


CONN_FIELDS = 12


def conn_array(conns: Sequence[Connection]) -> np.ndarray:
    """Connections as an (n, 12) int32 table in the C struct's field order:
    dst_block, dst_face, dst_lo[2], dst_hi[2], src_block, src_face, src_lo[2],
    transform[2]."""
    a = np.zeros((len(conns), CONN_FIELDS), dtype=np.int32)
    for n, c in enumerate(conns):
        a[n] = [c.dst_block, c.dst_face, c.dst_lo[0], c.dst_lo[1], c.dst_hi[0], c.dst_hi[1],
                c.src_block, c.src_face, c.src_lo[0], c.src_lo[1], c.transform[0], c.transform[1]]
    return a


BC_FIELDS = 7


def bc_arrays(bcs: Sequence[BCPatch]):
    """Boundary patches as an (n, 7) int32 table (block, face, lo[2], hi[2],
    kind) and an (n, 5) float64 table of primitive states."""
    a = np.zeros((len(bcs), BC_FIELDS), dtype=np.int32)
    st = np.zeros((len(bcs), 5), dtype=np.float64)
    for n, b in enumerate(bcs):
        a[n] = [b.block, b.face, b.lo[0], b.lo[1], b.hi[0], b.hi[1], b.kind]
        st[n] = b.state
    return a, st
