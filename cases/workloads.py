"""Seeded synthetic workloads shaped like the paper's cases.

The paper's own grids (2D inlet, NACA 0012 C-grid, ONERA M6 wing; Section 8)
are not available, so these synthetic problems stand in for them:

* ``vortex_2d``          2D single block, periodic (isentropic vortex).
* ``mms_3d``             3D single curvilinear block with a manufactured solution.
* ``multiblock_batched`` 64 uneven Cartesian blocks with seeded connections.
* ``large_periodic``     one large periodic Cartesian block, Mach 2 + density bumps.
* ``inlet_2d``           2D supersonic compression-ramp channel: inflow, outflow, walls
                         (stands in for the paper's 2D inlet; inflow of its table).
* ``ellipse_ogrid``      O-grid around a 12 % ellipse, wall + farfield + periodic cut,
                         2D or extruded 3D (stands in for the airfoil / wing cases;
                         free stream of the airfoil table).
* ``channel_uniform``    uniform flow in a perturbed box with every boundary kind
                         (free-stream preservation).

Every array is produced from fixed constants or from ``numpy.random.default_rng``
with the stated seed.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

from .core import (GAMMA, GHOST, BC_EXTRAPOLATE, BC_FARFIELD, BC_SLIP_WALL,
                   BC_SUPERSONIC_INFLOW, BCPatch, BlockDesc, Connection, Problem,
                   default_params, ghosted_shape, nominal_dt, pack_state,
                   periodic_connections, prim_to_cons, unpack_state)

# ---------------------------------------------------------------------------
# geometry helpers (node coordinates and sampling points; no metrics)
# ---------------------------------------------------------------------------

def _node_grid(n_lo, n_hi, h, x0=0.0):
    return x0 + h * np.arange(n_lo, n_hi + 1, dtype=np.float64)


def perturbed_nodes(ni: int, nj: int, nk: int, amp: float = 0.1, lo_pad: int = 0,
                    hi_pad: int = 0) -> np.ndarray:
    """Nodes of a sinusoidally perturbed unit-cube grid (shape (nk+1,nj+1,ni+1,3)
    plus optional padding layers).  With X,Y,Z the uniform node coordinates and
    h the spacing along each axis:
      x = X + amp*hx*sin(2 pi Y) sin(2 pi Z)
      y = Y + amp*hy*sin(2 pi Z) sin(2 pi X)
      z = Z + amp*hz*sin(2 pi X) sin(2 pi Y)
    A node on a boundary face of [0,1]^3 moves only along that face's normal
    (the boundary faces are wavy, not planar)."""
    hx, hy, hz = 1.0 / ni, 1.0 / nj, 1.0 / nk
    X = _node_grid(-lo_pad, ni + hi_pad, hx)
    Y = _node_grid(-lo_pad, nj + hi_pad, hy)
    Z = _node_grid(-lo_pad, nk + hi_pad, hz)
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    s = np.sin
    tp = 2.0 * math.pi
    nodes = np.empty(Xg.shape + (3,), dtype=np.float64)
    nodes[..., 0] = Xg + amp * hx * s(tp * Yg) * s(tp * Zg)
    nodes[..., 1] = Yg + amp * hy * s(tp * Zg) * s(tp * Xg)
    nodes[..., 2] = Zg + amp * hz * s(tp * Xg) * s(tp * Yg)
    return nodes


def _cell_points(nodes_padded: np.ndarray) -> np.ndarray:
    """Sampling point of each cell: the mean of its 8 corner nodes."""
    n = nodes_padded
    return 0.125 * (n[:-1, :-1, :-1] + n[:-1, :-1, 1:] + n[:-1, 1:, :-1] + n[:-1, 1:, 1:]
                    + n[1:, :-1, :-1] + n[1:, :-1, 1:] + n[1:, 1:, :-1] + n[1:, 1:, 1:])


def _cartesian_points(b: BlockDesc, pad: int) -> np.ndarray:
    """Cell centres of a Cartesian block (including ``pad`` ghost layers)."""
    x = b.x0[0] + b.h[0] * (np.arange(-pad, b.ni + pad) + 0.5)
    y = b.x0[1] + b.h[1] * (np.arange(-pad, b.nj + pad) + 0.5)
    z = b.x0[2] + b.h[2] * (np.arange(-pad, b.nk + pad) + 0.5)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


# ---------------------------------------------------------------------------
# Manufactured solution (smooth sin/cos fields in rho, u, v, w, p)
# ---------------------------------------------------------------------------

# phi = phi0 + phix sin(ax pi x) + phiy cos(ay pi y) + phiz sin(az pi z), L = 1
_MMS = {
    "rho": (1.0, 0.15, -0.1, 0.1, 1.0, 0.5, 1.0 / 3.0),
    "u": (0.4, 0.05, 0.03, 0.02, 1.5, 0.6, 0.5),
    "v": (0.3, -0.04, 0.05, 0.02, 0.5, 2.0 / 3.0, 1.0),
    "w": (0.25, 0.03, 0.02, -0.04, 1.0 / 3.0, 1.0, 0.5),
    "p": (1.0 / GAMMA, 0.02, 0.01, -0.015, 2.0, 1.0, 1.5),
}
_MMS_ORDER = ("rho", "u", "v", "w", "p")
# the same form with wave numbers that make every field 1-periodic in x, y, z
_MMS_PERIODIC = {
    "rho": (1.0, 0.15, -0.1, 0.1, 2.0, 2.0, 2.0),
    "u": (0.4, 0.05, 0.03, 0.02, 2.0, 4.0, 2.0),
    "v": (0.3, -0.04, 0.05, 0.02, 4.0, 2.0, 2.0),
    "w": (0.25, 0.03, 0.02, -0.04, 2.0, 2.0, 4.0),
    "p": (1.0 / GAMMA, 0.02, 0.01, -0.015, 2.0, 2.0, 2.0),
}


def mms_primitives(x, y, z, table=None):
    """Manufactured primitive fields (rho,u,v,w,p) and their gradients.
    Returns (P, dPdx, dPdy, dPdz), each of shape (5,) + x.shape."""
    pi = math.pi
    P, Dx, Dy, Dz = [], [], [], []
    for name in _MMS_ORDER:
        f0, fx, fy, fz, ax, ay, az = (table or _MMS)[name]
        P.append(f0 + fx * np.sin(ax * pi * x) + fy * np.cos(ay * pi * y) + fz * np.sin(az * pi * z))
        Dx.append(fx * ax * pi * np.cos(ax * pi * x))
        Dy.append(-fy * ay * pi * np.sin(ay * pi * y))
        Dz.append(fz * az * pi * np.cos(az * pi * z))
    return np.array(P), np.array(Dx), np.array(Dy), np.array(Dz)


def mms_second_derivatives(x, y, z, table=None):
    """d2P/dx2, d2P/dy2, d2P/dz2 of the manufactured fields (each field is a
    sum of one-variable functions, so every mixed derivative is zero)."""
    pi = math.pi
    Dxx, Dyy, Dzz = [], [], []
    for name in _MMS_ORDER:
        f0, fx, fy, fz, ax, ay, az = (table or _MMS)[name]
        Dxx.append(-fx * (ax * pi) ** 2 * np.sin(ax * pi * x))
        Dyy.append(-fy * (ay * pi) ** 2 * np.cos(ay * pi * y))
        Dzz.append(-fz * (az * pi) ** 2 * np.sin(az * pi * z))
    return np.array(Dxx), np.array(Dyy), np.array(Dzz)


def viscosity(T, params: dict):
    """Laminar viscosity and dmu/dT: constant, or Sutherland's law
    mu = mu_ref (T/T_ref)^(3/2) (T_ref + S)/(T + S)."""
    mu0 = params["mu"]
    if not params.get("sutherland", 0):
        return mu0 * np.ones_like(T), np.zeros_like(T)
    Tr, S = params["t_ref"], params["s_suth"]
    mu = mu0 * (T / Tr) ** 1.5 * (Tr + S) / (T + S)
    return mu, mu * (1.5 / T - 1.0 / (T + S))


def mms_viscous_divergence(x, y, z, params: dict, table=None) -> np.ndarray:
    """div F_v of the manufactured fields (Section 2: tau by Stokes's
    hypothesis, Theta = tau.u + k grad T, k = mu c_p / Pr,
    c_p = gamma R/(gamma - 1), T = p/(rho R)).  With every mixed derivative
    zero, d_j tau_ij = mu (lap u_i + d_i div u / 3) + A_ij d_j mu, A = tau / mu."""
    g, R, Pr = params["gamma"], params["r_gas"], params["prandtl"]
    cp = g * R / (g - 1.0)
    P, Dx, Dy, Dz = mms_primitives(x, y, z, table)
    D2 = mms_second_derivatives(x, y, z, table)
    D1 = (Dx, Dy, Dz)
    rho, p = P[0], P[4]
    T = p / (rho * R)
    dT = [(D1[j][4] / rho - p * D1[j][0] / rho ** 2) / R for j in range(3)]
    d2T = [(D2[j][4] / rho - 2 * D1[j][4] * D1[j][0] / rho ** 2 - p * D2[j][0] / rho ** 2
            + 2 * p * D1[j][0] ** 2 / rho ** 3) / R for j in range(3)]
    mu, dmu_dT = viscosity(T, params)
    dmu = [dmu_dT * dT[j] for j in range(3)]
    vel = [P[1], P[2], P[3]]
    G = [[D1[j][1 + i] for j in range(3)] for i in range(3)]       # G[i][j] = d u_i / d x_j
    div = G[0][0] + G[1][1] + G[2][2]
    A = [[G[i][j] + G[j][i] - (2.0 / 3.0 if i == j else 0.0) * div for j in range(3)] for i in range(3)]
    out = np.zeros_like(P)
    divtau = []
    for i in range(3):
        lap = D2[0][1 + i] + D2[1][1 + i] + D2[2][1 + i]
        t = mu * (lap + D2[i][1 + i] / 3.0) + sum(A[i][j] * dmu[j] for j in range(3))
        divtau.append(t)
        out[1 + i] = t
    k = mu * cp / Pr
    dk = [cp / Pr * dmu[j] for j in range(3)]
    out[4] = (sum(divtau[i] * vel[i] for i in range(3))
              + mu * sum(A[i][j] * G[i][j] for i in range(3) for j in range(3))
              + k * (d2T[0] + d2T[1] + d2T[2]) + sum(dk[j] * dT[j] for j in range(3)))
    return out


def mms_source(x, y, z, gamma: float = GAMMA, table=None) -> np.ndarray:
    """Source S = div F(Q_exact) of the steady Euler equations for the
    manufactured fields, by the chain rule on the analytic gradients.  This is
    the manufactured PDE's own right-hand side (Section 2: S may come from the
    method of manufactured solutions), a property of the problem, not of the
    discretisation."""
    P, Dx, Dy, Dz = mms_primitives(x, y, z, table)
    rho, u, v, w, p = P
    vel = (u, v, w)
    q2 = u * u + v * v + w * w
    rhoH = gamma / (gamma - 1.0) * p + 0.5 * rho * q2
    S = np.zeros_like(P)
    for a, D in enumerate((Dx, Dy, Dz)):
        drho, du, dv, dw, dp = D
        dvel = (du, dv, dw)
        ua, dua = vel[a], dvel[a]
        m = rho * ua
        dm = drho * ua + rho * dua
        S[0] += dm
        for b in range(3):
            S[1 + b] += dm * vel[b] + m * dvel[b] + (dp if a == b else 0.0)
        drhoH = gamma / (gamma - 1.0) * dp + 0.5 * drho * q2 + rho * (u * du + v * dv + w * dw)
        S[4] += dua * rhoH + ua * drhoH
    return S


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def vortex_2d(n: int = 64, beta: float = 5.0, mach: float = 0.5, cfl: float = 0.5,
              **param_over) -> Problem:
    """2D isentropic vortex on [-5,5]^2, periodic, n x n Cartesian cells.

    Free stream rho = p = 1 (T = 1, c = sqrt(gamma)), speed mach*c at 45 degrees;
    vortex of strength beta centred at the origin:
      du = -beta/(2 pi) y e^{(1-r^2)/2},  dv = beta/(2 pi) x e^{(1-r^2)/2},
      T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) e^{1-r^2},  rho = T^{1/(gamma-1)},
      p = rho^gamma.  Point values at cell centres, unit depth in z."""
    g = GAMMA
    h = 10.0 / n
    b = BlockDesc(n, n, 1, None, (-5.0, -5.0, 0.0), (h, h, 1.0))
    pts = _cartesian_points(b, GHOST)[GHOST:GHOST + 1]  # k ghosts take the k=0 values
    X, Y = pts[..., 0], pts[..., 1]
    r2 = X * X + Y * Y
    cinf = math.sqrt(g)
    uinf = vinf = mach * cinf / math.sqrt(2.0)
    e = np.exp(0.5 * (1.0 - r2))
    u = uinf - beta / (2 * math.pi) * Y * e
    v = vinf + beta / (2 * math.pi) * X * e
    T = 1.0 - (g - 1.0) * beta ** 2 / (8.0 * g * math.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (g - 1.0))
    p = rho ** g
    prim = np.array([rho, u, v, np.zeros_like(u), p])
    prim = np.repeat(prim, 1 + 2 * GHOST, axis=1)
    q = prim_to_cons(prim)
    interior = prim[:, GHOST:GHOST + 1, GHOST:GHOST + n, GHOST:GHOST + n]
    dt = nominal_dt([interior], [b.h], cfl, 2)
    conns = periodic_connections(0, b, axes=(0, 1))
    return Problem([b], conns, 2, pack_state([b], [q]), None, dt,
                   default_params(**param_over), "vortex_2d_%d" % n)


def _mms_block(n_or_dims, curvilinear: bool, amp: float):
    if isinstance(n_or_dims, int):
        ni = nj = nk = n_or_dims
    else:
        ni, nj, nk = n_or_dims
    padded = perturbed_nodes(ni, nj, nk, amp if curvilinear else 0.0, GHOST, GHOST)
    nodes = np.ascontiguousarray(padded[GHOST:GHOST + nk + 1, GHOST:GHOST + nj + 1, GHOST:GHOST + ni + 1])
    if curvilinear:
        b = BlockDesc(ni, nj, nk, nodes)
    else:
        b = BlockDesc(ni, nj, nk, None, (0.0, 0.0, 0.0), (1.0 / ni, 1.0 / nj, 1.0 / nk))
    return b, padded


def mms_3d(n=128, curvilinear: bool = True, amp: float = 0.1, cfl: float = 0.5,
           with_source: bool = True, **param_over) -> Problem:
    """3D manufactured-solution block on [0,1]^3 (perturbed-curvilinear when
    ``curvilinear``).  Initial state and all ghost cells (fixed, Dirichlet) hold
    the exact fields at the cell sampling points; the source is the
    manufactured S at the interior sampling points (per unit volume), of the
    Euler equations, or of the laminar Navier-Stokes equations when the
    parameters set visc = 1."""
    b, padded = _mms_block(n, curvilinear, amp)
    pts = _cell_points(padded)                       # ghosted cell points
    P, _, _, _ = mms_primitives(pts[..., 0], pts[..., 1], pts[..., 2])
    q = prim_to_cons(P)
    g = GHOST
    src = None
    params = default_params(**param_over)
    if with_source:
        ip = pts[g:g + b.nk, g:g + b.nj, g:g + b.ni]
        S = mms_source(ip[..., 0], ip[..., 1], ip[..., 2])
        if params["visc"]:
            S = S - mms_viscous_divergence(ip[..., 0], ip[..., 1], ip[..., 2], params)
        src = [np.ascontiguousarray(S)]
    interior = P[:, g:g + b.nk, g:g + b.nj, g:g + b.ni]
    dt = nominal_dt([interior], [(1.0 / b.ni, 1.0 / b.nj, 1.0 / b.nk)], cfl, 3)
    name = "mms_3d_%s%s%s" % ("x".join(map(str, (b.ni, b.nj, b.nk))), "_curv" if curvilinear else "",
                              "_ns" if params["visc"] else "")
    return Problem([b], [], 3, pack_state([b], [q]), src, dt, params, name)


def mms_periodic_3d(n=64, curvilinear: bool = True, amp: float = 0.1, cfl: float = 0.5,
                    with_source: bool = True, **param_over) -> Problem:
    """Manufactured solution with 1-periodic fields (wave numbers 2 pi and
    4 pi) on the periodic unit cube, perturbed-curvilinear when
    ``curvilinear`` (the perturbation is periodic too).  Ghost cells come from
    the periodic connections, so every ghost value and the geometry behind it
    are those of real neighbour cells.  Initial state = the exact fields at
    the cell sampling points; source = the manufactured S (Euler, or laminar
    Navier-Stokes when visc = 1) there."""
    b, padded = _mms_block(n, curvilinear, amp)
    pts = _cell_points(padded)
    P, _, _, _ = mms_primitives(pts[..., 0], pts[..., 1], pts[..., 2], _MMS_PERIODIC)
    q = prim_to_cons(P)
    g = GHOST
    params = default_params(**param_over)
    src = None
    ip = pts[g:g + b.nk, g:g + b.nj, g:g + b.ni]
    if with_source:
        S = mms_source(ip[..., 0], ip[..., 1], ip[..., 2], table=_MMS_PERIODIC)
        if params["visc"]:
            S = S - mms_viscous_divergence(ip[..., 0], ip[..., 1], ip[..., 2], params, _MMS_PERIODIC)
        src = [np.ascontiguousarray(S)]
    interior = P[:, g:g + b.nk, g:g + b.nj, g:g + b.ni]
    dt = nominal_dt([interior], [(1.0 / b.ni, 1.0 / b.nj, 1.0 / b.nk)], cfl, 3)
    if params["visc"] and params["mu"] > 0:
        h = 1.0 / max(b.ni, b.nj, b.nk)
        dt = min(dt, 0.4 * cfl * h * h * float(interior[0].min()) / params["mu"])
    name = "mms_periodic_%d%s%s" % (b.ni, "_curv" if curvilinear else "", "_ns" if params["visc"] else "")
    return Problem([b], periodic_connections(0, b), 3, pack_state([b], [q]), src, dt, params, name)


def uniform_3d(n=16, curvilinear: bool = True, amp: float = 0.1, seed: Optional[int] = None,
               **param_over) -> Problem:
    """Uniform free stream (rho=1.2, u=(0.3,-0.2,0.25), p=0.9) on a
    perturbed grid with all ghosts fixed at the same state."""
    b, _ = _mms_block(n, curvilinear, amp)
    prim = np.array([1.2, 0.3, -0.2, 0.25, 0.9]).reshape(5, 1, 1, 1) * np.ones((1,) + ghosted_shape(b)[1:])
    q = prim_to_cons(prim)
    dt = nominal_dt([prim], [(1.0 / b.ni, 1.0 / b.nj, 1.0 / b.nk)], 0.5, 3)
    return Problem([b], [], 3, pack_state([b], [q]), None, dt, default_params(**param_over), "uniform")


def _tangential_axes(face):
    a = face // 2
    return [x for x in range(3) if x != a]


def multiblock_batched(nblocks: int = 64, lo: int = 16, hi: int = 96, seed: int = 2012,
                       p_connect: float = 0.5, h: float = 1.0 / 64, cfl: float = 0.5,
                       **param_over) -> Problem:
    """Uneven Cartesian blocks with a seeded connection table.

    Block extents are drawn uniformly from [lo, hi] per axis.  Faces are
    visited in a seeded random order; each still-free face is, with
    probability ``p_connect``, connected (both ways) to another random free
    face with a random orientation (a signed tangential axis map) over the
    largest patch both faces hold, placed at random origins.  Unconnected
    faces keep fixed free-stream ghosts.  The initial state is uniform flow
    (rho=1, p=1/gamma so c=1, velocity 0.5(1,1,1)/sqrt(3), M=0.5) with each
    interior conserved variable scaled by 1 + 0.01 U(-1,1) (seed+1)."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(lo, hi + 1, size=(nblocks, 3))
    blocks = [BlockDesc(int(d[0]), int(d[1]), int(d[2]), None, (0.0, 0.0, 0.0), (h, h, h)) for d in dims]
    faces = [(b, f) for b in range(nblocks) for f in range(6)]
    order = rng.permutation(len(faces))
    free = {fc: True for fc in faces}
    conns: List[Connection] = []
    for idx in order:
        A = faces[idx]
        if not free[A] or rng.random() >= p_connect:
            continue
        cands = [fc for fc in faces if free[fc] and fc != A]
        if not cands:
            break
        B = cands[rng.integers(len(cands))]
        ba, fa = A
        bb, fb = B
        ea = [(blocks[ba].ni, blocks[ba].nj, blocks[ba].nk)[x] for x in _tangential_axes(fa)]
        eb = [(blocks[bb].ni, blocks[bb].nj, blocks[bb].nk)[x] for x in _tangential_axes(fb)]
        t0 = int(rng.choice([1, 2]))
        s0 = int(rng.choice([-1, 1]))
        s1 = int(rng.choice([-1, 1]))
        T = (s0 * t0, s1 * (3 - t0))
        L = [min(ea[0], eb[t0 - 1]), min(ea[1], eb[(3 - t0) - 1])]
        dlo = [int(rng.integers(0, ea[t] - L[t] + 1)) for t in range(2)]
        # src start along each src axis
        slo = [0, 0]
        for t in range(2):
            u = abs(T[t]) - 1
            start = int(rng.integers(0, eb[u] - L[t] + 1))
            slo[u] = start if T[t] > 0 else start + L[t] - 1
        conns.append(Connection(ba, fa, tuple(dlo), (dlo[0] + L[0], dlo[1] + L[1]), bb, fb,
                                tuple(slo), T))
        # reverse connection: B's ghosts from A
        rlo, rhi, rsrc, rT = [0, 0], [0, 0], [0, 0], [0, 0]
        for t in range(2):
            u = abs(T[t]) - 1
            s = 1 if T[t] > 0 else -1
            if s > 0:
                rlo[u], rhi[u] = slo[u], slo[u] + L[t]
                rsrc[t] = dlo[t]
            else:
                rlo[u], rhi[u] = slo[u] - L[t] + 1, slo[u] + 1
                rsrc[t] = dlo[t] + L[t] - 1
            rT[u] = s * (t + 1)
        conns.append(Connection(bb, fb, tuple(rlo), tuple(rhi), ba, fa, tuple(rsrc), tuple(rT)))
        free[A] = False
        free[B] = False
    g = GAMMA
    base = np.array([1.0, *(0.5 / math.sqrt(3.0) * np.ones(3)), 1.0 / g])
    prng = np.random.default_rng(seed + 1)
    arrays, prims = [], []
    for b in blocks:
        shp = ghosted_shape(b)
        prim = base.reshape(5, 1, 1, 1) * np.ones((1,) + shp[1:])
        prims.append(prim[:, :1, :1, :1])
        q = prim_to_cons(prim)
        pert = 1.0 + 0.01 * prng.uniform(-1.0, 1.0, size=(5, b.nk, b.nj, b.ni))
        q[:, GHOST:GHOST + b.nk, GHOST:GHOST + b.nj, GHOST:GHOST + b.ni] *= pert
        arrays.append(q)
    dt = nominal_dt(prims, [b.h for b in blocks], cfl, 3) * (1.0 / 1.05)
    return Problem(blocks, conns, 3, pack_state(blocks, arrays), None, dt,
                   default_params(**param_over), "multiblock_%d_seed%d" % (nblocks, seed))


def large_periodic(ni: int = 512, nj: int = 512, nk: int = 256, seed: int = 5, mach: float = 2.0,
                   nbumps: int = 8, cfl: float = 0.5, **param_over) -> Problem:
    """One periodic Cartesian block, h = 1/ni, uniform Mach-2 flow along x
    (c = 1 at rho = 1, p = 1/gamma) with density
    rho = 1 + sum_n 0.1 exp(-|x-x_n|^2 / (2*0.05^2)) (minimum-image distance,
    bump centres x_n uniform in the box from ``seed``) at constant pressure."""
    h = 1.0 / ni
    b = BlockDesc(ni, nj, nk, None, (0.0, 0.0, 0.0), (h, h, h))
    L = np.array([ni * h, nj * h, nk * h])
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(nbumps, 3)) * L
    g = GHOST
    x = h * (np.arange(-g, ni + g) + 0.5)
    y = h * (np.arange(-g, nj + g) + 0.5)
    z = h * (np.arange(-g, nk + g) + 0.5)
    q = np.empty(ghosted_shape(b), dtype=np.float64)
    p = 1.0 / GAMMA
    u = mach
    for kk in range(z.size):
        rho = np.ones((y.size, x.size))
        dz = z[kk] - centres[:, 2]
        dz = dz - L[2] * np.round(dz / L[2])
        for n in range(nbumps):
            dx = x[None, :] - centres[n, 0]
            dx = dx - L[0] * np.round(dx / L[0])
            dy = y[:, None] - centres[n, 1]
            dy = dy - L[1] * np.round(dy / L[1])
            rho += 0.1 * np.exp(-(dx * dx + dy * dy + dz[n] * dz[n]) / (2 * 0.05 ** 2))
        q[0, kk] = rho
        q[1, kk] = rho * u
        q[2, kk] = 0.0
        q[3, kk] = 0.0
        q[4, kk] = p / (GAMMA - 1.0) + 0.5 * rho * u * u
    prim_max = np.array([1.0, u, 0.0, 0.0, p]).reshape(5, 1, 1, 1)
    dt = nominal_dt([prim_max], [b.h], cfl, 3)
    conns = periodic_connections(0, b)
    return Problem([b], conns, 3, pack_state([b], [q]), None, dt,
                   default_params(**param_over), "large_%dx%dx%d" % (ni, nj, nk))


# ---------------------------------------------------------------------------
# multi-block equivalents of single-block problems (for split-vs-unsplit checks)
# ---------------------------------------------------------------------------

def split_problem_i(pb: Problem, cuts: Sequence[int]) -> Problem:
    """Split a single-block problem along i at the given interior cut indices.
    Internal cuts become identity connections; periodic i-connections of the
    original link the last and first pieces; j/k connections of the original
    (periodic) become self-connections of each piece.  Ghost cells of the
    pieces start with the original's values at the same places."""
    assert len(pb.blocks) == 1
    b = pb.blocks[0]
    q = unpack_state(pb.blocks, pb.q)[0]
    edges = [0] + list(cuts) + [b.ni]
    pieces, arrays, srcs = [], [], []
    g = GHOST
    for lo, hi in zip(edges[:-1], edges[1:]):
        if b.nodes is not None:
            nb = BlockDesc(hi - lo, b.nj, b.nk, np.ascontiguousarray(b.nodes[:, :, lo:hi + 1]))
        else:
            nb = BlockDesc(hi - lo, b.nj, b.nk, None,
                           (b.x0[0] + lo * b.h[0], b.x0[1], b.x0[2]), tuple(b.h))
        pieces.append(nb)
        arrays.append(np.ascontiguousarray(q[:, :, :, lo:hi + 2 * g]))
        if pb.source is not None:
            srcs.append(np.ascontiguousarray(pb.source[0][:, :, :, lo:hi]))
    npc = len(pieces)
    conns: List[Connection] = []
    for n in range(npc - 1):
        ext = (b.nj, b.nk)
        conns.append(Connection(n, 1, (0, 0), ext, n + 1, 0, (0, 0), (1, 2)))
        conns.append(Connection(n + 1, 0, (0, 0), ext, n, 1, (0, 0), (1, 2)))
    for c in pb.conns:
        a = c.dst_face // 2
        if a == 0:
            dst = 0 if c.dst_face == 0 else npc - 1
            src = npc - 1 if c.src_face == 1 else 0
            conns.append(Connection(dst, c.dst_face, c.dst_lo, c.dst_hi, src, c.src_face, c.src_lo, c.transform))
        else:
            for n, nb in enumerate(pieces):
                hi0 = nb.ni
                conns.append(Connection(n, c.dst_face, (0, c.dst_lo[1]), (hi0, c.dst_hi[1]), n,
                                        c.src_face, (0, c.src_lo[1]), c.transform))
    return Problem(pieces, conns, pb.dim, pack_state(pieces, arrays), srcs if srcs else None,
                   pb.dt, dict(pb.params), pb.name + "_split%d" % npc)


def rotated_split_problem(pb: Problem, m: int) -> Problem:
    """Split a single curvilinear block (no connections) at i = m into A
    (i < m) and B (i >= m), and store B rotated by 90 degrees about k:
    B's (i', j', k') = (j, L-1-(i-m), k) with L = ni - m.  A's imax face
    connects to B's jmax face and back, with identity tangential maps."""
    assert len(pb.blocks) == 1 and not pb.conns and pb.blocks[0].nodes is not None
    b = pb.blocks[0]
    L = b.ni - m
    g = GHOST
    q = unpack_state(pb.blocks, pb.q)[0]
    A = BlockDesc(m, b.nj, b.nk, np.ascontiguousarray(b.nodes[:, :, :m + 1]))
    qa = np.ascontiguousarray(q[:, :, :, :m + 2 * g])
    # B nodes: nodesB[kn, jn', in'] = nodes[kn, in', m + L - jn']
    nb = b.nodes[:, :, m:]                       # (nk+1, nj+1, L+1, 3)
    nodesB = np.ascontiguousarray(np.transpose(nb, (0, 2, 1, 3))[:, ::-1, :, :])
    B = BlockDesc(b.nj, L, b.nk, nodesB)
    # B state incl. ghosts: QB[v, k', j', i'] = Q[v, k, j = i', i = m + L - 1 - j'] (ghosted indices)
    qb_src = q[:, :, :, m:m + L + 2 * g]          # ghosted i range of B in original frame
    qb = np.ascontiguousarray(np.transpose(qb_src, (0, 1, 3, 2))[:, :, ::-1, :])
    conns = [Connection(0, 1, (0, 0), (b.nj, b.nk), 1, 3, (0, 0), (1, 2)),
             Connection(1, 3, (0, 0), (b.nj, b.nk), 0, 1, (0, 0), (1, 2))]
    srcs = None
    if pb.source is not None:
        s = pb.source[0]
        sa = np.ascontiguousarray(s[:, :, :, :m])
        sb = np.ascontiguousarray(np.transpose(s[:, :, :, m:], (0, 1, 3, 2))[:, :, ::-1, :])
        srcs = [sa, sb]
    return Problem([A, B], conns, pb.dim, pack_state([A, B], [qa, qb]), srcs, pb.dt,
                   dict(pb.params), pb.name + "_rot")


# ---------------------------------------------------------------------------
# physical-boundary workloads (Section 8 cases, synthetic geometry)
# ---------------------------------------------------------------------------

R_AIR = 287.0   # J/(kg K), the gas constant used to turn the tables' (p, T) into rho


def table_state(mach: float, p: float, T: float, alpha_deg: float = 0.0, gamma: float = GAMMA):
    """Primitive (rho, u, v, w, p) of a free stream given by Mach number,
    static pressure [Pa], temperature [K] and angle of attack (in the x-y
    plane), with rho = p / (R T)."""
    rho = p / (R_AIR * T)
    c = math.sqrt(gamma * p / rho)
    a = math.radians(alpha_deg)
    return np.array([rho, mach * c * math.cos(a), mach * c * math.sin(a), 0.0, p])


INLET_INFLOW = dict(mach=4.0, p=12270.0, T=217.0)            # Section 8.1 table
AIRFOIL_FARFIELD = dict(mach=0.25, p=84307.0, T=300.0, alpha_deg=5.0)   # Section 8.2 table
WING_FARFIELD = dict(mach=0.8395, p=315979.763, T=255.556, alpha_deg=3.06)   # Section 8.3 table


def _perturbed_state(prim0: np.ndarray, shape, perturb: float, seed: Optional[int]) -> np.ndarray:
    """prim0 broadcast over ``shape`` with rho and p scaled by 1 + perturb*N(0,1)
    and the velocity shifted by perturb*|u0|*N(0,1) per component (seeded)."""
    prim = prim0.reshape(5, 1, 1, 1) * np.ones((1,) + tuple(shape))
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        speed = max(float(np.linalg.norm(prim0[1:4])), 1e-12)
        prim[0] *= 1.0 + perturb * rng.standard_normal(shape)
        prim[4] *= 1.0 + perturb * rng.standard_normal(shape)
        for c in (1, 2, 3):
            prim[c] += perturb * speed * rng.standard_normal(shape)
    return prim


def _min_spacing(nodes: np.ndarray, dim: int):
    """Smallest node-to-node distance along each index direction."""
    d = []
    for ax in (2, 1, 0)[:dim]:
        diff = np.diff(nodes, axis=ax)
        d.append(float(np.sqrt((diff ** 2).sum(-1)).min()))
    while len(d) < 3:
        d.append(1.0)
    return d


def inlet_2d(ni: int = 416, nj: int = 128, ramp_deg: float = 10.0, perturb: float = 0.0,
             seed: Optional[int] = None, cfl: float = 0.5, **param_over) -> Problem:
    """2D supersonic channel x in [0, 3] between a lower wall that turns up by
    ``ramp_deg`` at x = 1 and a flat upper wall at y = 1 (nodes clustered
    towards the lower wall, eta = (e^{2s} - 1)/(e^2 - 1)).  Inflow (i = 0) is the
    paper's inlet table (Mach 4, 12270 Pa, 217 K), outflow (i = ni) is
    extrapolated, both walls are slip walls.  The initial state is the inflow
    everywhere (optionally perturbed, seeded)."""
    x = 3.0 * np.arange(ni + 1) / ni
    yl = np.where(x > 1.0, (x - 1.0) * math.tan(math.radians(ramp_deg)), 0.0)
    s = np.arange(nj + 1) / nj
    eta = (np.exp(2.0 * s) - 1.0) / (math.exp(2.0) - 1.0)
    nodes = np.zeros((2, nj + 1, ni + 1, 3))
    for kk in range(2):
        nodes[kk, :, :, 0] = x[None, :]
        nodes[kk, :, :, 1] = yl[None, :] + (1.0 - yl[None, :]) * eta[:, None]
        nodes[kk, :, :, 2] = float(kk)
    b = BlockDesc(ni, nj, 1, nodes)
    V0 = table_state(**INLET_INFLOW)
    prim = _perturbed_state(V0, ghosted_shape(b)[1:], perturb, seed)
    q = prim_to_cons(prim)
    dt = nominal_dt([prim], [_min_spacing(nodes, 2)], cfl, 2)
    bcs = [BCPatch(0, 0, (0, 0), (nj, 1), BC_SUPERSONIC_INFLOW, tuple(V0)),
           BCPatch(0, 1, (0, 0), (nj, 1), BC_EXTRAPOLATE),
           BCPatch(0, 2, (0, 0), (ni, 1), BC_SLIP_WALL),
           BCPatch(0, 3, (0, 0), (ni, 1), BC_SLIP_WALL)]
    return Problem([b], [], 2, pack_state([b], [q]), None, dt, default_params(**param_over),
                   "inlet_2d_%dx%d" % (ni, nj), bcs)


def ellipse_ogrid(ni: int = 512, nj: int = 128, nk: int = 1, thickness: float = 0.12,
                  radius: float = 20.0, span: float = 1.0, beta: float = 6.0, perturb: float = 0.0,
                  seed: Optional[int] = None, cfl: float = 0.5, **param_over) -> Problem:
    """O-grid around an ellipse of chord 1 and the given thickness ratio,
    blended to a circle of ``radius``: node (i, j) at angle
    theta_i = -2 pi i / ni (clockwise, so that (i, j, k) is right-handed) is
    (1 - w) (cos t / 2, thickness sin t / 2) + w radius (cos t, sin t) with
    w = (e^{beta s} - 1)/(e^beta - 1), s = j / nj.  The i = 0 / i = ni cut is a
    periodic self-connection, j = 0 is a slip wall, j = nj a farfield.  nk = 1
    is the 2D case, with the paper's airfoil table (Mach 0.25, 84307 Pa, 300 K,
    5 degrees); nk > 1 extrudes it over ``span`` in z with slip walls on both k
    faces (symmetry planes) and takes the wing table (Mach 0.8395,
    315979.763 Pa, 255.556 K, 3.06 degrees)."""
    dim = 2 if nk == 1 else 3
    th = -2.0 * math.pi * np.arange(ni + 1) / ni
    s = np.arange(nj + 1) / nj
    w = (np.exp(beta * s) - 1.0) / (math.exp(beta) - 1.0)
    xe, ye = 0.5 * np.cos(th), 0.5 * thickness * np.sin(th)
    xo, yo = radius * np.cos(th), radius * np.sin(th)
    X = (1.0 - w[:, None]) * xe[None, :] + w[:, None] * xo[None, :]
    Y = (1.0 - w[:, None]) * ye[None, :] + w[:, None] * yo[None, :]
    X[:, ni] = X[:, 0]
    Y[:, ni] = Y[:, 0]
    zs = np.arange(nk + 1) * (span / nk if dim == 3 else 1.0)
    nodes = np.zeros((nk + 1, nj + 1, ni + 1, 3))
    nodes[..., 0] = X[None]
    nodes[..., 1] = Y[None]
    nodes[..., 2] = zs[:, None, None]
    b = BlockDesc(ni, nj, nk, nodes)
    V0 = table_state(**(AIRFOIL_FARFIELD if dim == 2 else WING_FARFIELD))
    prim = _perturbed_state(V0, ghosted_shape(b)[1:], perturb, seed)
    q = prim_to_cons(prim)
    dt = nominal_dt([prim], [_min_spacing(nodes, dim)], cfl, dim)
    conns = periodic_connections(0, b, axes=(0,))
    bcs = [BCPatch(0, 2, (0, 0), (ni, nk), BC_SLIP_WALL),
           BCPatch(0, 3, (0, 0), (ni, nk), BC_FARFIELD, tuple(V0))]
    if dim == 3:
        bcs += [BCPatch(0, 4, (0, 0), (ni, nj), BC_SLIP_WALL),
                BCPatch(0, 5, (0, 0), (ni, nj), BC_SLIP_WALL)]
    return Problem([b], conns, dim, pack_state([b], [q]), None, dt, default_params(**param_over),
                   "ellipse_%dx%dx%d" % (ni, nj, nk), bcs)


def channel_uniform(n: int = 12, supersonic: bool = True, amp: float = 0.1, **param_over) -> Problem:
    """Uniform flow along x through the unit box with perturbed interior nodes
    (every boundary node stays on its planar face).  Supersonic (Mach 2): inflow at i = 0, extrapolated outflow at
    i = n, slip walls on the four other faces.  Subsonic (Mach 0.5): farfield
    on every face.  Either way the exact discrete residual is zero."""
    # x_d = X_d + amp h sin(2 pi X) sin(2 pi Y) sin(2 pi Z): every boundary node stays put
    X = np.arange(n + 1) / n
    Zg, Yg, Xg = np.meshgrid(X, X, X, indexing="ij")
    bump = amp / n * np.sin(2 * math.pi * Xg) * np.sin(2 * math.pi * Yg) * np.sin(2 * math.pi * Zg)
    nodes = np.stack([Xg + bump, Yg - bump, Zg + bump], axis=-1)
    b = BlockDesc(n, n, n, nodes)
    mach = 2.0 if supersonic else 0.5
    V0 = np.array([1.2, mach * math.sqrt(GAMMA * 0.9 / 1.2), 0.0, 0.0, 0.9])
    prim = V0.reshape(5, 1, 1, 1) * np.ones((1,) + ghosted_shape(b)[1:])
    q = prim_to_cons(prim)
    dt = nominal_dt([prim], [(1.0 / n,) * 3], 0.5, 3)
    if supersonic:
        bcs = [BCPatch(0, 0, (0, 0), (n, n), BC_SUPERSONIC_INFLOW, tuple(V0)),
               BCPatch(0, 1, (0, 0), (n, n), BC_EXTRAPOLATE)]
        bcs += [BCPatch(0, f, (0, 0), (n, n), BC_SLIP_WALL) for f in (2, 3, 4, 5)]
    else:
        bcs = [BCPatch(0, f, (0, 0), (n, n), BC_FARFIELD, tuple(V0)) for f in range(6)]
    return Problem([b], [], 3, pack_state([b], [q]), None, dt, default_params(**param_over),
                   "channel_%s_%d" % ("sup" if supersonic else "sub", n), bcs)
