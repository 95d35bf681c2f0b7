"""Pins of the oracle's physical boundaries (Section 2: slip wall,
supersonic inflow, extrapolated outflow and farfield enforced through ghost
cells; Section 7.2, V7: wall and farfield face fluxes overwritten).

What fixes them independently of the oracle's own code: the 1D Riemann
invariants and the entropy of the characteristic farfield state; exactness
of the linear wall-pressure extrapolation for a linear profile; free-stream
preservation with every boundary kind; mirror symmetry (a slip wall is a
symmetry plane: a half domain with walls reproduces the full symmetric
domain); the closed-box momentum balance (wall forces) and mass/energy
conservation; the wiring of inflow/outflow ghosts; the paper's table values
of the workloads; and the oblique-shock pressure ratio on a compression ramp
at Mach 4 (theta-beta-M relation).
"""
import json
import math
import os

import numpy as np
import pytest

import cases
import oracle
from cases.core import default_params

HERE = os.path.dirname(os.path.abspath(__file__))
FREE = json.load(open(os.path.join(HERE, "golden", "freestreams.json")))
G = 1.4


def sound(V):
    return math.sqrt(G * V[4] / V[0])


def prim(q):
    return oracle.cons_to_prim(q)


# ------------------------------------------------------ farfield state ---

def _random_state(rng, mach_n, n):
    rho = 0.8 + 0.4 * rng.random()
    p = 0.7 + 0.6 * rng.random()
    c = math.sqrt(G * p / rho)
    t = rng.standard_normal(3)
    t -= t.dot(n) * n
    u = mach_n * c * n + 0.3 * c * t
    return np.array([rho, u[0], u[1], u[2], p])


@pytest.mark.parametrize("seed", range(6))
def test_farfield_subsonic_riemann_invariants(seed):
    """Subsonic: V_n + 2c/(g-1) comes from the interior, V_n - 2c/(g-1) from
    the free stream; entropy p/rho^g and the tangential velocity come from
    the side the flow enters from."""
    rng = np.random.default_rng(seed)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    Vi = _random_state(rng, rng.uniform(-0.6, 0.6), n)
    Vf = _random_state(rng, rng.uniform(-0.6, 0.6), n)
    Vb = oracle.farfield_state(Vi, Vf, n)
    vn = lambda V: V[1:4].dot(n)
    rp = lambda V: vn(V) + 2 * sound(V) / (G - 1)
    rm = lambda V: vn(V) - 2 * sound(V) / (G - 1)
    assert rp(Vb) == pytest.approx(rp(Vi), rel=1e-13)
    assert rm(Vb) == pytest.approx(rm(Vf), rel=1e-13, abs=1e-13 * abs(rp(Vi)))
    up = Vi if vn(Vb) >= 0 else Vf
    assert Vb[4] / Vb[0] ** G == pytest.approx(up[4] / up[0] ** G, rel=1e-12)
    tang = lambda V: V[1:4] - vn(V) * n
    assert np.allclose(tang(Vb), tang(up), rtol=0, atol=1e-13 * np.abs(Vi[1:4]).max())


def test_farfield_of_free_stream_is_free_stream():
    rng = np.random.default_rng(3)
    for _ in range(5):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        for mach in (-0.7, -0.2, 0.0, 0.3, 0.9):
            V = _random_state(rng, mach, n)
            assert np.allclose(oracle.farfield_state(V, V, n), V, rtol=1e-13, atol=1e-14)


def test_farfield_supersonic_branches():
    n = np.array([1.0, 0.0, 0.0])
    Vf = np.array([1.0, 0.1, 0.2, 0.0, 1.0 / G])
    Vout = np.array([1.1, 1.5, 0.1, 0.05, 0.8])        # u/c > 1 outward: all from inside
    assert Vout[1] / sound(Vout) > 1
    assert np.array_equal(oracle.farfield_state(Vout, Vf, n), Vout)
    Vin = np.array([1.1, -1.5, 0.1, 0.05, 0.8])        # u/c < -1: all from the free stream
    assert np.array_equal(oracle.farfield_state(Vin, Vf, n), Vf)


# ----------------------------------------------------------- wall flux ---

def test_wall_flux_pressure_only_and_linear_exact():
    """Mass and energy through a wall vanish; the momentum flux is p_w S, and
    the two-cell extrapolation is exact for a linear pressure profile (cell
    centres at h/2 and 3h/2 from the wall)."""
    S = np.array([0.3, -0.2, 0.5])
    a, slope, h = 2.0, -0.7, 0.1
    p1, p2 = a + slope * h / 2, a + slope * 3 * h / 2
    F = oracle.wall_flux(p1, p2, S)
    assert F[0] == 0.0 and F[4] == 0.0
    assert np.allclose(F[1:4], a * S, rtol=1e-14)


# -------------------------------------------- whole-residual behaviour ---

def _flux_scale(o, pb):
    Smax = max(np.sqrt((m[0] ** 2).sum(0)).max() for m in o.metrics)
    V = prim(pb.q.reshape(5, -1)[:, 0])
    return Smax * (abs(V[0]) * (abs(V[1]) + abs(V[2]) + 1) * max(1.0, np.abs(V[1:4]).max()) + V[4])


@pytest.mark.parametrize("supersonic", [True, False])
def test_free_stream_with_every_boundary_kind(supersonic):
    pb = cases.channel_uniform(8, supersonic)
    o = oracle.Oracle(pb)
    R = o.residual(o.fill_ghosts(pb.q.copy()))
    assert np.abs(R).max() < 1e-13 * _flux_scale(o, pb)


def _symmetric_field(X, Y):
    """Smooth field, periodic with period 1 in x and 2 in y, even about y = 0
    and y = 1 in rho, u, p and odd in v (so both lines are symmetry planes)."""
    rho = 1.0 + 0.2 * np.cos(math.pi * Y) + 0.1 * np.sin(2 * math.pi * X)
    u = 0.5 + 0.1 * np.cos(math.pi * Y) * np.cos(2 * math.pi * X)
    v = 0.2 * np.sin(math.pi * Y) * (1.0 + 0.3 * np.cos(2 * math.pi * X))
    p = 1.0 + 0.1 * np.cos(math.pi * Y) + 0.05 * np.sin(2 * math.pi * X)
    return np.array([rho, u, v, np.zeros_like(u), p])


def _cartesian_2d(ni, nj, y0, h, with_walls):
    b = cases.BlockDesc(ni, nj, 1, None, (0.0, y0, 0.0), (1.0 / ni, h, 1.0))
    pts = cases.workloads._cartesian_points(b, cases.GHOST)
    P = _symmetric_field(pts[..., 0], pts[..., 1])
    q = cases.prim_to_cons(P)
    if with_walls:
        conns = cases.periodic_connections(0, b, axes=(0,))
        bcs = [cases.BCPatch(0, 2, (0, 0), (ni, 1), cases.BC_SLIP_WALL),
               cases.BCPatch(0, 3, (0, 0), (ni, 1), cases.BC_SLIP_WALL)]
    else:
        conns = cases.periodic_connections(0, b, axes=(0, 1))
        bcs = []
    return cases.Problem([b], conns, 2, cases.pack_state([b], [q]), None, 1e-3, default_params(), "sym", bcs)


def test_slip_wall_is_a_symmetry_plane():
    """Half domain y in [0,1] with slip walls vs the periodic full domain
    y in [-1,1] of a field symmetric about y = 0 and y = 1: the wall ghosts
    equal the full domain's mirrored cells, every residual row not touching
    a wall is identical, and the mass and energy residuals of the wall rows
    are identical too (the Roe flux through a symmetry plane carries neither)."""
    ni, nj = 16, 8
    h = 1.0 / nj
    half = _cartesian_2d(ni, nj, 0.0, h, True)
    full = _cartesian_2d(ni, 2 * nj, -1.0, h, False)
    oh, of = oracle.Oracle(half), oracle.Oracle(full)
    qh = oh.fill_ghosts(half.q.copy())
    qf = of.fill_ghosts(full.q.copy())
    g = cases.GHOST
    Qh = qh.reshape(cases.ghosted_shape(half.blocks[0]))
    Qf = qf.reshape(cases.ghosted_shape(full.blocks[0]))
    # half-domain ghost rows j = -1, -2 <-> full rows nj - 1, nj - 2 (y < 0)
    for d in (1, 2):
        assert np.allclose(Qh[:, g, g - d, g:g + ni], Qf[:, g, g + nj - d, g:g + ni], rtol=1e-14, atol=1e-15)
        assert np.allclose(Qh[:, g, g + nj - 1 + d, g:g + ni], Qf[:, g, g + 2 * nj - 1 + d, g:g + ni],
                           rtol=1e-14, atol=1e-15)
    Rh = oh.residual(qh).reshape(5, nj, ni)
    Rf = of.residual(qf).reshape(5, 2 * nj, ni)[:, nj:]
    scale = np.abs(Rf).max()
    assert np.abs(Rh[:, 1:nj - 1] - Rf[:, 1:nj - 1]).max() < 1e-13 * scale
    for n in (0, 4):
        assert np.abs(Rh[n, [0, nj - 1]] - Rf[n, [0, nj - 1]]).max() < 1e-13 * scale
    # wall rows: the momentum differs only by the wall pressure rule
    assert np.abs(Rh[2, 0] - Rf[2, 0]).max() > 1e-6 * scale


def test_closed_box_conservation_and_wall_forces():
    """Six slip walls around a perturbed box with a random smooth state:
    total mass and energy residuals vanish, and the total momentum residual
    is the wall pressure force sum(p_w S) over the boundary faces, with
    p_w = (3 p_1 - p_2)/2 computed here from the cell pressures."""
    n = 8
    base = cases.channel_uniform(n, True)
    b = base.blocks[0]
    rng = np.random.default_rng(11)
    shape = cases.ghosted_shape(b)[1:]
    P = np.empty((5,) + shape)
    P[0] = 1.0 + 0.1 * rng.random(shape)
    P[1:4] = 0.3 * rng.standard_normal((3,) + shape)
    P[4] = 1.0 + 0.1 * rng.random(shape)
    q = cases.prim_to_cons(P)
    bcs = [cases.BCPatch(0, f, (0, 0), (n, n), cases.BC_SLIP_WALL) for f in range(6)]
    pb = cases.Problem([b], [], 3, cases.pack_state([b], [q]), None, 1e-3, default_params(), "box", bcs)
    o = oracle.Oracle(pb)
    qf = o.fill_ghosts(pb.q.copy())
    R = o.residual(qf).reshape(5, -1).sum(1)
    g = cases.GHOST
    pc = P[4, g:g + n, g:g + n, g:g + n]          # (k, j, i); boundary nodes unmoved: area h^2, unit axes
    a = (1.0 / n) ** 2
    force = np.zeros(3)
    for ax, (lo1, lo2, hi1, hi2) in enumerate([
            (pc[:, :, 0], pc[:, :, 1], pc[:, :, -1], pc[:, :, -2]),
            (pc[:, 0, :], pc[:, 1, :], pc[:, -1, :], pc[:, -2, :]),
            (pc[0], pc[1], pc[-1], pc[-2])]):
        # the outward face vector is -e_ax on the min face, +e_ax on the max face
        force[ax] = a * ((1.5 * hi1 - 0.5 * hi2).sum() - (1.5 * lo1 - 0.5 * lo2).sum())
    scale = np.abs(force).max() + 1.0
    assert abs(R[0]) < 1e-13 * scale and abs(R[4]) < 1e-12 * scale
    assert np.allclose(R[1:4], force, rtol=0, atol=1e-12 * scale)


def test_farfield_face_flux_is_the_boundary_state_flux():
    """Walls on five faces, a subsonic farfield on imax: the total mass and
    energy residuals are the fluxes of the characteristic boundary states
    (built here from each first interior cell with the pinned farfield
    state) through the imax faces, whose outward vector is (h^2, 0, 0)."""
    n = 6
    b = cases.channel_uniform(n, True).blocks[0]
    rng = np.random.default_rng(21)
    shape = cases.ghosted_shape(b)[1:]
    P = np.empty((5,) + shape)
    P[0] = 1.0 + 0.1 * rng.random(shape)
    P[1:4] = 0.2 * rng.standard_normal((3,) + shape)
    P[4] = 1.0 + 0.1 * rng.random(shape)
    Vf = np.array([1.1, 0.3, -0.1, 0.05, 0.9])
    bcs = [cases.BCPatch(0, f, (0, 0), (n, n), cases.BC_SLIP_WALL) for f in (0, 2, 3, 4, 5)]
    bcs.append(cases.BCPatch(0, 1, (0, 0), (n, n), cases.BC_FARFIELD, tuple(Vf)))
    pb = cases.Problem([b], [], 3, cases.pack_state([b], [cases.prim_to_cons(P)]), None, 1e-3,
                       default_params(), "ff", bcs)
    o = oracle.Oracle(pb)
    R = o.residual(o.fill_ghosts(pb.q.copy())).reshape(5, -1).sum(1)
    g = cases.GHOST
    a = (1.0 / n) ** 2
    mass = energy = 0.0
    for k in range(n):
        for j in range(n):
            Vb = oracle.farfield_state(P[:, g + k, g + j, g + n - 1], Vf, np.array([1.0, 0.0, 0.0]))
            un = Vb[1] * a
            mass += Vb[0] * un
            energy += (G / (G - 1) * Vb[4] + 0.5 * Vb[0] * (Vb[1:4] ** 2).sum()) * un
    assert R[0] == pytest.approx(mass, rel=1e-12, abs=1e-14)
    assert R[4] == pytest.approx(energy, rel=1e-12, abs=1e-14)


def test_inflow_and_outflow_ghost_wiring():
    pb = cases.inlet_2d(20, 8, perturb=0.05, seed=4)
    o = oracle.Oracle(pb)
    q = o.fill_ghosts(pb.q.copy())
    Q = q.reshape(cases.ghosted_shape(pb.blocks[0]))
    g = cases.GHOST
    qin = cases.prim_to_cons(np.array(pb.bcs[0].state).reshape(5, 1))[:, 0]
    for d in (1, 2):
        assert np.allclose(Q[:, g, g:g + 8, g - d], qin[:, None], rtol=1e-15)
        assert np.array_equal(Q[:, g, g:g + 8, g + 20 - 1 + d], Q[:, g, g:g + 8, g + 20 - 1])


def test_farfield_ghost_orientation():
    """Flow along +x at Mach 2: at the imax farfield it leaves supersonically
    (ghost = interior cell), at imin it enters supersonically (ghost = free
    stream): pins the outward-normal sign on both faces."""
    pb = cases.channel_uniform(6, False)
    b = pb.blocks[0]
    Vf = np.array([1.0, 2.2, 0.0, 0.0, 1.0 / G])        # Mach 2.2
    pb.bcs = [cases.BCPatch(0, f, (0, 0), (6, 6), cases.BC_FARFIELD, tuple(Vf)) for f in (0, 1)]
    shape = cases.ghosted_shape(b)[1:]
    rng = np.random.default_rng(5)
    P = np.empty((5,) + shape)
    P[0] = 1.0 + 0.05 * rng.random(shape)
    P[1] = 2.5
    P[2:4] = 0.0
    P[4] = 1.0 / G
    pb.q = cases.pack_state([b], [cases.prim_to_cons(P)])
    o = oracle.Oracle(pb)
    Q = o.fill_ghosts(pb.q.copy()).reshape(cases.ghosted_shape(b))
    g = cases.GHOST
    qf = cases.prim_to_cons(Vf.reshape(5, 1))[:, 0]
    assert np.allclose(Q[:, g:g + 6, g:g + 6, g - 1], qf[:, None, None], rtol=1e-14)
    assert np.allclose(Q[:, g:g + 6, g:g + 6, g + 6], Q[:, g:g + 6, g:g + 6, g + 5], rtol=1e-14)


def test_workloads_use_the_paper_tables():
    R = FREE["gas_constant"]
    for wl, key in ((cases.INLET_INFLOW, "inlet_2d"), (cases.AIRFOIL_FARFIELD, "naca0012"),
                    (cases.WING_FARFIELD, "onera_m6")):
        t = FREE[key]
        V = cases.table_state(**wl)
        assert V[4] == t["pressure_pa"]
        assert V[0] == pytest.approx(t["pressure_pa"] / (R * t["temperature_k"]), rel=1e-15)
        speed = math.hypot(V[1], V[2])
        assert speed / sound(V) == pytest.approx(t["mach"], rel=1e-14)
        assert math.degrees(math.atan2(V[2], V[1])) == pytest.approx(t["alpha_deg"], abs=1e-12)
    assert cases.inlet_2d(8, 4).bcs[0].state == tuple(cases.table_state(**cases.INLET_INFLOW))


def _oblique_shock_pressure_ratio(M, theta):
    """Textbook theta-beta-M relation (weak branch) and the normal-shock
    pressure ratio of the normal Mach number M sin(beta)."""
    def f(beta):
        return 2 / math.tan(beta) * (M * M * math.sin(beta) ** 2 - 1) / (M * M * (G + math.cos(2 * beta)) + 2) \
            - math.tan(theta)
    lo, hi = math.asin(1 / M) + 1e-9, math.radians(64.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0:
            hi = mid
        else:
            lo = mid
    Mn = M * math.sin(0.5 * (lo + hi))
    return 1 + 2 * G / (G + 1) * (Mn * Mn - 1)


@pytest.mark.slow
def test_ramp_wall_pressure_matches_oblique_shock():
    """Mach 4 over a 10 degree compression ramp run to a steady state: the
    wall pressure on the ramp upstream of the reflected shock is the
    oblique-shock value (1.5 % discretisation tolerance on 104 x 32 cells;
    the converged coarse-grid values lie within 0.7 %)."""
    pb = cases.inlet_2d(104, 32, ramp_deg=10.0)
    o = oracle.Oracle(pb)
    q = pb.q.copy()
    for _ in range(2):
        q = o.run(q, pb.dt, 4 * 400)
    V = np.array([prim(c) for c in o.interior(q)[0][:, 0, 0, :].T])
    x = 3.0 * (np.arange(104) + 0.5) / 104
    p_inf = pb.bcs[0].state[4]
    ratio = _oblique_shock_pressure_ratio(4.0, math.radians(10.0))
    sel = (x > 1.3) & (x < 2.8)
    got = V[sel, 4] / p_inf
    assert np.all(np.abs(got / ratio - 1) < 0.015), (got, ratio)
