"""Pins of the oracle's laminar Navier-Stokes terms (Section 2: viscous flux
F_v with Stokes's-hypothesis stresses and Theta = tau.u + k grad T; face
gradients by Green's theorem with a wider stencil).

Independent facts: the manufactured viscous source against nested central
differences of the analytic fields; exactness of the face gradient and of
the viscous flux for linear fields on an arbitrary parallelepiped cell (the
dual-basis identity); Sutherland's law in closed form; second-order
truncation of the viscous operator on a perturbed periodic grid; the decay
rate nu k^2 of a shear wave; discrete conservation; free-stream
preservation; bit-exact 1-block vs 3-block equivalence (the paper's
parallel-vs-serial check of Section 8, here including the ghost geometry and
the edge ghosts); no-slip wall ghosts and an adiabatic, work-free closed box.
"""
import math

import numpy as np
import pytest

import cases
import oracle
from cases.core import default_params
from cases.workloads import mms_primitives, mms_viscous_divergence, viscosity

G = 1.4


def _ns(**kw):
    p = dict(visc=1, mu=0.05, prandtl=0.72, r_gas=1.0)
    p.update(kw)
    return default_params(**p)


def test_manufactured_viscous_source_vs_central_differences():
    """div F_v of the manufactured fields (with Sutherland's law) against a
    second, purely numerical derivation: F_v from central-difference
    gradients, then its divergence by central differences."""
    pr = _ns(sutherland=1, t_ref=0.7, s_suth=0.3)

    def Fv(x, y, z, h=1e-5):
        P0 = mms_primitives(x, y, z)[0]
        grads = [(mms_primitives(x + h * (a == 0), y + h * (a == 1), z + h * (a == 2))[0]
                  - mms_primitives(x - h * (a == 0), y - h * (a == 1), z - h * (a == 2))[0]) / (2 * h)
                 for a in range(3)]
        R, Pr = pr["r_gas"], pr["prandtl"]
        cp = G * R / (G - 1)
        T = P0[4] / (P0[0] * R)
        mu, _ = viscosity(T, pr)
        Gm = [[grads[j][1 + i] for j in range(3)] for i in range(3)]
        div = Gm[0][0] + Gm[1][1] + Gm[2][2]
        tau = [[mu * (Gm[i][j] + Gm[j][i] - (2 / 3 if i == j else 0) * div) for j in range(3)] for i in range(3)]
        dT = [(grads[j][4] / P0[0] - P0[4] * grads[j][0] / P0[0] ** 2) / R for j in range(3)]
        F = np.zeros((3, 5) + np.shape(x))
        for j in range(3):
            for i in range(3):
                F[j, 1 + i] = tau[i][j]
            F[j, 4] = sum(tau[i][j] * P0[1 + i] for i in range(3)) + mu * cp / Pr * dT[j]
        return F

    rng = np.random.default_rng(0)
    x, y, z = rng.random(6), rng.random(6), rng.random(6)
    h = 1e-4
    num = sum((Fv(x + h * (a == 0), y + h * (a == 1), z + h * (a == 2))[a]
               - Fv(x - h * (a == 0), y - h * (a == 1), z - h * (a == 2))[a]) / (2 * h) for a in range(3))
    ana = mms_viscous_divergence(x, y, z, pr)
    assert np.abs(num - ana).max() < 1e-6 * np.abs(ana).max()


def _parallelepiped_stencil(rng, axis):
    """Cells of a uniform parallelepiped grid with edge vectors e0, e1, e2:
    positions of L, R and the tangential neighbours, and the geometry (Omega,
    Sbar per family) shared by all its cells."""
    E = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    if np.linalg.det(E) < 0:
        E[2] *= -1
    e = [E[0], E[1], E[2]]
    Om = e[0].dot(np.cross(e[1], e[2]))
    Sbar = [np.cross(e[1], e[2]), np.cross(e[2], e[0]), np.cross(e[0], e[1])]
    geo = np.concatenate([[Om], Sbar[0], Sbar[1], Sbar[2]])
    a, b, c = axis, (1 if axis == 0 else 0), (1 if axis == 2 else 2)
    xL = rng.standard_normal(3)
    xR = xL + e[a]
    pos = [xL, xR, xL - e[b], xL + e[b], xR - e[b], xR + e[b], xL - e[c], xL + e[c], xR - e[c], xR + e[c]]
    S = Sbar[a]
    return pos, geo, S, xL + 0.5 * e[a]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("seed", [1, 2])
def test_viscous_face_exact_for_linear_fields(axis, seed):
    """u = u0 + Gu x and T linear (rho constant, p = rho R T) on a
    parallelepiped grid: the Green's-theorem gradient is exact (sum_d
    (g.e_d) Sbar_d = Omega g), hence F_v = (0, tau S, (tau u_f) S + k gradT S)
    with tau = mu (Gu + Gu^T - 2/3 tr Gu I) exactly."""
    rng = np.random.default_rng(seed)
    pos, geo, S, xf = _parallelepiped_stencil(rng, axis)
    Gu, u0 = rng.standard_normal((3, 3)), rng.standard_normal(3)
    gT, T0 = 0.1 * rng.standard_normal(3), 2.0
    rho, R, mu = 1.3, 1.0, 0.07
    V10 = []
    for x in pos:
        T = T0 + gT.dot(x)
        V10.append([rho, *(u0 + Gu @ x), rho * R * T])
    pr = _ns(mu=mu, r_gas=R)
    out = oracle.viscous_face(pr, np.array(V10), np.stack([geo, geo]), axis, S)
    tau = mu * (Gu + Gu.T - 2.0 / 3.0 * np.trace(Gu) * np.eye(3))
    k = mu * G * R / (G - 1) / pr["prandtl"]
    uf = u0 + Gu @ xf
    assert out[0] == 0.0
    assert np.allclose(out[1:4], tau @ S, rtol=1e-12, atol=1e-13)
    assert out[4] == pytest.approx((tau @ S).dot(uf) + k * gT.dot(S), rel=1e-11, abs=1e-13)


def test_sutherland_law():
    """A pure shear u = y through a unit face normal to y gives tau_xy = mu(T):
    mu(T_ref) = mu_ref and mu ~ T^1.5 (T_ref + S)/(T + S)."""
    pos, geo, S, _ = _parallelepiped_stencil(np.random.default_rng(3), 1)
    e = np.eye(3)
    geo = np.concatenate([[1.0], e[0], e[1], e[2]])
    pos = [np.zeros(3), e[1], -e[0], e[0], e[1] - e[0], e[1] + e[0], -e[2], e[2], e[1] - e[2], e[1] + e[2]]
    Tr, Sc, mur = 300.0, 110.4, 1.8e-5
    for T in (150.0, 300.0, 1000.0):
        V10 = [[1.0, x[1], 0.0, 0.0, 287.0 * T] for x in pos]
        pr = _ns(mu=mur, r_gas=287.0, sutherland=1, t_ref=Tr, s_suth=Sc)
        out = oracle.viscous_face(pr, np.array(V10), np.stack([geo, geo]), 1, e[1])
        assert out[1] == pytest.approx(mur * (T / Tr) ** 1.5 * (Tr + Sc) / (T + Sc), rel=1e-13)


@pytest.mark.parametrize("suth", [0, 1])
def test_viscous_operator_second_order_on_perturbed_periodic_grid(suth):
    """(R_NS - R_Euler)/Omega = div F_v - sum F_v.S/Omega, the viscous
    truncation error under the periodic manufactured solution: order 2."""
    kw = dict(mu=0.05, limiter=0, sutherland=suth, t_ref=0.7, s_suth=0.3)
    errs = []
    for n in (16, 32):
        Rs = []
        for visc in (0, 1):
            pb = cases.mms_periodic_3d(n, curvilinear=True, visc=visc, **kw)
            o = oracle.Oracle(pb)
            Rs.append(o.residual(o.fill_ghosts(pb.q.copy())).reshape(5, -1) / o.metrics[0][3].ravel())
        errs.append(np.sqrt(np.mean((Rs[1] - Rs[0])[1:] ** 2, axis=1)))
    order = np.log2(errs[0] / errs[1])
    assert np.all(order > 1.9), order


def test_shear_wave_decays_at_nu_k2():
    """u = U sin(2 pi y) in a periodic box (rho = 1, p = 1/gamma, U = 0.01):
    the amplitude decays as exp(-nu k^2 t), nu = mu / rho, k = 2 pi."""
    n, mu, U = 32, 0.01, 0.01
    b = cases.BlockDesc(4, n, 1, None, (0.0, 0.0, 0.0), (1.0 / 4, 1.0 / n, 1.0))
    pts = cases.workloads._cartesian_points(b, cases.GHOST)
    y = pts[..., 1]
    P = np.array([np.ones_like(y), U * np.sin(2 * math.pi * y), 0 * y, 0 * y, np.ones_like(y) / G])
    pb = cases.Problem([b], cases.periodic_connections(0, b, axes=(0, 1)), 2,
                       cases.pack_state([b], [cases.prim_to_cons(P)]), None, 0.0,
                       _ns(mu=mu, limiter=0), "shear")
    o = oracle.Oracle(pb)
    dt, steps = 2e-3, 250
    q = o.run(pb.q.copy(), dt, 4 * steps)
    u = o.interior(q)[0][1, 0, :, 0] / o.interior(q)[0][0, 0, :, 0]
    yc = (np.arange(n) + 0.5) / n
    amp = 2 * np.mean(u * np.sin(2 * math.pi * yc))
    expect = U * math.exp(-mu * (2 * math.pi) ** 2 * dt * steps)
    assert amp == pytest.approx(expect, rel=5e-3)


def test_conservation_and_free_stream():
    pb = cases.mms_periodic_3d(8, curvilinear=True, visc=1, mu=0.05)
    o = oracle.Oracle(pb)
    q = o.fill_ghosts(pb.q.copy())
    R = o.residual(q).reshape(5, -1)
    SO = (pb.source[0].reshape(5, -1) * o.metrics[0][3].ravel())
    tot = (R + SO).sum(1)
    assert np.abs(tot).max() < 1e-13 * np.abs(R).sum(1).max()
    # uniform state on the same grid: zero residual with the viscous terms on
    pu = cases.mms_periodic_3d(8, curvilinear=True, visc=1, mu=0.05, with_source=False)
    V = np.array([1.2, 0.3, -0.2, 0.25, 0.9]).reshape(5, 1, 1, 1) * np.ones((1,) + cases.ghosted_shape(pu.blocks[0])[1:])
    pu.q = cases.pack_state(pu.blocks, [cases.prim_to_cons(V)])
    ou = oracle.Oracle(pu)
    Ru = ou.residual(ou.fill_ghosts(pu.q.copy()))
    assert np.abs(Ru).max() < 1e-14


def test_one_block_equals_three_blocks_bitwise():
    pb = cases.mms_periodic_3d(12, curvilinear=True, visc=1, mu=0.05, sutherland=1, t_ref=0.7, s_suth=0.3)
    sp = cases.split_problem_i(pb, [4, 7])
    o1, o3 = oracle.Oracle(pb), oracle.Oracle(sp)
    R1 = o1.residual(o1.fill_ghosts(pb.q.copy())).reshape(5, 12, 12, 12)
    R3 = o3.residual(o3.fill_ghosts(sp.q.copy()))
    parts = [R3[o3.roffs[n]:o3.roffs[n + 1]].reshape(5, 12, 12, -1) for n in range(3)]
    assert np.array_equal(np.concatenate(parts, axis=3), R1)
    q1 = o1.run(pb.q.copy(), pb.dt, 4)
    q3 = o3.run(sp.q.copy(), sp.dt, 4)
    i1 = o1.interior(q1)[0]
    i3 = np.concatenate(o3.interior(q3), axis=3)
    assert np.array_equal(i1, i3)


def test_noslip_wall_ghosts_and_adiabatic_box():
    """Six no-slip walls around a Cartesian box with a random state: the
    ghosts mirror the interior with the velocity reversed, and the total mass
    and energy residuals vanish (no flux, no work, no heat through the walls)."""
    n = 6
    b = cases.BlockDesc(n, n, n, None, (0.0, 0.0, 0.0), (1.0 / n,) * 3)
    rng = np.random.default_rng(8)
    shape = cases.ghosted_shape(b)[1:]
    P = np.empty((5,) + shape)
    P[0] = 1.0 + 0.1 * rng.random(shape)
    P[1:4] = 0.2 * rng.standard_normal((3,) + shape)
    P[4] = 1.0 + 0.1 * rng.random(shape)
    bcs = [cases.BCPatch(0, f, (0, 0), (n, n), cases.BC_NOSLIP_WALL) for f in range(6)]
    pb = cases.Problem([b], [], 3, cases.pack_state([b], [cases.prim_to_cons(P)]), None, 1e-3, _ns(), "box", bcs)
    o = oracle.Oracle(pb)
    q = o.fill_ghosts(pb.q.copy())
    Q = q.reshape(cases.ghosted_shape(b))
    g = cases.GHOST
    for d in (1, 2):
        assert np.array_equal(Q[0, g:g + n, g:g + n, g - d], Q[0, g:g + n, g:g + n, g + d - 1])
        assert np.array_equal(Q[1:4, g:g + n, g:g + n, g - d], -Q[1:4, g:g + n, g:g + n, g + d - 1])
        assert np.array_equal(Q[4, g:g + n, g:g + n, g - d], Q[4, g:g + n, g:g + n, g + d - 1])
    R = o.residual(q).reshape(5, -1).sum(1)
    scale = np.abs(o.residual(q)).max()
    assert abs(R[0]) < 1e-13 * scale and abs(R[4]) < 1e-13 * scale


def test_rotated_block_geometry_mapping():
    """The 90-degree rotated second block (its jmax face joined to the first
    block's imax face, so one index direction reverses): the donor geometry
    reaches the ghosts with its face families permuted and sign-flipped, and
    the residual matches the single block to rounding."""
    pb = cases.mms_3d(10, curvilinear=True, visc=1, mu=0.05)
    rs = cases.rotated_split_problem(pb, 4)
    o1, o2 = oracle.Oracle(pb), oracle.Oracle(rs)
    R1 = o1.residual(o1.fill_ghosts(pb.q.copy())).reshape(5, 10, 10, 10)
    R2 = o2.residual(o2.fill_ghosts(rs.q.copy()))
    A = R2[o2.roffs[0]:o2.roffs[1]].reshape(5, 10, 10, 4)
    B = R2[o2.roffs[1]:o2.roffs[2]].reshape(5, 10, 6, 10)      # (v, k, j', i') with i' = j, j' = 5 - (i - 4)
    Bo = np.transpose(B[:, :, ::-1, :], (0, 1, 3, 2))
    got = np.concatenate([A, Bo], axis=3)
    scale = np.abs(R1).max()
    assert np.abs(got - R1).max() < 1e-12 * scale
