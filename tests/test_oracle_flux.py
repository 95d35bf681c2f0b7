"""Pins of the oracle's per-face arithmetic against closed forms.

Each check is something the paper or the mathematics fixes independently of
the oracle's code: the inviscid normal flux F_{i,n} printed in Section 2
(consistency), the Roe decomposition's exact upwinding for supersonic states,
a stationary contact, mirror symmetry, limiter identities and the reductions
of Eq. (flux).  Freestream states are the paper's own tables (tests/golden).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from cases.core import default_params

HERE = os.path.dirname(os.path.abspath(__file__))
FREE = json.load(open(os.path.join(HERE, "golden", "freestreams.json")))


def physical_flux(V, S, gamma=1.4):
    """Section 2: F_{i,n} = (rho V_n, rho u V_n + n_x p, rho v V_n + n_y p,
    rho w V_n + n_z p, rho h_t V_n), h_t = gamma/(gamma-1) p/rho + |u|^2/2,
    times the face area |S|."""
    rho, u, v, w, p = V
    A = math.sqrt(S[0] ** 2 + S[1] ** 2 + S[2] ** 2)
    n = np.asarray(S) / A
    Vn = n[0] * u + n[1] * v + n[2] * w
    ht = gamma / (gamma - 1) * p / rho + 0.5 * (u * u + v * v + w * w)
    return A * np.array([rho * Vn, rho * u * Vn + n[0] * p, rho * v * Vn + n[1] * p,
                         rho * w * Vn + n[2] * p, rho * ht * Vn])


def dimensional_state(case, direction=(1.0, 0.0, 0.0)):
    c = FREE[case]
    R, g = FREE["gas_constant"], FREE["gamma"]
    rho = c["pressure_pa"] / (R * c["temperature_k"])
    a = math.sqrt(g * R * c["temperature_k"])
    al = math.radians(c["alpha_deg"])
    speed = c["mach"] * a
    d = np.array(direction, dtype=float)
    vel = speed * np.array([math.cos(al) * d[0] - math.sin(al) * d[1],
                            math.sin(al) * d[0] + math.cos(al) * d[1], d[2]])
    return np.array([rho, vel[0], vel[1], vel[2], c["pressure_pa"]]), a


def rand_state(rng, n=1):
    rho = rng.uniform(0.5, 2.0)
    u, v, w = rng.uniform(-0.6, 0.6, size=3)
    p = rng.uniform(0.5, 2.0)
    return np.array([rho, u, v, w, p])


@pytest.mark.parametrize("harten", [0.0, 0.1])
def test_consistency_equal_states(harten):
    P = default_params(harten=harten)
    rng = np.random.default_rng(1)
    for _ in range(50):
        V = rand_state(rng)
        S = rng.normal(size=3) * 0.01
        got = oracle.roe_flux(P, V, V, S)
        ref = physical_flux(V, S)
        assert np.allclose(got, ref, rtol=1e-14, atol=1e-16 * np.abs(ref).max())


@pytest.mark.parametrize("case", ["inlet_2d", "naca0012", "onera_m6"])
def test_consistency_paper_freestreams(case):
    V, _ = dimensional_state(case)
    S = np.array([0.3, -0.2, 0.1])
    got = oracle.roe_flux(default_params(), V, V, S)
    ref = physical_flux(V, S)
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_supersonic_upwinding(sign):
    """With every eigenvalue of the Roe matrix positive (negative), the Roe
    flux must equal the left (right) physical flux exactly: the wave
    decomposition sum_k lambda_k alpha_k r_k reproduces F(V_R) - F(V_L)
    (Roe's property), so any wrong strength, eigenvector or average fails."""
    V0, a = dimensional_state("inlet_2d")          # Mach 4, Section 8.1 table
    rng = np.random.default_rng(2)
    P = default_params(harten=0.1)
    S = np.array([1.0, 0.0, 0.0]) * 0.02
    for _ in range(20):
        VL = V0 * (1 + 0.05 * rng.uniform(-1, 1, size=5))
        VR = V0 * (1 + 0.05 * rng.uniform(-1, 1, size=5))
        VL[1:4] *= sign
        VR[1:4] *= sign
        got = oracle.roe_flux(P, VL, VR, S)
        ref = physical_flux(VL if sign > 0 else VR, S)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), (got - ref)


def test_supersonic_upwinding_oblique_face():
    rng = np.random.default_rng(3)
    P = default_params(harten=0.0)
    n = np.array([0.6, -0.48, 0.64])
    for _ in range(20):
        VL = np.array([1.0, 0, 0, 0, 1.0]) * (1 + 0.1 * rng.uniform(-1, 1, 5))
        VR = np.array([1.0, 0, 0, 0, 1.0]) * (1 + 0.1 * rng.uniform(-1, 1, 5))
        VL[1:4] = 3.0 * n + 0.1 * rng.normal(size=3)
        VR[1:4] = 3.0 * n + 0.1 * rng.normal(size=3)
        S = n * 0.5
        got = oracle.roe_flux(P, VL, VR, S)
        ref = physical_flux(VL, S)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_stationary_contact():
    """u = 0 on both sides, equal pressure, different density: the exact
    Riemann solution is the contact at rest, flux (0, p n, 0)."""
    P = default_params(harten=0.1)
    S = np.array([0.3, 0.4, -0.2])
    A = np.linalg.norm(S)
    VL = np.array([1.4, 0.0, 0.0, 0.0, 0.9])
    VR = np.array([0.3, 0.0, 0.0, 0.0, 0.9])
    got = oracle.roe_flux(P, VL, VR, S)
    ref = np.array([0.0, 0.9 * S[0] / A * A, 0.9 * S[1] / A * A, 0.9 * S[2] / A * A, 0.0])
    assert np.allclose(got, ref, rtol=1e-15, atol=1e-16)


def test_mirror_symmetry():
    """F^(V_L, V_R, n) = -F^(V_R, V_L, -n): the same face seen from the other side."""
    rng = np.random.default_rng(4)
    for harten, fix_all in ((0.0, 0), (0.1, 0), (0.1, 1)):
        P = default_params(harten=harten, fix_all=fix_all)
        for _ in range(30):
            VL, VR = rand_state(rng), rand_state(rng)
            S = rng.normal(size=3)
            a = oracle.roe_flux(P, VL, VR, S)
            b = oracle.roe_flux(P, VR, VL, -S)
            assert np.allclose(a, -b, rtol=1e-13, atol=1e-14 * np.abs(a).max())


def test_dissipation_sign():
    """A jump in density alone (a pure entropy wave moving right) must be
    upwinded: the mass flux is rho_L V_n (from the left), not the average."""
    P = default_params(harten=0.0)
    VL = np.array([1.0, 0.5, 0.0, 0.0, 1.0])
    VR = np.array([0.5, 0.5, 0.0, 0.0, 1.0])
    got = oracle.roe_flux(P, VL, VR, [1.0, 0.0, 0.0])
    assert got[0] == pytest.approx(1.0 * 0.5, rel=1e-14)


# ---------------------------------------------------------------- limiters ---

@pytest.mark.parametrize("lim", [1, 2])
def test_limiter_identities(lim):
    P = default_params(limiter=lim, va_delta2=0.0)
    rng = np.random.default_rng(5)
    for _ in range(100):
        b = rng.normal()
        # Psi(1) = 1
        assert oracle.limited(P, b, b) == pytest.approx(b, rel=1e-15)
        a = rng.normal()
        # Psi(r)/r = Psi(1/r)  <=>  Psi(a/b) b = Psi(b/a) a
        assert oracle.limited(P, a, b) == pytest.approx(oracle.limited(P, b, a), rel=1e-14, abs=1e-300)


def test_van_leer_closed_forms():
    P = default_params(limiter=1)
    rng = np.random.default_rng(6)
    for _ in range(100):
        a, b = rng.normal(size=2)
        got = oracle.limited(P, a, b)
        if a * b <= 0:
            assert got == 0.0                       # Psi(r) = 0 for r <= 0
        else:
            assert got == pytest.approx(2 * a * b / (a + b), rel=1e-14)  # harmonic mean
    # Psi -> 2 as r -> infinity
    assert oracle.limited(P, 1e12, 1.0) == pytest.approx(2.0, rel=1e-11)
    # zero denominator guard: exactly zero slope
    assert oracle.limited(P, 1.0, 0.0) == 0.0
    assert oracle.limited(P, 0.0, 0.0) == 0.0


def test_van_albada_closed_form():
    P = default_params(limiter=2, va_delta2=0.0)
    rng = np.random.default_rng(7)
    for _ in range(100):
        a, b = rng.normal(size=2)
        r = a / b
        psi = (r * r + r) / (1 + r * r)
        assert oracle.limited(P, a, b) == pytest.approx(psi * b, rel=1e-12, abs=1e-15)


# ------------------------------------------------------------------ MUSCL ---

def test_muscl_first_order_when_eps_zero():
    P = default_params(eps=0.0)
    L, R = oracle.muscl(P, [0.3, 1.1, 2.5, 2.0])
    assert (L, R) == (1.1, 2.5)


@pytest.mark.parametrize("kappa", [-1.0, 0.0, 1.0 / 3.0, 1.0])
@pytest.mark.parametrize("lim", [0, 1, 2])
def test_muscl_exact_for_linear_data(kappa, lim):
    P = default_params(kappa=kappa, limiter=lim, va_delta2=0.0)
    a, s = 0.7, 0.25
    v = [a + s * x for x in (-1, 0, 1, 2)]
    L, R = oracle.muscl(P, v)
    assert L == pytest.approx(a + 0.5 * s, rel=1e-15)
    assert R == pytest.approx(a + 0.5 * s, rel=1e-15)


def test_muscl_van_leer_kappa_minus_one_is_harmonic_slope():
    """eps=1, kappa=-1: V^L = V_i + 1/2 * 2 D- D+ / (D- + D+) (van Leer 1979)."""
    P = default_params(eps=1.0, kappa=-1.0, limiter=1)
    rng = np.random.default_rng(8)
    for _ in range(50):
        v = np.cumsum(rng.uniform(0.1, 1.0, size=4))
        dm, d0 = v[1] - v[0], v[2] - v[1]
        L, _ = oracle.muscl(P, v)
        assert L == pytest.approx(v[1] + dm * d0 / (dm + d0), rel=1e-14)


def test_muscl_extremum_is_first_order():
    """At a local extremum the van Leer slopes vanish: V^L = V_i, V^R = V_{i+1}."""
    P = default_params(limiter=1)
    L, R = oracle.muscl(P, [0.0, 1.0, 0.5, 2.0])
    assert L == 1.0 and R == 0.5


def test_primitive_recovery():
    """Primitive recovery (Section 2: V from Q) against facts fixed outside
    the oracle: it inverts the seeded generators' own conserved map
    (cases.prim_to_cons, rho E = p/(gamma-1) + rho |u|^2/2) on random states;
    a gas at rest has p = (gamma - 1) rho E; and for the inflow of
    the paper's inlet table (Mach 4, 12270 Pa, 217 K, air with R = 287) the
    recovered state gives the textbook sound speed sqrt(gamma R T) = 295.3 m/s
    and the Mach number 4."""
    import cases
    rng = np.random.default_rng(31)
    for _ in range(200):
        V = rand_state(rng)
        q = cases.prim_to_cons(V.reshape(5, 1)).ravel()
        W = oracle.cons_to_prim(q)
        assert np.allclose(W, V, rtol=1e-13, atol=1e-15 * np.abs(V).max())
    W = oracle.cons_to_prim(np.array([1.3, 0.0, 0.0, 0.0, 2.5]))
    assert W[4] == pytest.approx((1.4 - 1.0) * 2.5, rel=1e-15) and (W[1:4] == 0.0).all()
    R, T, p = 287.0, 217.0, 12270.0
    rho = p / (R * T)
    c = np.sqrt(1.4 * R * T)
    assert c == pytest.approx(295.3, abs=0.05)
    V = np.array([rho, 4.0 * c, 0.0, 0.0, p])
    W = oracle.cons_to_prim(cases.prim_to_cons(V.reshape(5, 1)).ravel())
    assert np.sqrt(1.4 * W[4] / W[0]) == pytest.approx(c, rel=1e-13)
    assert W[1] / np.sqrt(1.4 * W[4] / W[0]) == pytest.approx(4.0, rel=1e-13)


# ------------------------------------------------- flux-vector splittings ---

FVS = [1, 2]   # van Leer, Steger-Warming (Section 2 lists both beside Roe)


@pytest.mark.parametrize("flux", FVS)
def test_fvs_consistency(flux):
    """F+(V) + F-(V) = F(V): each splitting of Section 2's normal flux
    sums back to it, subsonic and supersonic."""
    rng = np.random.default_rng(20 + flux)
    P = default_params(flux=flux)
    for _ in range(60):
        V = rand_state(rng)
        V[1:4] *= rng.choice([0.3, 1.0, 4.0])          # subsonic and supersonic
        S = rng.normal(size=3) * 0.05
        got = oracle.face_flux(P, V, V, S)
        ref = physical_flux(V, S)
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("flux", FVS)
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_fvs_supersonic_upwinding(flux, sign):
    V0, _ = dimensional_state("inlet_2d")              # Mach 4, Section 8.1 table
    rng = np.random.default_rng(30 + flux)
    P = default_params(flux=flux)
    S = np.array([0.02, 0.0, 0.0])
    for _ in range(20):
        VL = V0 * (1 + 0.05 * rng.uniform(-1, 1, size=5))
        VR = V0 * (1 + 0.05 * rng.uniform(-1, 1, size=5))
        VL[1:4] *= sign
        VR[1:4] *= sign
        got = oracle.face_flux(P, VL, VR, S)
        ref = physical_flux(VL if sign > 0 else VR, S)
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("flux", FVS)
def test_fvs_mirror_symmetry(flux):
    rng = np.random.default_rng(40 + flux)
    P = default_params(flux=flux)
    for _ in range(40):
        VL, VR = rand_state(rng), rand_state(rng)
        S = rng.normal(size=3)
        a = oracle.face_flux(P, VL, VR, S)
        b = oracle.face_flux(P, VR, VL, -S)
        assert np.allclose(a, -b, rtol=1e-13, atol=1e-14 * np.abs(a).max())


def test_van_leer_splitting_is_continuous_at_sonic_points():
    """van Leer's split fluxes join the full flux continuously at M = +-1:
    the face flux just below and just above a sonic state agrees to O(dM)."""
    P = default_params(flux=1)
    c = np.sqrt(1.4)
    for M in (1.0, -1.0):
        lo = np.array([1.0, (M - 1e-7) * c, 0, 0, 1.0])
        hi = np.array([1.0, (M + 1e-7) * c, 0, 0, 1.0])
        S = [1.0, 0.0, 0.0]
        fl = oracle.face_flux(P, lo, lo, S)
        fh = oracle.face_flux(P, hi, hi, S)
        assert np.allclose(fl, fh, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("flux", FVS)
def test_fvs_dissipative_for_a_density_jump(flux):
    """A subsonic rightward entropy wave: the upwind splittings move the mass
    flux from the central average towards the upstream (left) state."""
    P = default_params(flux=flux)
    VL = np.array([1.0, 0.5, 0.0, 0.0, 1.0])
    VR = np.array([0.5, 0.5, 0.0, 0.0, 1.0])
    got = oracle.face_flux(P, VL, VR, [1.0, 0.0, 0.0])
    central = 0.5 * (1.0 * 0.5 + 0.5 * 0.5)
    assert got[0] > central + 0.1 * (0.5 - central)
