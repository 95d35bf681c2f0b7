"""Pins of the oracle's whole-residual and RK behaviour.

Invariants fixed by the mathematics of the finite-volume method (Section 2,
Eq. (governing)): free-stream preservation on a curvilinear grid (closed cell
surfaces), discrete conservation on periodic domains, second-order truncation
error under a manufactured solution, second-order convergence of a moving
isentropic vortex, the Runge-Kutta amplification polynomial, geometric
identities of the metrics, ghost-exchange consistency, multi-block
equivalence (the paper's parallel-vs-serial check, Section 8) and the
dual-number JVP against central differences.
"""
import math

import numpy as np
import pytest

import cases
import oracle
from cases.core import default_params


def flux_scale(o: oracle.Oracle, q):
    """Typical magnitude of one face flux: max |F(V)| * max |S|."""
    Smax = max(np.sqrt((m[0] ** 2).sum(0)).max() for m in o.metrics)
    V = [oracle.cons_to_prim(x) for x in np.stack([a.reshape(5, -1)[:, 0] for a in o.interior(q)])]
    Fmax = max(abs(v[0]) * (abs(v[1]) + 1) + abs(v[4]) for v in V)
    return Smax * max(Fmax, 1.0)


# ---------------------------------------------------------------- metrics ---

def test_metrics_cartesian_from_nodes_match_spacing():
    n = 6
    b, _ = cases.workloads._mms_block(n, curvilinear=False, amp=0.0)
    nodes = cases.perturbed_nodes(n, n, n, amp=0.0)
    pb = cases.Problem([cases.BlockDesc(n, n, n, nodes)], [], 3, np.zeros(cases.packed_size([b])))
    pb.params = default_params()
    o = oracle.Oracle(pb)
    Sxi, Seta, Szeta, vol = o.metrics[0]
    h = 1.0 / n
    assert np.allclose(Sxi[0], h * h, rtol=1e-13) and np.allclose(Sxi[1:], 0, atol=1e-18)
    assert np.allclose(Seta[1], h * h, rtol=1e-13) and np.allclose(Seta[[0, 2]], 0, atol=1e-18)
    assert np.allclose(Szeta[2], h * h, rtol=1e-13) and np.allclose(Szeta[:2], 0, atol=1e-18)
    assert np.allclose(vol, h ** 3, rtol=1e-13)


def test_metrics_affine_volume_and_closure():
    """Affine maps keep faces planar: every volume is |det A| h^3; and on any
    grid the six outward face vectors of a cell sum to zero."""
    n = 5
    A = np.array([[1.0, 0.2, 0.1], [-0.1, 0.9, 0.3], [0.05, -0.2, 1.1]])
    base = cases.perturbed_nodes(n, n, n, amp=0.0)
    nodes = base @ A.T
    pb = cases.Problem([cases.BlockDesc(n, n, n, np.ascontiguousarray(nodes))], [], 3, np.zeros(1))
    pb.params = default_params()
    o = oracle.Oracle(pb)
    vol = o.metrics[0][3]
    assert np.allclose(vol, abs(np.linalg.det(A)) / n ** 3, rtol=1e-12)
    wavy = cases.mms_3d(7, curvilinear=True, with_source=False)
    o = oracle.Oracle(wavy)
    Sxi, Seta, Szeta, vol = o.metrics[0]
    close = (Sxi[:, :, :, 1:] - Sxi[:, :, :, :-1]) + (Seta[:, :, 1:, :] - Seta[:, :, :-1, :]) \
        + (Szeta[:, 1:, :, :] - Szeta[:, :-1, :, :])
    assert np.abs(close).max() < 1e-17
    assert (vol > 0).all()


# ------------------------------------------------------------- invariants ---

@pytest.mark.parametrize("lim", [1, 2])
def test_free_stream_preservation_curvilinear(lim):
    pb = cases.uniform_3d(12, curvilinear=True, limiter=lim)
    o = oracle.Oracle(pb)
    R = o.residual(pb.q.copy())
    assert np.abs(R).max() <= 1e-13 * flux_scale(o, pb.q)


def test_conservation_periodic_vortex():
    pb = cases.vortex_2d(32)
    o = oracle.Oracle(pb)
    q = o.exchange(pb.q.copy())
    R = o.residual(q).reshape(5, -1)
    scale = flux_scale(o, q)
    # every interior face is counted once with + and once with -
    assert np.abs(R.sum(axis=1)).max() <= 1e-13 * scale
    # and the total of Omega*Q is invariant across a full RK step
    vol = o.metrics[0][3].ravel()
    q1 = o.run(q, pb.dt, 4)
    m0 = (o.interior(q)[0].reshape(5, -1) * vol).sum(axis=1)
    m1 = (o.interior(q1)[0].reshape(5, -1) * vol).sum(axis=1)
    assert np.allclose(m0, m1, rtol=1e-13, atol=1e-13)


def test_conservation_periodic_3d_curvilinear_interior():
    """3D periodic Cartesian block with a non-uniform state: sum R = 0."""
    pb = cases.large_periodic(12, 10, 8, nbumps=3)
    o = oracle.Oracle(pb)
    q = o.exchange(pb.q.copy())
    R = o.residual(q).reshape(5, -1)
    assert np.abs(R.sum(axis=1)).max() <= 1e-13 * flux_scale(o, q)


@pytest.mark.parametrize("curv", [False, True])
def test_mms_truncation_error_second_order(curv):
    """Unlimited MUSCL (Psi = 1): the residual of the exact manufactured
    solution, R/Omega, falls as h^2 in L2 and Linf."""
    errs = []
    for n in (8, 16, 32):
        pb = cases.mms_3d(n, curvilinear=curv, limiter=0)
        o = oracle.Oracle(pb)
        tau = o.residual(pb.q.copy()).reshape(5, n, n, n) / o.metrics[0][3]
        errs.append((math.sqrt((tau ** 2).mean()), np.abs(tau).max()))
    e = np.array(errs)
    orders = np.log2(e[:-1] / e[1:])
    assert (orders > 1.9).all() and (orders < 2.2).all(), orders


def _vortex_exact_rho(n, T):
    g = 1.4
    h = 10.0 / n
    x = -5 + h * (np.arange(n) + 0.5)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ui = 0.5 * math.sqrt(g) / math.sqrt(2)
    dx = (X - ui * T + 5) % 10 - 5
    dy = (Y - ui * T + 5) % 10 - 5
    Tt = 1 - (g - 1) * 25 / (8 * g * math.pi ** 2) * np.exp(1 - dx * dx - dy * dy)
    return Tt ** (1 / (g - 1))


def test_vortex_converges_second_order():
    T = 1.0
    errs = []
    for n in (32, 64):
        pb = cases.vortex_2d(n)
        nsteps = int(math.ceil(T / pb.dt))
        o = oracle.Oracle(pb)
        q = o.run(pb.q.copy(), T / nsteps, 4 * nsteps)
        e = o.interior(q)[0][0, 0] - _vortex_exact_rho(n, T)
        errs.append(math.sqrt((e ** 2).mean()))
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_rk_amplification_polynomial():
    """Stage sequencing on R = lambda Omega Q: one 4-stage JST step multiplies
    Q by 1 + z + z^2/2 + z^3/6 + z^4/24 with z = -lambda dt; two stages of the
    2-stage scheme by 1 + z + z^2/2."""
    for M, poly in ((4, lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24),
                    (2, lambda z: 1 + z + z * z / 2)):
        pb = cases.mms_3d(4, curvilinear=True, with_source=False, n_stages=M)
        o = oracle.Oracle(pb)
        lam, dt = 0.7, 0.3
        vols = o.metrics[0][3]

        def R(q):
            return (lam * o.interior(q)[0] * vols).ravel()
        q1 = o.run(pb.q.copy(), dt, M, residual_fn=R)
        ratio = o.interior(q1)[0] / o.interior(pb.q)[0]
        assert np.allclose(ratio, poly(-lam * dt), rtol=1e-14)


# --------------------------------------------------------------- exchange ---

def _tag_state(o):
    q = np.zeros(int(o.offs[-1] + 5 * cases.core.ghosted_cells(o.blocks[-1])))
    for n, b in enumerate(o.blocks):
        v = o.block_view(q, n).reshape(cases.ghosted_shape(b))
        kk, jj, ii = np.meshgrid(np.arange(b.nk + 4) - 2, np.arange(b.nj + 4) - 2,
                                 np.arange(b.ni + 4) - 2, indexing="ij")
        v[0] = n
        v[1], v[2], v[3] = ii, jj, kk
        v[4] = -1.0
    return q


def test_exchange_periodic_closed_form():
    pb = cases.vortex_2d(8)
    o = oracle.Oracle(pb)
    q = o.exchange(_tag_state(o))
    v = q.reshape(cases.ghosted_shape(pb.blocks[0]))
    n = 8
    for d in (1, 2):
        assert (v[1, 2, 2:-2, 2 - d] == n - d).all()       # i = -d <- i = n - d
        assert (v[1, 2, 2:-2, n + 1 + d] == d - 1).all()    # i = n-1+d <- i = d-1
        assert (v[2, 2, 2 - d, 2:-2] == n - d).all()
        assert (v[2, 2, n + 1 + d, 2:-2] == d - 1).all()


def test_exchange_two_way_consistency_random_table():
    """For each two-way connection A<->B of the seeded table: if A's depth-1
    ghost next to A-interior cell a reads B-interior cell b, then B's depth-1
    ghost next to b reads a.  Also every connected ghost reads an interior
    cell of the src block at the right depth."""
    pb = cases.multiblock_batched(nblocks=10, lo=4, hi=9, seed=11)
    o = oracle.Oracle(pb)
    q = o.exchange(_tag_state(o))
    views = [o.block_view(q, n).reshape(cases.ghosted_shape(b)) for n, b in enumerate(o.blocks)]
    normal = lambda f, ext, d: -d if f % 2 == 0 else ext[f // 2] - 1 + d
    inner = lambda f, ext, d: d - 1 if f % 2 == 0 else ext[f // 2] - d
    checked = 0
    for c in pb.conns:
        A, B = pb.blocks[c.dst_block], pb.blocks[c.src_block]
        eA, eB = (A.ni, A.nj, A.nk), (B.ni, B.nj, B.nk)
        ta = [x for x in range(3) if x != c.dst_face // 2]
        for a in range(c.dst_lo[0], c.dst_hi[0]):
            for bb in range(c.dst_lo[1], c.dst_hi[1]):
                for d in (1, 2):
                    g = [0, 0, 0]
                    g[ta[0]], g[ta[1]] = a, bb
                    g[c.dst_face // 2] = normal(c.dst_face, eA, d)
                    cell = views[c.dst_block][:, g[2] + 2, g[1] + 2, g[0] + 2]
                    assert cell[0] == c.src_block
                    src = [int(cell[1]), int(cell[2]), int(cell[3])]
                    assert src[c.src_face // 2] == inner(c.src_face, eB, d)
                    assert all(0 <= src[x] < eB[x] for x in range(3))
                    if d == 1:
                        # B's ghost across the face from src reads A's cell next to g
                        gb = list(src)
                        gb[c.src_face // 2] = normal(c.src_face, eB, 1)
                        back = views[c.src_block][:, gb[2] + 2, gb[1] + 2, gb[0] + 2]
                        ai = list(g)
                        ai[c.dst_face // 2] = inner(c.dst_face, eA, 1)
                        assert back[0] == c.dst_block and [int(x) for x in back[1:4]] == ai
                        checked += 1
    assert checked > 50


# ------------------------------------------------------------ multi-block ---

def test_split_blocks_bitwise_equal():
    """Section 8's parallel-vs-serial check, in one process: the same domain
    as one block or as three i-slabs with connected faces gives the same
    residual and the same state after 8 stages, bit for bit."""
    pb = cases.mms_3d(10, curvilinear=True)
    sp = cases.split_problem_i(pb, [3, 7])
    o1, o2 = oracle.Oracle(pb), oracle.Oracle(sp)
    R1 = o1.residual(pb.q.copy()).reshape(5, 10, 10, 10)
    R2 = [r.reshape(5, 10, 10, -1) for r in np.split(o2.residual(o2.exchange(sp.q.copy())),
                                                       np.cumsum([5 * 10 * 10 * w for w in (3, 4)]))]
    assert np.array_equal(R1, np.concatenate(R2, axis=3))
    q1 = o1.run(pb.q.copy(), pb.dt, 8)
    q2 = o2.run(sp.q.copy(), sp.dt, 8)
    assert np.array_equal(o1.interior(q1)[0], np.concatenate(o2.interior(q2), axis=3))


def test_split_periodic_vortex_bitwise_equal():
    pb = cases.vortex_2d(16)
    sp = cases.split_problem_i(pb, [5, 11])
    o1, o2 = oracle.Oracle(pb), oracle.Oracle(sp)
    q1 = o1.run(pb.q.copy(), pb.dt, 8)
    q2 = o2.run(sp.q.copy(), sp.dt, 8)
    assert np.array_equal(o1.interior(q1)[0], np.concatenate(o2.interior(q2), axis=3))


def test_rotated_split_matches_to_roundoff():
    """A second block stored rotated by 90 degrees (index transform) gives
    the same residual up to rounding of its face vectors."""
    pb = cases.mms_3d(8, curvilinear=True)
    rs = cases.rotated_split_problem(pb, 3)
    o1, o2 = oracle.Oracle(pb), oracle.Oracle(rs)
    R1 = o1.residual(pb.q.copy()).reshape(5, 8, 8, 8)
    R2 = o2.residual(o2.exchange(rs.q.copy()))
    RA = R2[:5 * 8 * 8 * 3].reshape(5, 8, 8, 3)
    RB = R2[5 * 8 * 8 * 3:].reshape(5, 8, 5, 8)            # (v, k, j', i') with i' = j
    RB_orig = np.transpose(RB[:, :, ::-1, :], (0, 1, 3, 2))  # -> (v, k, j, i-3)
    got = np.concatenate([RA, RB_orig], axis=3)
    scale = np.abs(R1).max(axis=(1, 2, 3), keepdims=True)
    assert (np.abs(got - R1) / scale).max() < 1e-12


# ------------------------------------------------------------------- JVP ---

@pytest.mark.parametrize("lim,fix_all", [(2, 1), (1, 0)])
def test_jvp_matches_central_differences(lim, fix_all):
    pb = cases.mms_3d(6, curvilinear=True, limiter=lim, fix_all=fix_all)
    o = oracle.Oracle(pb)
    rng = np.random.default_rng(9)
    q = pb.q.copy()
    dq = rng.normal(size=q.shape) * np.abs(q) * 1e-2
    R, dR = o.residual_jvp(q, dq)
    assert np.array_equal(R, o.residual(q))
    h = 1e-6
    fd = (o.residual(q + h * dq) - o.residual(q - h * dq)) / (2 * h)
    assert np.abs(fd - dR).max() <= 1e-6 * np.abs(dR).max()


@pytest.mark.parametrize("flux", [1, 2])
def test_fvs_truncation_error_second_order_and_free_stream(flux):
    """The flux-vector splittings keep the scheme's properties: second-order
    truncation error under the manufactured solution (unlimited) and
    free-stream preservation on the perturbed grid."""
    errs = []
    for n in (8, 16, 32):
        pb = cases.mms_3d(n, curvilinear=True, limiter=0, flux=flux)
        o = oracle.Oracle(pb)
        tau = o.residual(pb.q.copy()).reshape(5, n, n, n) / o.metrics[0][3]
        errs.append(math.sqrt((tau ** 2).mean()))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders > 1.8).all(), orders
    pb = cases.uniform_3d(12, curvilinear=True, flux=flux)
    o = oracle.Oracle(pb)
    assert np.abs(o.residual(pb.q.copy())).max() <= 1e-13 * flux_scale(o, pb.q)
