"""Discrete adjoint of the RK stage (fv_adjoint_vjp) through the C ABI.

* Dot-product test against the oracle's dual-number JVP of the same stage map
  (<VJP(lam), v> = <lam, JVP(v)>, relative 1e-10), on a curvilinear block with
  fixed ghosts, a periodic 2D block (transpose of the self-connections) and a
  seeded multi-block table with rotated connections; face sweeps in binary64
  and in double-float arithmetic (fv_set_adjoint_arith).
* Central finite differences (step 1e-7 relative to each state entry) of a
  multi-stage objective through the torch.autograd chain with stage
  checkpointing, on the van Albada / entropy-fix-everywhere setting of the
  adjoint workload, and the full-size 96^3 x 50-stage case: on directions
  that cannot cancel (d_i = sign(g_i) |q_i| on every interior cell, on a
  seeded tenth of them, and in a box at the objective's face) the plain
  |fd - ad| / |ad| <= 1e-6; on 20 seeded random directions
  d_i = U(-1, 1) |q_i|, whose <g, d> may cancel, the error relative to
  sum |g_i d_i| <= 1e-6.
* Segment recomputation (torch.utils.checkpoint over runs of steps) gives
  the plain chain's gradient bit for bit.
"""
import numpy as np
import pytest

import cases
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


ARITHS = ["fp64", "df64"]


def make(pb, arith="fp64"):
    import paper_2012_02925_gb300 as fv
    s = fv.Solver.from_problem(pb, precision="fp64")
    s.set_adjoint_arith(arith)
    s.set_state(torch.from_numpy(pb.q).cuda())
    if pb.source is not None:
        s.set_source(torch.from_numpy(np.concatenate([x.ravel() for x in pb.source])).cuda())
    return s


def oracle_stage_jvp(o, qin, v, m, dt):
    """d Q^(m) for a tangent v of Q^(m-1) (interior), ghosts via the exchange."""
    qx = o.exchange(qin.copy())
    vx = o.exchange(v.copy())
    _, dR = o.residual_jvp(qx, vx)
    out = np.empty_like(dR)
    for n, b in enumerate(o.blocks):
        vol = o.metrics[n][3].ravel()
        seg = dR[o.roffs[n]:o.roffs[n + 1]].reshape(5, -1)
        out[o.roffs[n]:o.roffs[n + 1]] = (-o.alpha[m - 1] * dt * seg / vol).ravel()
    return out


def interior_mask(o, q):
    m = np.zeros_like(q, dtype=bool)
    for n, b in enumerate(o.blocks):
        view = o.block_view(m, n).reshape(cases.ghosted_shape(b))
        view[:, 2:-2, 2:-2, 2:-2] = True
    return m


PROBLEMS = {
    "curvilinear_fixed": lambda: cases.mms_3d((14, 11, 9), curvilinear=True, limiter=2, fix_all=1),
    "vortex_periodic": lambda: cases.vortex_2d(24, limiter=2, fix_all=1),
    "multiblock_rotated": lambda: cases.multiblock_batched(nblocks=6, lo=5, hi=12, seed=8, limiter=2, fix_all=1),
    "van_leer_default": lambda: cases.mms_3d((12, 10, 8), curvilinear=True),
}


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("m", [1, 3])
def test_dot_product_against_oracle_jvp(name, m, arith):
    pb = PROBLEMS[name]()
    o = oracle.Oracle(pb)
    s = make(pb, arith)
    rng = np.random.default_rng(7)
    qin = pb.q * (1.0 + 1e-3 * rng.uniform(-1, 1, size=pb.q.shape))
    mask = interior_mask(o, qin)
    qin = np.where(mask, qin, pb.q)           # perturb the interior only: fixed ghosts stay exact
    fld = s.field_size
    for trial in range(3):
        v = np.where(mask, rng.normal(size=qin.shape) * np.abs(qin), 0.0)
        lam = rng.normal(size=fld)
        jvp = oracle_stage_jvp(o, qin, v, m, pb.dt)
        lam_in = torch.empty(fld, dtype=torch.float64, device="cuda")
        lam_q0 = torch.zeros(fld, dtype=torch.float64, device="cuda")
        s.adjoint_vjp(m, pb.dt, torch.from_numpy(qin).cuda(), torch.from_numpy(lam).cuda(), lam_in, lam_q0)
        vi = np.concatenate([x.ravel() for x in o.interior(v)])
        lhs = float(np.dot(lam_in.cpu().numpy(), vi))
        rhs = float(np.dot(lam, jvp))
        assert abs(lhs - rhs) <= 1e-10 * max(abs(rhs), 1e-300), (lhs, rhs)
        assert np.array_equal(lam_q0.cpu().numpy(), lam)
    s.close()


def objective(pb, o, dtype=torch.float64):
    """J = sum over the k=0 cells of p * |S_zeta| at the kmin face."""
    Sz = o.metrics[0][2][:, 0]                      # (3, nj, ni) face vectors at k = 0
    area = torch.from_numpy(np.sqrt((Sz ** 2).sum(0)).ravel()).cuda()
    b = pb.blocks[0]
    g = (b.nk + 4, b.nj + 4, b.ni + 4)
    gamma = pb.params["gamma"]

    def J(q):
        Q = q.view(5, *g)[:, 2, 2:-2, 2:-2].reshape(5, -1)
        p = (gamma - 1.0) * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
        return (p * area).sum()
    return J


def _fd_check(n, nstages, ndirs, arith="fp64", seed=7, eps=1e-7):
    """(worst plain relative error on non-cancelling directions, worst
    error relative to sum |g_i d_i| on random directions)."""
    from paper_2012_02925_gb300.autograd import run_stages
    pb = cases.mms_3d(n, curvilinear=True, with_source=False, limiter=2, fix_all=1)
    o = oracle.Oracle(pb)
    s = make(pb, arith)
    J = objective(pb, o)
    q0 = torch.from_numpy(pb.q).cuda()
    mask = torch.from_numpy(interior_mask(o, pb.q)).cuda()
    x = q0.clone().requires_grad_(True)
    Jv = J(run_stages(s, x, pb.dt, nstages))
    Jv.backward()
    grad = x.grad.detach()
    rng = np.random.default_rng(seed)

    def fd_and_ad(d):
        Jp = J(run_stages(s, q0 + eps * d, pb.dt, nstages)).item()
        Jm = J(run_stages(s, q0 - eps * d, pb.dt, nstages)).item()
        return (Jp - Jm) / (2 * eps), float((grad * d).sum())

    worst_plain = worst_sum = 0.0
    with torch.no_grad():
        aligned = torch.sign(grad) * q0.abs() * mask
        b = pb.blocks[0]
        box = torch.zeros((5, b.nk + 4, b.nj + 4, b.ni + 4), dtype=torch.float64, device="cuda")
        i0, j0 = int(rng.integers(2, b.ni - 4)), int(rng.integers(2, b.nj - 4))
        box[:, 2:6, j0:j0 + 4, i0:i0 + 4] = 1.0
        subset = torch.from_numpy(rng.random(pb.q.shape) < 0.1).cuda()
        for d in (aligned, aligned * subset, aligned.abs() * box.reshape(-1)):
            fd, ad = fd_and_ad(d)
            assert ad != 0.0
            worst_plain = max(worst_plain, abs(fd - ad) / abs(ad))
        for _ in range(ndirs):
            d = torch.from_numpy(rng.uniform(-1.0, 1.0, size=pb.q.shape)).cuda() * q0.abs() * mask
            fd, ad = fd_and_ad(d)
            # a random direction can make <g, d> itself tiny while the central
            # difference's error (eps^2 truncation + rounding/eps) does not
            # shrink with it: measured against sum |g_i d_i|
            worst_sum = max(worst_sum, abs(fd - ad) / float((grad * d).abs().sum()))
    s.close()
    return worst_plain, worst_sum


@pytest.mark.parametrize("arith", ARITHS)
def test_autograd_chain_matches_central_differences(arith):
    plain, rel_sum = _fd_check(16, 10, 4, arith)
    assert plain <= 1e-6 and rel_sum <= 1e-6, (plain, rel_sum)


@pytest.mark.parametrize("arith", ARITHS)
def test_adjoint_workload_full_size(arith):
    """96^3 curvilinear block, van Albada, Harten fix on every eigenvalue,
    J = integrated pressure on the k=0 face after 50 stages, 20 directions."""
    plain, rel_sum = _fd_check(96, 50, 20, arith)
    assert plain <= 1e-6 and rel_sum <= 1e-6, (plain, rel_sum)


def test_segment_recomputation_gives_the_same_gradient():
    from paper_2012_02925_gb300.autograd import run_stages
    pb = cases.mms_3d(14, curvilinear=True, with_source=False, limiter=2, fix_all=1)
    o = oracle.Oracle(pb)
    s = make(pb)
    J = objective(pb, o)
    q0 = torch.from_numpy(pb.q).cuda()
    grads = []
    for seg in (0, 2, 3):
        x = q0.clone().requires_grad_(True)
        J(run_stages(s, x, pb.dt, 22, segment=seg)).backward()
        grads.append(x.grad.detach().cpu().numpy())
    s.close()
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[0], grads[2])
