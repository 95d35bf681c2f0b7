"""Discrete adjoint of the RK stage (fv_adjoint_vjp) through the C ABI.

* Dot-product test against the oracle's dual-number JVP of the same stage map
  (<VJP(lam), v> = <lam, JVP(v)>, relative 1e-10), on a curvilinear block with
  fixed ghosts, a periodic 2D block (transpose of the self-connections) and a
  seeded multi-block table with rotated connections.
* Central finite differences (step 1e-7 relative to each state entry) of a
  multi-stage objective through the torch.autograd chain with stage
  checkpointing (1e-6, relative to sum |g_i d_i|), on the
  van Albada / entropy-fix-everywhere setting of the adjoint workload, and
  the full-size 96^3 x 50-stage case on 20 seeded directions.
"""
import numpy as np
import pytest

import cases
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make(pb):
    import paper_2012_02925_gb300 as fv
    s = fv.Solver.from_problem(pb, precision="fp64")
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


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("m", [1, 3])
def test_dot_product_against_oracle_jvp(name, m):
    pb = PROBLEMS[name]()
    o = oracle.Oracle(pb)
    s = make(pb)
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


def _fd_check(n, nstages, ndirs, seed=7, eps=1e-7):
    from paper_2012_02925_gb300.autograd import run_stages
    pb = cases.mms_3d(n, curvilinear=True, with_source=False, limiter=2, fix_all=1)
    o = oracle.Oracle(pb)
    s = make(pb)
    J = objective(pb, o)
    q0 = torch.from_numpy(pb.q).cuda()
    mask = torch.from_numpy(interior_mask(o, pb.q)).cuda()
    x = q0.clone().requires_grad_(True)
    Jv = J(run_stages(s, x, pb.dt, nstages))
    Jv.backward()
    grad = x.grad.detach()
    rng = np.random.default_rng(seed)
    worst = 0.0
    with torch.no_grad():
        for _ in range(ndirs):
            d = torch.from_numpy(rng.uniform(-1.0, 1.0, size=pb.q.shape)).cuda() * q0.abs() * mask
            Jp = J(run_stages(s, q0 + eps * d, pb.dt, nstages)).item()
            Jm = J(run_stages(s, q0 - eps * d, pb.dt, nstages)).item()
            fd = (Jp - Jm) / (2 * eps)
            ad = float((grad * d).sum())
            # relative to the cancellation-free size of the directional
            # derivative, sum |g_i d_i|: a random direction can make
            # <g, d> itself tiny, and the central difference's error
            # (eps^2 truncation + rounding/eps) does not shrink with it
            scale = float((grad * d).abs().sum())
            worst = max(worst, abs(fd - ad) / scale)
    s.close()
    return worst


def test_autograd_chain_matches_central_differences():
    assert _fd_check(16, 10, 4) <= 1e-6


def test_adjoint_workload_full_size():
    """96^3 curvilinear block, van Albada, Harten fix on every eigenvalue,
    J = integrated pressure on the k=0 face after 50 stages, 20 directions."""
    assert _fd_check(96, 50, 20) <= 1e-6
