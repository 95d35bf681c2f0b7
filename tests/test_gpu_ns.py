"""Laminar Navier-Stokes terms on the GPU vs the CPU oracle, through the C ABI.

Viscous flux with Green's-theorem face gradients (Section 2), the edge ghost
fill it needs, ghost geometry across connections (plain, split into slabs,
and a 90-degree rotated block), the adiabatic no-slip wall, Sutherland's law,
every arithmetic form.  Tolerances as for the inviscid suite: 1e-12 (one
residual) and 1e-10 (RK stages) for the binary64 and double-float forms,
1e-5 for the binary32-flux form.
"""
import numpy as np
import pytest

import cases
import oracle
from test_gpu_parity import TOL_RES_NS as TOL_RES, rel_err_fields, rel_err_states, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp64", "df64", "fp32flux"]
TOL_STEPS = {"fp64": 1e-10, "df64": 1e-10, "fp32flux": 1e-5}
NS = dict(visc=1, mu=0.05)
SUTH = dict(visc=1, mu=0.05, sutherland=1, t_ref=0.7, s_suth=0.3)


def _ogrid_ns(nk, seed):
    pb = cases.ellipse_ogrid(40, 12, nk, perturb=0.02, seed=seed)
    pb.params.update(visc=1, mu=0.5, r_gas=287.0, sutherland=1, t_ref=273.15, s_suth=110.4)
    pb.bcs = [cases.BCPatch(p.block, p.face, p.lo, p.hi,
                            cases.BC_NOSLIP_WALL if p.kind == cases.BC_SLIP_WALL else p.kind, p.state)
              for p in pb.bcs]
    return pb


CASES = {
    "mms_periodic": lambda: cases.mms_periodic_3d((19, 14, 11), curvilinear=True, **NS),
    "mms_sutherland": lambda: cases.mms_periodic_3d(12, curvilinear=True, **SUTH),
    "mms_fixed_ghosts": lambda: cases.mms_3d((17, 9, 7), curvilinear=True, **NS),
    "split3": lambda: cases.split_problem_i(cases.mms_periodic_3d(15, curvilinear=True, **NS), [5, 9]),
    "rotated": lambda: cases.rotated_split_problem(cases.mms_3d(12, curvilinear=True, **NS), 5),
    "ogrid2d_noslip": lambda: _ogrid_ns(1, 4),
    "ogrid3d_noslip": lambda: _ogrid_ns(7, 5),
}


def rel_err_ghosted(a, b):
    A, B = a.reshape(5, -1), b.reshape(5, -1)
    mags = np.abs(B).max(axis=1)
    scale = [mags[0], mags[1:4].max(), mags[1:4].max(), mags[1:4].max(), mags[4]]
    return max(np.abs(A[v] - B[v]).max() / scale[v] for v in range(5))


@pytest.mark.parametrize("case", sorted(CASES))
def test_ghost_and_edge_fill(case):
    pb = CASES[case]()
    o = oracle.Oracle(pb)
    ref = o.fill_ghosts(pb.q.copy())
    s = solver(pb, "fp64")
    s.exchange_ghosts(0)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_ghosted(got, ref) <= 1e-13


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_residual(prec, case):
    pb = CASES[case]()
    o = oracle.Oracle(pb)
    q = o.fill_ghosts(pb.q.copy())
    ref = o.residual(q)
    s = solver(pb, prec)
    s.exchange_ghosts(0)
    r = s.residual(0).cpu().numpy()
    s.close()
    assert rel_err_fields(r, ref, o, q) <= TOL_RES[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", ["mms_periodic", "split3", "ogrid3d_noslip"])
def test_rk_steps(prec, case):
    pb = CASES[case]()
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 8)
    s = solver(pb, prec)
    s.rk_step(pb.dt, use_graph=False)
    s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_states(got, ref, o) <= TOL_STEPS[prec]


@pytest.mark.parametrize("prec,tile", [("fp64", 3), ("df64", 8), ("df64", 2), ("fp32flux", 5), ("fp32flux", 7)])
def test_tile_shapes(prec, tile):
    pb = cases.mms_periodic_3d((37, 13, 9), curvilinear=True, **NS)
    o = oracle.Oracle(pb)
    q = o.fill_ghosts(pb.q.copy())
    ref = o.residual(q)
    s = solver(pb, prec, tile=tile, kchunk=3)
    s.exchange_ghosts(0)
    r = s.residual(0).cpu().numpy()
    s.close()
    assert rel_err_fields(r, ref, o, q) <= TOL_RES[prec]


def test_viscous_part_is_not_negligible_in_the_tests():
    """Guard for the suite itself: on the cases above the viscous part of R
    is a sizeable fraction of R (a wrong viscous term could not hide under
    the tolerances)."""
    pb = CASES["mms_periodic"]()
    o = oracle.Oracle(pb)
    R1 = o.residual(o.fill_ghosts(pb.q.copy()))
    pe = cases.mms_periodic_3d((19, 14, 11), curvilinear=True, visc=0)
    oe = oracle.Oracle(pe)
    R0 = oe.residual(oe.fill_ghosts(pe.q.copy()))
    src_diff = np.concatenate([(s1 - s0).ravel() for s1, s0 in zip(pb.source, pe.source)])
    vol = o.metrics[0][3].ravel()
    visc_part = (R1 - R0) + src_diff * np.tile(vol, 5)
    assert np.abs(visc_part).max() > 1e-3 * np.abs(R1).max()


def test_adjoint_refuses_viscous_handles():
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_periodic_3d(8, curvilinear=True, **NS)
    s = solver(pb, "fp64")
    lam = torch.zeros(s.field_size, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError) as e:
        s.adjoint_vjp(1, pb.dt, torch.from_numpy(pb.q).cuda(), lam, torch.zeros_like(lam), torch.zeros_like(lam))
    assert e.value.code == fv.FV_ERR_UNSUPPORTED
    s.close()
