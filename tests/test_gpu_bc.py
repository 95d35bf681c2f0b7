"""Physical boundaries on the GPU vs the CPU oracle, through the C ABI.

Ghost fill (slip wall, supersonic inflow, extrapolated outflow, farfield;
Section 2 and Section 7.2 V2/V3) and the overwritten wall / farfield face
fluxes (Section 7.2 V7), on the synthetic inlet, the 2D and 3D ellipse
O-grids (periodic cut + wall + farfield) and the uniform channel.

Tolerances: the residual and state bars of the interior parity suite
(1e-12 / 1e-10 for the binary64 and double-float forms, 1e-5 for the
binary32-flux form).  Ghost values: 1e-13 (binary64; the farfield state
goes through pow), 1e-12 (double-float: the boundary normals are stored as
binary32 pairs), 1e-6 (binary32 flux form: its normals are binary32).
"""
import numpy as np
import pytest

import cases
import oracle
from test_gpu_parity import TOL_RES, flux_scale, rel_err_fields, rel_err_states, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp64", "df64", "fp32flux"]
TOL_GHOST = {"fp64": 1e-13, "df64": 1e-12, "fp32flux": 1e-6}
TOL_STEPS = {"fp64": 1e-10, "df64": 1e-10, "fp32flux": 1e-5}

CASES = {
    "inlet": lambda: cases.inlet_2d(52, 16, perturb=0.02, seed=1),
    "ellipse2d": lambda: cases.ellipse_ogrid(72, 20, 1, perturb=0.02, seed=2),
    "ellipse3d": lambda: cases.ellipse_ogrid(40, 14, 9, perturb=0.02, seed=3),
}


def rel_err_ghosted(a, b):
    A, B = a.reshape(5, -1), b.reshape(5, -1)
    mags = np.abs(B).max(axis=1)
    scale = [mags[0], mags[1:4].max(), mags[1:4].max(), mags[1:4].max(), mags[4]]
    return max(np.abs(A[v] - B[v]).max() / scale[v] for v in range(5))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_ghost_fill(prec, case):
    pb = CASES[case]()
    o = oracle.Oracle(pb)
    ref = o.fill_ghosts(pb.q.copy())
    s = solver(pb, prec)
    s.exchange_ghosts(0)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_ghosted(got, ref) <= TOL_GHOST[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_residual_with_overwritten_boundary_faces(prec, case):
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
@pytest.mark.parametrize("case", sorted(CASES))
def test_rk_steps_with_boundaries(prec, case):
    pb = CASES[case]()
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 8)
    s = solver(pb, prec)
    s.rk_step(pb.dt, use_graph=False)
    s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_states(got, ref, o) <= TOL_STEPS[prec]


@pytest.mark.parametrize("prec,tile", [("fp64", 3), ("fp64", 9), ("df64", 1), ("df64", 8), ("df64", 10),
                                       ("fp32flux", 5), ("fp32flux", 6)])
def test_boundary_faces_in_every_tile_position(prec, tile):
    """Ragged tiles and k-chunks so that boundary faces fall on tile edges,
    chunk starts and chunk ends."""
    pb = cases.ellipse_ogrid(45, 13, 11, perturb=0.02, seed=7)
    o = oracle.Oracle(pb)
    q = o.fill_ghosts(pb.q.copy())
    ref = o.residual(q)
    s = solver(pb, prec, tile=tile, kchunk=3)
    s.exchange_ghosts(0)
    r = s.residual(0).cpu().numpy()
    s.close()
    assert rel_err_fields(r, ref, o, q) <= TOL_RES[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("supersonic", [True, False])
def test_free_stream_with_every_boundary_kind(prec, supersonic):
    pb = cases.channel_uniform(10, supersonic)
    o = oracle.Oracle(pb)
    s = solver(pb, prec)
    s.exchange_ghosts(0)
    r = s.residual(0).cpu().numpy().reshape(5, -1)
    s.close()
    fs = flux_scale(o, pb.q)
    for v in range(5):
        assert np.abs(r[v]).max() <= TOL_RES[prec] * fs.max()


def test_boundary_patch_validation_and_clearing():
    import paper_2012_02925_gb300 as fv
    pb = cases.inlet_2d(20, 8)
    s = solver(pb, "fp64")
    bad = [cases.BCPatch(0, 4, (0, 0), (20, 8), cases.BC_SLIP_WALL),                 # k face in 2D
           cases.BCPatch(0, 0, (0, 0), (9, 1), cases.BC_EXTRAPOLATE),                 # j range past nj
           cases.BCPatch(3, 0, (0, 0), (8, 1), cases.BC_EXTRAPOLATE),                 # no block 3
           cases.BCPatch(0, 0, (0, 0), (8, 1), cases.BC_FARFIELD, (0.0, 1, 0, 0, 1)),  # rho = 0
           cases.BCPatch(0, 0, (0, 0), (8, 1), 9)]                                      # unknown kind
    for p in bad:
        with pytest.raises(fv.FvError) as e:
            s.set_boundaries([p])
        assert e.value.code == fv.FV_ERR_INVALID_ARG
    # the valid set survives the failed calls; clearing leaves fixed ghosts
    s.exchange_ghosts(0)
    with_bc = s.get_state(0).cpu().numpy()
    s.set_state(torch.from_numpy(pb.q).cuda())
    s.set_boundaries([])
    s.exchange_ghosts(0)
    cleared = s.get_state(0).cpu().numpy()
    s.close()
    o = oracle.Oracle(pb)
    assert rel_err_ghosted(with_bc, o.fill_ghosts(pb.q.copy())) <= 1e-13
    assert np.array_equal(cleared, pb.q)


def test_adjoint_refuses_boundary_patches():
    import paper_2012_02925_gb300 as fv
    pb = cases.ellipse_ogrid(24, 8, 1, perturb=0.01, seed=1)
    s = solver(pb, "fp64")
    n = s.field_size
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    qin = torch.from_numpy(pb.q).cuda()
    with pytest.raises(fv.FvError) as e:
        s.adjoint_vjp(1, pb.dt, qin, lam, torch.zeros_like(lam), torch.zeros_like(lam))
    assert e.value.code == fv.FV_ERR_UNSUPPORTED
    s.close()
