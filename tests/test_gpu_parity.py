"""CUDA library vs CPU oracle, element by element, through the C ABI.

Tolerances (relative L-infinity per variable; paper Section 8 compares
parallel and serial solutions the same way at 1e-12).  States are normalised
by the field's largest magnitude.  Residuals are normalised by the larger of
max|R| and the magnitude of the terms R sums (the largest physical normal
flux times the largest face area): on a smooth field R cancels down to the
truncation error, and rounding in any evaluation order is relative to the
terms, not to R.
  FP64 and DF64 forms: 1e-12 on one residual, 1e-10 after 100 RK stages;
  FP32-flux form: 3e-6 on one inviscid residual (1e-5 with the laminar
  terms, whose gradients amplify the primitives' rounding), and at the
  benchmark size also a bound on the plain error max|R - R_ref| / max|R_ref|
  and on its drift over 100 stages (test_gpu_fullsize.py).
Setting FVGB_PARITY_LOG=<file> makes the tests append every measured error
(both normalisations, per variable) to that file as JSON lines.
Sizes span several tiles with ragged tails in i, j and k.
"""
import json
import os

import numpy as np
import pytest

import cases
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# binary32 flux form: unit roundoff 6e-8 grown over the ~25 dependent
# operations of a face (1.7e-6 of the term scale measured at worst, on the
# 64-block batch)
TOL_RES = {"fp64": 1e-12, "df64": 1e-12, "fp32flux": 3e-6}
# laminar Navier-Stokes terms (binary32 form: 5.3e-6 measured on the 128^3
# manufactured block, see the tolerance notes of the viscous kernels)
TOL_RES_NS = {"fp64": 1e-12, "df64": 1e-12, "fp32flux": 1e-5}
TOL_RUN = {"fp64": 1e-10, "df64": 1e-10}


def log_errors(test, **kw):
    """Append measured errors to $FVGB_PARITY_LOG (JSON lines), if set."""
    path = os.environ.get("FVGB_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(dict(test=test, **kw)) + "\n")


def solver(pb, precision, **kw):
    import paper_2012_02925_gb300 as fv
    s = fv.Solver.from_problem(pb, precision=precision, **kw)
    s.set_state(torch.from_numpy(pb.q).cuda())
    if pb.source is not None:
        s.set_source(torch.from_numpy(np.concatenate([x.ravel() for x in pb.source])).cuda())
    return s


def flux_scale(o, q):
    """Per-variable magnitude of the terms a residual sums: the largest
    physical normal flux |F_v(V_c) . e_d| over cells and axis directions times
    the largest face area.  Rounding in any correct evaluation of R is relative
    to this, not to R itself, which cancels down to the truncation error for a
    manufactured solution or to zero for a free stream."""
    scales = np.zeros(5)
    smax = max(np.sqrt((m[d] ** 2).sum(0)).max() for m in o.metrics for d in range(3))
    gm1 = o.params["gamma"] - 1.0
    for qi in o.interior(q):
        rho = qi[0]
        u, v, w = qi[1] / rho, qi[2] / rho, qi[3] / rho
        p = gm1 * (qi[4] - 0.5 * rho * (u * u + v * v + w * w))
        H = (qi[4] + p) / rho
        for d, vel in enumerate((u, v, w)):
            F = (rho * vel, rho * u * vel + (d == 0) * p, rho * v * vel + (d == 1) * p,
                 rho * w * vel + (d == 2) * p, rho * H * vel)
            for x in range(5):
                scales[x] = max(scales[x], np.abs(F[x]).max())
    return scales * smax


def _fields(a, o):
    return np.concatenate([a[o.roffs[n]:o.roffs[n + 1]].reshape(5, -1) for n in range(len(o.blocks))], axis=1)


def field_errors(a, b, o, q=None):
    """Per variable, over all blocks' packed interior fields:
    (max|a-b| / max(max|b|, term scale), max|a-b| / max|b|)."""
    A, B = _fields(a, o), _fields(b, o)
    fs = flux_scale(o, q if q is not None else o.pb.q)
    term, plain = [], []
    for v in range(5):
        d = float(np.abs(A[v] - B[v]).max())
        m = float(np.abs(B[v]).max())
        scale = max(m, fs[v])
        term.append(d / scale if scale > 0 else 0.0)
        plain.append(d / m if m > 0 else (0.0 if d == 0 else float("inf")))
    return term, plain


def rel_err_fields(a, b, o, q=None):
    """max over variables of max|a-b| / max(max|b|, term scale) over all
    blocks' packed interior fields (both normalisations are logged)."""
    term, plain = field_errors(a, b, o, q)
    log_errors(os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], kind="residual", term=term, plain=plain)
    return max(term)


def rel_err_states(qa, qb, o):
    """max over variables of max|a-b| / scale; the momentum components share
    one scale (the largest momentum component), so a component that is zero
    up to rounding (a transverse momentum) is compared to the momentum
    magnitude rather than to its own noise."""
    ia = np.concatenate([x.reshape(5, -1) for x in o.interior(qa)], axis=1)
    ib = np.concatenate([x.reshape(5, -1) for x in o.interior(qb)], axis=1)
    mags = np.abs(ib).max(axis=1)
    scale = [mags[0], mags[1:4].max(), mags[1:4].max(), mags[1:4].max(), mags[4]]
    errs = [float(np.abs(ia[v] - ib[v]).max() / scale[v]) if scale[v] > 0 else 0.0 for v in range(5)]
    log_errors(os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], kind="state", err=errs)
    return max(errs)


def residual_pair(pb, precision, exchange=True, **kw):
    o = oracle.Oracle(pb)
    q = pb.q.copy()
    if exchange:
        o.exchange(q)
    r_ref = o.residual(q)
    s = solver(pb, precision, **kw)
    if exchange:
        s.exchange_ghosts(0)
    r = s.residual(0).cpu().numpy()
    s.close()
    return r, r_ref, o


PRECS = ["fp64", "df64", "fp32flux"]


@pytest.mark.parametrize("prec", PRECS)
def test_residual_vortex_2d(prec):
    r, ref, o = residual_pair(cases.vortex_2d(64), prec)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(40, 19, 13), (24, 24, 24)])
def test_residual_mms_curvilinear(prec, dims):
    r, ref, o = residual_pair(cases.mms_3d(dims, curvilinear=True), prec, exchange=False)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("opts", [dict(limiter=2, fix_all=1), dict(limiter=0), dict(kappa=1.0 / 3.0),
                                  dict(eps=0.0), dict(harten=0.0)])
def test_residual_method_options(prec, opts):
    r, ref, o = residual_pair(cases.mms_3d((20, 11, 9), curvilinear=True, **opts), prec, exchange=False)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]


SHAPES = [(p, t) for p in PRECS for t in range(1, 12) if t not in (6, 7) or p == "fp32flux"]


@pytest.mark.parametrize("prec,tile", SHAPES)
def test_every_tile_shape_residual_and_step(prec, tile):
    pb = cases.mms_3d((37, 21, 11), curvilinear=True)
    r, ref, o = residual_pair(pb, prec, exchange=False, tile=tile, kchunk=3)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]
    s = solver(pb, prec, tile=tile, kchunk=4)
    s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    ref_q = o.run(pb.q.copy(), pb.dt, 4)
    assert rel_err_states(got, ref_q, o) <= (1e-6 if prec == "fp32flux" else 1e-12)


@pytest.mark.parametrize("prec", PRECS)
def test_reruns_are_bit_equal(prec):
    """Fixed summation orders and no floating-point atomics: with many more
    tiles than persistent CTAs (the hand-out order through the device
    counter differs from launch to launch) a residual and three graph RK
    steps on seeded uneven blocks with rotated connections repeat bit for
    bit, on the same handle and on a second one."""
    pb = cases.multiblock_batched(nblocks=10, lo=12, hi=48, seed=11)
    a, b = solver(pb, prec, tile=3, kchunk=2), solver(pb, prec, tile=3, kchunk=2)
    assert a.launch()["tiles"] > a.launch()["ctas"]
    res = []
    for s in (a, a, b):
        s.exchange_ghosts(0)
        res.append(s.residual(0).cpu().numpy())
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
    for _ in range(3):
        a.rk_step(pb.dt, use_graph=True)
        b.rk_step(pb.dt, use_graph=True)
    qa, qb = a.get_state(0).cpu().numpy(), b.get_state(0).cpu().numpy()
    a.close()
    b.close()
    assert np.array_equal(qa, qb)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 2, 1), (1, 7, 5), (17, 1, 3), (2, 9, 2), (33, 9, 2)])
def test_thin_blocks_every_shape(prec, dims):
    """Blocks thinner than a tile and than the two-cell halo, one k-plane per
    tile (the binary64 slope pass then recomputes the zeta slopes below and
    above every plane): residual and one RK step against the oracle in the
    tile shapes with and without the shared slopes' two-CTA layouts."""
    pb = cases.mms_3d(dims, curvilinear=True)
    o = oracle.Oracle(pb)
    ref_q = o.run(pb.q.copy(), pb.dt, 4)
    for tile, kchunk in ((3, 1), (8, 2), (9, 1), (10, 3)):
        r, ref, _ = residual_pair(pb, prec, exchange=False, tile=tile, kchunk=kchunk)
        assert rel_err_fields(r, ref, o) <= TOL_RES[prec], (tile, kchunk)
        s = solver(pb, prec, tile=tile, kchunk=kchunk)
        s.rk_step(pb.dt, use_graph=False)
        got = s.get_state(0).cpu().numpy()
        s.close()
        assert rel_err_states(got, ref_q, o) <= (1e-6 if prec == "fp32flux" else 1e-12), (tile, kchunk)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_autotuned_launch_keeps_parity(prec):
    pb = cases.multiblock_batched(nblocks=8, lo=6, hi=40, seed=6)
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 4)
    s = solver(pb, prec)
    cfg = s.autotune(pb.dt, reps=1)
    s.set_state(torch.from_numpy(pb.q).cuda())
    s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert cfg["tiles"] > 0
    assert rel_err_states(got, ref, o) <= TOL_RUN[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_free_stream_preserved(prec):
    pb = cases.uniform_3d(20, curvilinear=True)
    o = oracle.Oracle(pb)
    s = solver(pb, prec)
    r = s.residual(0).cpu().numpy()
    s.close()
    Smax = max(np.sqrt((m[0] ** 2).sum(0)).max() for m in o.metrics)
    bound = {"fp64": 1e-13, "df64": 1e-13, "fp32flux": 1e-6}[prec]
    assert np.abs(r).max() <= bound * Smax * 2.0


@pytest.mark.parametrize("prec", PRECS)
def test_residual_multiblock_random_connections(prec):
    pb = cases.multiblock_batched(nblocks=12, lo=5, hi=21, seed=3)
    r, ref, o = residual_pair(pb, prec)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]


def test_exchange_bit_exact():
    pb = cases.multiblock_batched(nblocks=12, lo=5, hi=21, seed=4)
    o = oracle.Oracle(pb)
    rng = np.random.default_rng(0)
    q = pb.q + rng.normal(size=pb.q.shape) * 1e-3
    s = solver(pb, "fp64")
    s.set_state(torch.from_numpy(q).cuda())
    s.exchange_ghosts(0)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert np.array_equal(got, o.exchange(q.copy()))


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_100_stages_vortex(prec):
    pb = cases.vortex_2d(64)
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 100)
    s = solver(pb, prec)
    for st in range(100):
        s.rk_stage(st % 4 + 1, pb.dt)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_states(got, ref, o) <= TOL_RUN[prec]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_100_stages_mms_graph(prec):
    pb = cases.mms_3d((18, 13, 11), curvilinear=True)
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 100)
    s = solver(pb, prec)
    for _ in range(25):
        s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_states(got, ref, o) <= TOL_RUN[prec]


def test_fp32flux_one_step_close():
    pb = cases.mms_3d((18, 13, 11), curvilinear=True)
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 4)
    s = solver(pb, "fp32flux")
    s.rk_step(pb.dt, use_graph=False)
    got = s.get_state(0).cpu().numpy()
    s.close()
    # binary32 face fluxes carry ~1e-6 relative error (unit roundoff 6e-8 grown
    # over the ~100 operations of a face); one step moves Q by dt R / Omega
    assert rel_err_states(got, ref, o) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_multiblock_8_stages(prec):
    pb = cases.multiblock_batched(nblocks=10, lo=5, hi=17, seed=5)
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 8)
    s = solver(pb, prec)
    s.rk_step(pb.dt, use_graph=True)
    s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert rel_err_states(got, ref, o) <= TOL_RUN[prec]


def test_rotated_split_gpu_matches_oracle():
    pb = cases.rotated_split_problem(cases.mms_3d(12, curvilinear=True), 5)
    r, ref, o = residual_pair(pb, "fp64")
    assert rel_err_fields(r, ref, o) <= 1e-12


def test_residual_norms_match_oracle():
    pb = cases.vortex_2d(64)
    o = oracle.Oracle(pb)
    q = o.exchange(pb.q.copy())
    l2_ref, linf_ref = o.norms(o.residual(q))
    s = solver(pb, "fp64")
    l2, linf = s.residual_norms(0)
    s.close()
    assert np.allclose(l2, l2_ref, rtol=1e-12, atol=1e-300)
    assert np.allclose(linf, linf_ref, rtol=1e-12, atol=1e-300)


def test_residual_norms_flag_nonfinite():
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d(8, curvilinear=True)
    q = pb.q.copy()
    q[((3 + 2) * 12 + (3 + 2)) * 12 + (3 + 2)] = np.nan  # density of interior cell (3,3,3)
    s = solver(pb, "fp64")
    s.set_state(torch.from_numpy(q).cuda())
    with pytest.raises(fv.FvError) as e:
        s.residual_norms(0)
    assert e.value.code == fv.FV_ERR_NONFINITE
    s.close()


def test_thin_blocks_and_fixed_ghosts():
    pb = cases.mms_3d((1, 3, 5), curvilinear=True)
    r, ref, o = residual_pair(pb, "fp64", exchange=False)
    assert rel_err_fields(r, ref, o) <= 1e-12


def test_host_buffers_roundtrip():
    pb = cases.mms_3d((9, 7, 5), curvilinear=True)
    import paper_2012_02925_gb300 as fv
    s = fv.Solver.from_problem(pb, precision="fp64")
    s.set_state(pb.q)                       # host pointer
    out = np.zeros_like(pb.q)
    s.get_state(0, out=out)                 # host destination (synchronous)
    s.close()
    assert np.array_equal(out, pb.q)


def test_invalid_arguments_are_reported():
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d(6, curvilinear=True)
    bad = cases.Connection(0, 1, (0, 0), (7, 6), 0, 0, (0, 0), (1, 2))   # patch wider than the face
    with pytest.raises(fv.FvError) as e:
        fv.Solver(pb.blocks, [bad], 3, pb.params)
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    s = solver(pb, "fp64")
    with pytest.raises(fv.FvError):
        s.rk_stage(9, 0.1)
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_zero_transverse_velocity_stays_finite(prec):
    """Uniform flow along x (v = w = 0) with density bumps: the transverse
    momenta carry only rounding noise, whose tiny differences must not break
    the limiter (zero slope below 1e-30)."""
    pb = cases.large_periodic(48, 40, 32, nbumps=3)
    o = oracle.Oracle(pb)
    ref = o.run(pb.q.copy(), pb.dt, 8)
    s = solver(pb, prec)
    s.rk_step(pb.dt, use_graph=True)
    s.rk_step(pb.dt, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert np.isfinite(got).all()
    ia = np.concatenate([x.reshape(5, -1) for x in o.interior(got)], axis=1)
    ib = np.concatenate([x.reshape(5, -1) for x in o.interior(ref)], axis=1)
    for v in (0, 1, 4):
        assert np.abs(ia[v] - ib[v]).max() <= (1e-10 if prec != "fp32flux" else 1e-5) * np.abs(ib[v]).max()
    for v in (2, 3):
        assert np.abs(ia[v]).max() <= (1e-12 if prec != "fp32flux" else 1e-6) * np.abs(ib[1]).max()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("flux", [1, 2])
def test_flux_vector_splittings(prec, flux):
    """van Leer and Steger-Warming face fluxes (Section 2): residual on a
    curvilinear block with ragged tiles, Mach-2 periodic flow (supersonic and
    subsonic faces) and one RK step."""
    r, ref, o = residual_pair(cases.mms_3d((37, 21, 11), curvilinear=True, flux=flux), prec, exchange=False)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]
    pb = cases.large_periodic(40, 24, 16, nbumps=3, flux=flux)
    r, ref, o = residual_pair(pb, prec)
    assert rel_err_fields(r, ref, o) <= TOL_RES[prec]
    if prec != "fp32flux":
        o = oracle.Oracle(pb)
        refq = o.run(pb.q.copy(), pb.dt, 8)
        s = solver(pb, prec)
        s.rk_step(pb.dt, use_graph=True)
        s.rk_step(pb.dt, use_graph=True)
        got = s.get_state(0).cpu().numpy()
        s.close()
        assert rel_err_states(got, refq, o) <= TOL_RUN[prec]


def test_adjoint_refuses_other_fluxes():
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d(6, curvilinear=True, flux=1)
    s = solver(pb, "fp64")
    n = s.field_size
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError) as e:
        s.adjoint_vjp(1, pb.dt, torch.from_numpy(pb.q).cuda(), z, z.clone(), z.clone())
    assert e.value.code == fv.FV_ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_zero_time_step_leaves_the_state(prec):
    """Degenerate step: with dt = 0 every stage's update alpha dt / Omega R
    vanishes, so Q^(M) = Q^(0) bit for bit in every form (graph and plain)."""
    pb = cases.mms_3d((19, 11, 7), curvilinear=True)
    s = solver(pb, prec)
    q0 = s.get_state(0).cpu().numpy().copy()
    s.rk_step(0.0, use_graph=False)
    s.rk_step(0.0, use_graph=True)
    got = s.get_state(0).cpu().numpy()
    s.close()
    assert np.array_equal(got, q0)


def test_staged_upload_equals_direct_set_state():
    """fv_stage_state + fv_set_state_staged (the upload overlapped on another
    stream) leave exactly the state fv_set_state leaves; without a staged
    state the second call is refused."""
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d((21, 13, 9), curvilinear=True)
    s = solver(pb, "df64")
    with pytest.raises(fv.FvError) as e:
        s.set_state_staged()
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    host = torch.from_numpy(pb.q).pin_memory()
    copy = torch.cuda.Stream()
    s.stage_state(host, stream=copy.cuda_stream)
    copy.synchronize()
    s.set_state_staged()
    s.rk_step(pb.dt, use_graph=False)
    a = s.get_state(0).cpu().numpy()
    s.set_state(host)
    s.rk_step(pb.dt, use_graph=False)
    b = s.get_state(0).cpu().numpy()
    s.close()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", PRECS)
def test_changing_dt_replays_one_graph(prec):
    """CFL-style stepping: 30 distinct time steps through fv_rk_step's graph
    (dt read from a device slot at replay) keep one cached graph and give,
    bit for bit, the states of the uncaptured stage sequence; the binary64
    and double-float forms also match the oracle stepped with the same dt
    sequence."""
    pb = cases.mms_3d((19, 11, 7), curvilinear=True)
    dts = pb.dt * (0.5 + 0.5 * np.random.default_rng(3).random(30))
    a, b = solver(pb, prec), solver(pb, prec)
    for dt in dts:
        a.rk_step(float(dt), use_graph=True)
        b.rk_step(float(dt), use_graph=False)
    assert a.graph_count() == 1
    qa, qb = a.get_state(0).cpu().numpy(), b.get_state(0).cpu().numpy()
    a.close()
    b.close()
    assert np.array_equal(qa, qb)
    if prec != "fp32flux":
        o = oracle.Oracle(pb)
        q = pb.q.copy()
        for dt in dts:
            q = o.run(q, float(dt), 4)
        assert rel_err_states(qa, q, o) <= TOL_RUN[prec]


def test_graph_cache_is_bounded_by_streams():
    """One graph per stream, at most eight: stepping on ten streams evicts
    the least recently used, and every replay still steps the state."""
    pb = cases.mms_3d((13, 9, 5), curvilinear=True)
    a, b = solver(pb, "fp64"), solver(pb, "fp64")
    streams = [torch.cuda.Stream() for _ in range(10)]
    for st in streams + streams[:3]:
        st.wait_stream(torch.cuda.current_stream())
        a.rk_step(pb.dt, use_graph=True, stream=st.cuda_stream)
        torch.cuda.current_stream().wait_stream(st)
        b.rk_step(pb.dt, use_graph=False)
    torch.cuda.synchronize()
    assert a.graph_count() == 8
    qa, qb = a.get_state(0).cpu().numpy(), b.get_state(0).cpu().numpy()
    a.close()
    b.close()
    assert np.array_equal(qa, qb)
