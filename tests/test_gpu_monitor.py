"""The residual monitor (fv_set_monitor / fv_monitor_norms) through the C ABI.

RK stage 1 records the norms of the residual it computes, R(Q^(0)): they
must equal the oracle's norms of the residual of the state the step starts
from (to 1e-12 of the terms' scale for the binary64 and double-float forms,
1e-5 for the binary32 flux form, as the residual parity tests measure R,
which cancels far below its terms) and the separate entry point's norms of
the same state (relative 1e-12 in every form: the same residual, reduced in
another order and arithmetic), with and without graph replay, on one block,
on a split multi-block problem and with the viscous terms.
"""
import numpy as np
import pytest

import cases
import oracle
from test_gpu_parity import TOL_RES_NS as TOL_RES, flux_scale, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp64", "df64", "fp32flux"]
CASES = {
    "mms": lambda: cases.mms_3d((37, 21, 11), curvilinear=True),
    "split": lambda: cases.split_problem_i(cases.mms_periodic_3d(15, curvilinear=True), [5, 9]),
    "ns": lambda: cases.mms_periodic_3d((19, 14, 11), curvilinear=True, visc=1, mu=0.05),
}


def close(a, b, tol):
    return np.all(np.abs(a - b) <= tol * np.abs(b))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_monitor_records_the_step_start_residual(prec, case):
    pb = CASES[case]()
    o = oracle.Oracle(pb)
    q0 = o.fill_ghosts(pb.q.copy())
    l2_o, linf_o = o.norms(o.residual(q0))
    atol = TOL_RES[prec] * flux_scale(o, q0)
    s = solver(pb, prec)
    s.set_monitor(True)
    for use_graph in (False, True):
        l2_ref, linf_ref = s.residual_norms(0)      # the state this step starts from
        s.rk_step(pb.dt, use_graph=use_graph)
        l2, linf = s.monitor_norms()
        assert close(l2, l2_ref, 1e-12) and close(linf, linf_ref, 1e-12)
        if not use_graph:
            assert np.all(np.abs(l2 - l2_o) <= atol) and np.all(np.abs(linf - linf_o) <= atol)
    s.close()


def test_monitor_off_or_not_run_is_an_error():
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d(8, curvilinear=True)
    s = solver(pb, "df64")
    with pytest.raises(fv.FvError) as e:
        s.monitor_norms()
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    s.set_monitor(True)
    with pytest.raises(fv.FvError) as e:
        s.monitor_norms()                            # no monitored stage yet
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    s.rk_stage(2, pb.dt)                             # not stage 1: records nothing
    with pytest.raises(fv.FvError) as e:
        s.monitor_norms()
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    s.rk_stage(1, pb.dt)
    s.monitor_norms()
    s.set_monitor(False)
    s.rk_step(pb.dt, use_graph=True)
    with pytest.raises(fv.FvError) as e:
        s.monitor_norms()
    assert e.value.code == fv.FV_ERR_INVALID_ARG
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_monitor_flags_nonfinite(prec):
    import paper_2012_02925_gb300 as fv
    pb = cases.mms_3d(8, curvilinear=True)
    q = pb.q.copy()
    q[((3 + 2) * 12 + (3 + 2)) * 12 + (3 + 2)] = np.nan  # density of interior cell (3,3,3)
    s = solver(pb, prec)
    s.set_state(torch.from_numpy(q).cuda())
    s.set_monitor(True)
    s.rk_step(pb.dt, use_graph=False)
    with pytest.raises(fv.FvError) as e:
        s.monitor_norms()
    assert e.value.code == fv.FV_ERR_NONFINITE
    s.close()
