"""The allocation-free norm entry point (fv_field_norms_noalloc) against the
allocating one (fv_residual_norms), through the C ABI.

Callers that may not allocate device memory (caching allocators, hosts
that forbid allocation after start-up, plugins) use the
allocation-free entry point; it must give the same norms.  Two calls in a row
share the library's fixed scratch array, so the second call also checks that
leftovers of the first do not leak into its result.  Named to be collected
last."""
import ctypes

import numpy as np
import pytest

import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12   # the relative tolerance of the norm parity tests


def _lib():
    import paper_2012_02925_gb300 as fv
    L = fv.load_library()
    f = L.fv_field_norms_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return fv, f


@pytest.mark.parametrize("dims", [(70, 50, 30), (24, 19, 13)])
def test_noalloc_norms_match_allocating_entry_point(dims):
    fv, f = _lib()
    pb = cases.mms_3d(dims, curvilinear=True)
    s = fv.Solver.from_problem(pb, precision="fp64")
    s.set_state(torch.from_numpy(pb.q).cuda())
    s.set_source(torch.from_numpy(pb.source[0].ravel()).cuda())
    l2_ref, linf_ref = s.residual_norms(0)            # allocating entry point
    s.exchange_ghosts(0)
    r = s.residual(0)                                 # 5 planes of n cells (one block)
    n = s.cell_count
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):                                # two calls in a row share the scratch
        out = torch.full((11,), -1.0, dtype=torch.float64, device="cuda")
        rc = f(r.data_ptr(), n, out.data_ptr(), stream)
        assert rc == fv.FV_OK
        outs.append(out.cpu().numpy())
    s.close()
    for o in outs:
        assert np.allclose(o[:5], l2_ref, rtol=TOL, atol=0.0)
        assert np.allclose(o[5:10], linf_ref, rtol=TOL, atol=0.0)
        assert o[10] == 0.0


def test_noalloc_flags_nonfinite_and_rejects_oversize():
    fv, f = _lib()
    n = 70000
    x = torch.ones(5 * n, dtype=torch.float64, device="cuda")
    x[2 * n + 12345] = float("nan")
    out = torch.zeros(11, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert f(x.data_ptr(), n, out.data_ptr(), stream) == fv.FV_OK
    o = out.cpu().numpy()
    assert o[10] == 1.0 and np.allclose(o[[0, 1, 3, 4]], 1.0) and np.allclose(o[[5, 6, 8, 9]], 1.0)
    # sizes beyond the fixed scratch are refused before any work is enqueued
    assert f(x.data_ptr(), (1 << 26) + 1, out.data_ptr(), stream) == fv.FV_ERR_INVALID_ARG
    assert f(None, n, out.data_ptr(), stream) == fv.FV_ERR_INVALID_ARG
