"""The benchmark's algorithmic operation count per face is the oracle's own
count (op-counting scalar), so the ALU roofline uses the method's arithmetic,
not the kernel's."""
import bench
import oracle
from cases.core import default_params


def test_face_op_count_matches_oracle():
    c = oracle.face_opcount(default_params())
    for k, v in bench.FACE_OPS.items():
        assert c[k] == v, (k, c[k], v)


def test_alu_peaks_are_derived_from_unit_counts():
    assert bench.alu_peak("fp64") == 1.25e12
    p = bench.alu_peak("df64")
    assert 3.0e12 < p < 4.5e12


def test_viscous_face_op_count_matches_oracle():
    c = oracle.viscous_opcount(default_params(visc=1, mu=0.05))
    for k, v in bench.VISC_FACE_OPS.items():
        assert c[k] == v, (k, c[k], v)


def test_traffic_applies_to_its_own_workload_and_sources_only():
    """The committed DRAM traffic is attached to the roofline only for the
    workload it was captured on and while the stage kernel's sources hash to
    the captured value."""
    import cases
    t = bench.load_traffic()
    if not t:                      # sources changed since the capture
        return
    assert t["kernel_hash"] == bench.kernel_hash()
    mms = cases.mms_3d(8, curvilinear=True)
    mms.name = t["workload"]
    other = cases.mms_3d(8, curvilinear=True)
    peaks = dict(hbm_gbs=6000.0)
    r = bench.roofline(mms, "df64", [1e-3] * 4, 0.0, True, peaks, "test", t)
    assert r["traffic"] == t["df64"]
    r = bench.roofline(other, "df64", [1e-3] * 4, 0.0, True, peaks, "test", t)
    assert r["traffic"] is None
