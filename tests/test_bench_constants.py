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


RATES = {"fp64_fma": 5.0e11, "fp64_add": 5.0e11, "fp64_mul": 5.0e11, "fp64_rcp": 6.0e10, "fp64_sqrt": 6.0e10,
         "fp32_fma": 3.3e13, "df64_add": 3.0e12, "df64_mul": 4.5e12, "df64_div": 1.2e12, "df64_sqrt": 1.3e12,
         "df64_abs": 1.6e13}


def test_alu_peaks_come_from_measured_rates():
    """binary64: an FMA counts two operations; double-float: the face's
    operation mix at the measured rate of each operation (harmonic mean
    weighted by the oracle's counts)."""
    p, how = bench.alu_peak("fp64", RATES)
    assert p == 1.0e12 and how.startswith("measured")
    p, how = bench.alu_peak("df64", RATES)
    n = sum(bench.FACE_OPS.values())
    t = (153 / 3.0e12 + 162 / 4.5e12 + 50 / 1.2e12 + 3 / 1.3e12 + 23 / 1.6e13)
    assert abs(p - n / t) < 1e-6 * p and how.startswith("measured")
    # a mix can run no faster than its fastest operation nor slower than its slowest
    assert 1.2e12 < p < 1.6e13
    assert bench.nominal_alu_peak("fp64") == 1.25e12
    assert 3.0e12 < bench.nominal_alu_peak("df64") < 4.5e12


def test_field_errors_are_plain_relative_linf():
    import numpy as np
    b = np.arange(1.0, 11.0).repeat(3)
    a = b.copy()
    a[4] += 0.5                    # variable 0: max |b| = 2
    a[20] -= 1.0                   # variable 3: max |b| = 8
    e = bench.field_errors(a, b)
    assert e[0] == 0.25 and e[3] == 1.0 / 8.0 and e[1] == e[2] == e[4] == 0.0


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
    prec = next(p for p in ("fp64", "df64", "fp32flux") if p in t)
    r = bench.roofline(mms, prec, [1e-3] * 4, 0.0, True, peaks, "test", t, RATES)
    assert r["traffic"] == t[prec]
    r = bench.roofline(other, prec, [1e-3] * 4, 0.0, True, peaks, "test", t, RATES)
    assert r["traffic"] is None
    for name, forms in t.get("workloads", {}).items():
        other.name = name
        for prec, v in forms.items():
            if prec in ("fp64", "df64", "fp32flux"):
                r = bench.roofline(other, prec, [1e-3] * 4, 0.0, True, peaks, "test", t, RATES)
                assert r["traffic"] == v
