"""The binary64 face code's reciprocal (fv_rcp64: the hardware's approximate
reciprocal refined by one third-order step of the geometric series of
1/(1 - e)) against CUDA's IEEE 1.0 / x, and its square root (fv_sqrt64: the
hardware's approximate reciprocal square root corrected by the binomial
series of (1 - e)^(-1/2) to its e^2 term) against CUDA's IEEE sqrt(x):
within one unit in the last place over magnitudes from 1e-300 to 1e300, and
equal to it on most inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_reciprocal_within_one_ulp_of_ieee():
    from paper_2012_02925_gb300._binding import check_rcp64
    rng = np.random.default_rng(11)
    n = 1 << 22
    mag = 10.0 ** rng.uniform(-300, 300, n)
    x = mag * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # the values the face code meets: densities, sound speeds, sums near 1
    x[:1 << 20] = rng.uniform(0.01, 10.0, 1 << 20)
    out = check_rcp64(torch.from_numpy(x).cuda()).cpu().numpy()
    mine, ieee = out[:, 0], out[:, 1]
    assert np.isfinite(mine).all()
    ulps = np.abs(mine.view(np.int64) - ieee.view(np.int64))
    assert ulps.max() <= 1, int(ulps.max())
    assert (ulps == 0).mean() > 0.9


def test_square_root_within_one_ulp_of_ieee():
    from paper_2012_02925_gb300._binding import check_sqrt64
    rng = np.random.default_rng(12)
    n = 1 << 22
    x = 10.0 ** rng.uniform(-300, 300, n)
    # the values the face code meets: density ratios and squared sound speeds
    x[:1 << 20] = rng.uniform(0.01, 10.0, 1 << 20)
    # every binade's ends (the seed's error is largest near powers of two)
    e = np.arange(-990, 990, dtype=np.float64)
    x[-4 * e.size:] = np.concatenate([2.0 ** e, np.nextafter(2.0 ** e, 0), np.nextafter(2.0 ** e, np.inf),
                                      1.5 * 2.0 ** e])
    out = check_sqrt64(torch.from_numpy(x).cuda()).cpu().numpy()
    mine, ieee = out[:, 0], out[:, 1]
    assert np.array_equal(ieee, np.sqrt(x))
    assert np.isfinite(mine).all()
    ulps = np.abs(mine.view(np.int64) - ieee.view(np.int64))
    assert ulps.max() <= 1, int(ulps.max())
    # faithful, not correctly rounded: the last fused multiply-add adds a
    # rounded correction s e (3/8 e + 1/2) to s (0.875 of these inputs equal
    # to IEEE on a GB300)
    assert (ulps == 0).mean() > 0.75


def test_probe_rates_are_ordered():
    """The measured rates the roofline is graded against: positive, binary32
    FMA far above binary64 FMA (GB300 runs binary64 at 1/64 of the binary32
    rate), add = multiply = FMA in binary64, the face code's reciprocal
    faster than the compiler's IEEE one, double-float operations between
    the two precisions' FMA rates."""
    import paper_2012_02925_gb300 as fv
    r = fv.probe_alu_rates()
    assert all(v > 0 for v in r.values())
    assert r["fp32_fma"] > 30 * r["fp64_fma"]
    assert abs(r["fp64_add"] / r["fp64_fma"] - 1) < 0.1 and abs(r["fp64_mul"] / r["fp64_fma"] - 1) < 0.1
    assert r["fp64_rcp_refined"] > r["fp64_rcp"]
    assert r["fp64_sqrt_refined"] > r["fp64_sqrt"]
    for k in ("df64_add", "df64_mul", "df64_div", "df64_sqrt"):
        assert r["fp64_fma"] < r[k] < r["fp32_fma"], k
