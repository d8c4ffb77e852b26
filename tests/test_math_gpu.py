"""The FP64 reciprocal and square root of the sweep against CUDA's IEEE
division and square root.

The sweep divides by a^0 (Eqs. pl15, pl20, pl21, pl30) and by T and a^p_0
(Eqs. pl23, pl5) with its own reciprocal instead of IEEE division: from the
FP32 reciprocal r of x, with e = 1 - x r (about 2^-23), one step
r + r (e + e^2) of the geometric series of r / (1 - e).  The truncation error
e^3 is far below the FP64 rounding, so the result must stay within one unit
in the last place of the IEEE quotient."""
import numpy as np
import pytest

import paper_1802_04243_gb300 as sim
from paper_1802_04243_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    sim.load()


def test_reciprocal_within_one_ulp_of_ieee_division():
    rng = np.random.default_rng(11)
    mags = 10.0 ** rng.uniform(-300, 300, 200_000)
    x = np.concatenate([
        mags * rng.choice([-1.0, 1.0], mags.size),
        rng.uniform(0.5, 2.0, 100_000),                              # the typical magnitudes of a^0
        np.nextafter(1.0, 2.0) * 2.0 ** np.arange(-120, 121),        # both sides of the FP32-seed range
        np.nextafter(2.0, 1.0) * 2.0 ** np.arange(-120, 121),
        [1.0, -1.0, 2.0, 0.5, 3.0, 1.0 / 3.0, 7.0, 1e-310, -1e-310, 1e308, 2.0 ** -100, 2.0 ** 100],
    ])
    ours, ieee = sim.recip_check(x)
    assert np.all(np.isfinite(ours) == np.isfinite(ieee))
    fin = np.isfinite(ieee)
    ulps = np.abs(ours[fin] - ieee[fin]) / np.spacing(np.abs(ieee[fin]))
    print("max ulp", ulps.max(), "exact", float(np.mean(ulps == 0)))
    assert ulps.max() <= 1.0


def test_reciprocal_of_exact_cases():
    x = np.array([1.0, 2.0, 4.0, 0.25, -8.0, 2.0 ** 60, 2.0 ** -60])
    ours, ieee = sim.recip_check(x)
    assert np.array_equal(ours, ieee)                                # powers of two are exact


def test_square_root_within_one_ulp_of_ieee_sqrt():
    # Gamma = T^(1/2) (Eq. pl37): two Newton-Raphson steps for s^2 = x from
    # the FP32 reciprocal square root take its error of about 2^-22 to about
    # 2^-65, so the root must stay within one ulp of the correctly rounded one
    rng = np.random.default_rng(13)
    x = np.concatenate([
        10.0 ** rng.uniform(-300, 300, 200_000),
        rng.uniform(0.2, 20.0, 200_000),                           # the temperatures of the workloads
        np.nextafter(1.0, 2.0) * 2.0 ** np.arange(-120, 121),      # both sides of the FP32-seed range
        np.nextafter(2.0, 1.0) * 2.0 ** np.arange(-120, 121),
        np.arange(1.0, 2000.0) ** 2,                               # perfect squares
        [1.0, 2.0, 0.5, 3.0, 1e-310, 1e308, 2.0 ** -100, 2.0 ** 100, 0.0],
    ])
    ours, ieee = sim.sqrt_check(x)
    ulps = np.abs(ours - ieee) / np.spacing(np.abs(ieee))
    print("max ulp", ulps.max(), "exact", float(np.mean(ulps == 0)))
    assert ulps.max() <= 1.0
    assert np.isnan(sim.sqrt_check(np.array([-1.0]))[0][0])
