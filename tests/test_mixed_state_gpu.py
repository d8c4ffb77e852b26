"""The FP64 state of the mixed-precision path.  Its sweep keeps u, v, T and
Gamma in FP32 only and the FP64 arrays are filled from them when the state is
read (the FP64 p and rho are its own).  Reading must not change the run, and
what is read must be what a sweep storing FP64 copies would hold: at every
position the sweep computes, the FP32 value widened exactly; everywhere else
the value the problem started with; on the outflow face the copy of its
western neighbour."""
import numpy as np
import pytest

import paper_1802_04243_gb300 as sim
import workloads as W
from paper_1802_04243_gb300 import build

pytestmark = pytest.mark.gpu

NAMES = ("u", "v", "p", "T", "rho", "gamma")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    sim.load()


def _case(implicit=True, tvd=False):
    # the 128x32 channel with its square obstacle: inflow west, outflow east,
    # walls south and north, seeded perturbation
    return W.c1_small().replace(precision=W.MIXED, implicit=implicit, tvd=tvd)


@pytest.mark.parametrize("implicit,tvd", [(True, False), (False, True)])
def test_reading_the_state_mid_run_does_not_change_the_run(implicit, tvd):
    case = _case(implicit, tvd)
    with sim.Simulation(case) as a:
        a.step(10)
        ref = a.fields(NAMES)
        rres = a.residuals()[0]
    with sim.Simulation(case) as b:
        for _ in range(5):
            b.step(2)
            b.fields(NAMES)                    # each read fills the FP64 view
            b.field_view("u")
        got = b.fields(NAMES)
        gres = b.residuals()[0]
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), k
    np.testing.assert_array_equal(gres, rres)


def test_fp64_view_holds_the_widened_fp32_values():
    case = _case()
    with sim.Simulation(case) as s:
        start = s.fields(NAMES)
        s.step(8)
        after = s.fields(NAMES)
    for k in ("u", "v", "T", "gamma"):
        a, b = start[k], after[k]
        changed = a != b
        # every value the sweep changed is an FP32 value (exactly representable)
        assert np.array_equal(b[changed], b[changed].astype(np.float32).astype(np.float64)), k
        # and most of the field is computed: the FP32 side carries the run
        assert changed.mean() > 0.8, (k, float(changed.mean()))
    # the outflow face (u at i = nx) copies its western neighbour
    u = after["u"]
    assert np.array_equal(u[:, -1], u[:, -2])
    # p and rho are the sweep's own FP64 values, not widened FP32 ones
    for k in ("p", "rho"):
        b = after[k]
        assert not np.array_equal(b, b.astype(np.float32).astype(np.float64)), k


def test_batch_and_strips_read_the_same_fp64_view():
    case = _case()
    cases = [case, case.replace(seed=case.seed + 1)]
    with sim.Simulation(case) as a:
        a.step(6)
        ref = a.fields(NAMES)
    with sim.Batch(cases) as b:
        b.step(3)
        b.fields(1, NAMES)                     # a read between steps changes nothing
        b.step(3)
        got = b.fields(0, NAMES)
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), ("batch", k)
    with sim.Strips(case, 3) as h:
        h.step(3)
        h.fields(NAMES)
        h.step(3)
        got = h.fields(NAMES)
    for k in NAMES:
        assert np.array_equal(got[k], ref[k]), ("strips", k)


@pytest.mark.parametrize("precision", [W.MIXED, W.FP64], ids=["mixed", "fp64"])
def test_fp64_view_ghosts_follow_the_symmetry_rule(precision):
    # symmetry planes south and north, an obstacle, inflow and outflow: after
    # a read the FP64 ghost rows hold the mirror of the rows inside, as the
    # FP64 sweep leaves them after its velocity update (the FP64 case checks
    # the check), and the interior matches a second read
    case = W.uniform_flow(nx=40, ny=18).replace(rects=[[9, 6, 13, 11]], perturb=1e-3, precision=precision)
    with sim.Simulation(case) as s:
        s.step(6)
        first = s.fields(NAMES)
        views = {k: s.field_view(k).cpu().numpy() for k in ("u", "v", "T", "gamma")}
        again = s.fields(NAMES)
    for k in NAMES:
        assert np.array_equal(first[k], again[k]), k
    ny = case.ny
    for k in ("T", "gamma"):
        a = views[k]                       # rows j = -2 .. ny + 1 at index j + 2
        assert np.array_equal(a[1, :case.nx + 4], a[2, :case.nx + 4]), k          # j = -1 mirrors j = 0
        assert np.array_equal(a[0, :case.nx + 4], a[3, :case.nx + 4]), k          # j = -2 mirrors j = 1
        assert np.array_equal(a[ny + 2, :case.nx + 4], a[ny + 1, :case.nx + 4]), k  # j = ny mirrors ny - 1
        assert np.array_equal(a[ny + 3, :case.nx + 4], a[ny, :case.nx + 4]), k      # j = ny + 1 mirrors ny - 2
    u = views["u"]
    assert np.array_equal(u[1], u[2]) and np.array_equal(u[0], u[3])
    v = views["v"]
    assert np.array_equal(v[1, :case.nx + 4], -v[3, :case.nx + 4])              # v(j=-1) = -v(j=1)
