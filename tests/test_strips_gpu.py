"""x-strips (sim_strips_*): one problem split into strips along x, each with
its own arrays over its owned columns and a halo, the halos exchanged once
per loop-2 iteration.  Every owned value is computed by the same kernels from
the same operands as in a whole-problem handle, so the fields and the
residuals must equal sim_create + sim_step bit for bit."""
import numpy as np
import pytest

import oracle
import paper_1802_04243_gb300 as sim
import workloads as W
from paper_1802_04243_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    sim.load()


def _compare(case, n_strips, steps, schemes=None):
    schemes = schemes or [sim.scheme_of(case.implicit, case.tvd)]
    with sim.Simulation(case) as a, sim.Strips(case, n_strips) as b:
        for sc in schemes:
            a.step(steps, sc)
            b.step(steps, sc)
        fa, fb = a.fields(("u", "v", "p", "T", "rho", "gamma")), b.fields(("u", "v", "p", "T", "rho", "gamma"))
        ra, rb = a.residuals()[0], b.residuals()[0]
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), (k, float(np.abs(fa[k] - fb[k]).max()))
    np.testing.assert_array_equal(ra, rb)
    return fa


@pytest.mark.parametrize("n_strips", [2, 3, 5])
@pytest.mark.parametrize("implicit,tvd", [(False, True), (True, False), (True, True), (False, False)])
def test_strips_equal_the_whole_problem_channel(implicit, tvd, n_strips):
    # the 128x32 channel: the square obstacle (columns 28-36) straddles the
    # boundary of the 2-strip split at column 64 only for some splits; inflow
    # west, outflow east
    case = W.c1_small().replace(implicit=implicit, tvd=tvd)
    _compare(case, n_strips, 12)


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64], ids=["fp64", "mixed", "df64"])
def test_strips_equal_the_whole_problem_every_precision(precision):
    # an obstacle across a strip boundary (columns 60-70 of 128), both schemes
    # of one run
    case = W.c1_small().replace(rects=[[60, 10, 70, 20]], precision=precision)
    _compare(case, 2, 6, [sim.SIM_EXPLICIT | sim.SIM_TVD, sim.SIM_IMPLICIT])


def test_strips_equal_the_whole_problem_walls_symmetry_nonuniform():
    # a closed box with moving walls on a non-uniform, ragged grid (61 columns
    # in 3 strips), and a box with symmetry planes on all four sides
    rng = np.random.default_rng(7)
    nx, ny = 61, 29
    dx, dy = rng.uniform(0.2, 0.35, nx), rng.uniform(0.2, 0.35, ny)
    box = W.closed_box(implicit=True, tvd=True).replace(
        nx=nx, ny=ny, dx=dx, dy=dy, lx=float(dx.sum()), ly=float(dy.sum()),
        rects=[[5, 4, 12, 9], [26, 15, 35, 25]], gx=0.01, gy=-0.02, iters=3, perturb=1e-3, seed=21)
    _compare(box, 3, 10)
    sym = W.closed_box(n=40, implicit=True, tvd=False).replace(
        side_kind=(W.SYMMETRY, W.SYMMETRY, W.SYMMETRY, W.SYMMETRY), rects=[[18, 15, 24, 22]], perturb=1e-3, seed=3)
    _compare(sym, 4, 10)


def test_strips_slip_and_jump_walls_paper_set_up():
    case = W.paper_channel(ny=40, nx=160, kn=0.05, side=8, inlet=24).replace(perturb=1e-3, seed=13)
    _compare(case, 4, 8)


def test_strips_full_size_channel_matches_the_oracle():
    # the 1024x256 channel in 8 strips, 20 steps: the whole-problem equality
    # above, and the FP64 bar against the oracle
    case = W.c2_medium()
    g = _compare(case, 8, 20)
    o, _, _ = oracle.run(case, nsteps=20, rows=True)
    for k in "uvpT":
        assert float(np.abs(g[k] - o[k]).max() / np.abs(o[k]).max()) <= 1e-9, k


def test_strips_reject_what_they_cannot_split():
    for bad, n in ((W.c1_small(), 17), (W.c1_small().replace(tol=1e-6), 2), (W.c1_small(), 0)):
        with pytest.raises(sim.SimError) as e:
            sim.Strips(bad, n)
        assert e.value.status == sim.SIM_EINVAL
