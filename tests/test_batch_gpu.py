"""Batches (sim_batch_*): one launch per kernel phase over many problems of
different sizes and parameters.  Every problem of a batch must come out
exactly as if it had been advanced alone with sim_step."""
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


def small_batch(n=5, precision=W.MIXED, implicit=True, tvd=False):
    cases = W.c5_batch(n=n, precision=precision)
    # keep the test quick: shrink every problem by 4 in each direction
    out = []
    for c in cases:
        nx, ny = c.nx // 4, c.ny // 4
        side = max(2, int(round(ny / 5.0)))
        out.append(W.channel(nx, ny, side, n_squares=len(c.rects), first_at_quarter=False, name=c.name,
                             mach_in=c.mach_in, reynolds=c.reynolds, seed=c.seed, implicit=implicit, tvd=tvd,
                             precision=precision))
    return out


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64])
@pytest.mark.parametrize("implicit,tvd", [(True, False), (False, True)])
def test_batch_equals_problems_advanced_alone(precision, implicit, tvd):
    cases = small_batch(precision=precision, implicit=implicit, tvd=tvd)
    assert len({c.nx for c in cases}) > 1                      # uneven sizes
    with sim.Batch(cases) as b:
        b.step(7)
        got = [b.fields(q) for q in range(len(cases))]
        res = [b.residuals(q)[0] for q in range(len(cases))]
    for q, c in enumerate(cases):
        with sim.Simulation(c) as s:
            s.step(7)
            ref = s.fields()
            rres, _, _ = s.residuals()
        for k in "uvpT":
            assert np.array_equal(got[q][k], ref[k]), (q, k)
        np.testing.assert_array_equal(res[q], rres)


def test_batch_fp64_matches_oracle():
    cases = small_batch(n=3, precision=W.FP64)
    with sim.Batch(cases) as b:
        b.step(10)
        got = [b.fields(q) for q in range(len(cases))]
    for q, c in enumerate(cases):
        o, _, _ = oracle.run(c, nsteps=10)
        err = max(float(np.abs(got[q][k] - o[k]).max() / np.abs(o[k]).max()) for k in "uvpT")
        assert err <= 1e-9, (q, err)


def test_tuning_keeps_the_state_and_the_results():
    cases = small_batch(n=4)
    with sim.Batch(cases) as a, sim.Batch(cases) as b:
        a.step(3)
        b.step(3)
        tx, ty, grid = b.tune()
        assert tx * ty in (128, 256) and grid >= 1
        a.step(4)
        b.step(4)                                  # replays graphs built for the tuned tiles
        for q in range(len(cases)):
            fa, fb = a.fields(q), b.fields(q)
            for k in "uvpT":
                assert np.array_equal(fa[k], fb[k]), (q, k)


@pytest.mark.parametrize("shape", [(16, 16, 0), (64, 4, 0), (128, 2, 304), (256, 1, 0), (32, 8, 152), (32, 2, 0),
                                   (32, 1, 0), (16, 4, 0)])
def test_every_tile_shape_gives_the_same_bits(shape):
    # sim_batch_set_tiles: any distribution of the positions over threads and
    # CTAs gives the bits of the default one (32 x 8, one CTA per tile)
    cases = small_batch(n=3, precision=W.FP64)
    with sim.Batch(cases) as a, sim.Batch(cases) as b:
        b.set_tiles(*shape)
        a.step(5)
        b.step(5)
        for q in range(len(cases)):
            fa, fb = a.fields(q), b.fields(q)
            for k in "uvpT":
                assert np.array_equal(fa[k], fb[k]), (q, k)


def test_set_tiles_rejects_other_shapes():
    with sim.Batch(small_batch(n=1)) as b:
        for bad in [(32, 3, 0), (8, 32, 0), (512, 1, 0), (32, 8, -1), (64, 8, 0)]:
            with pytest.raises(sim.SimError) as e:
                b.set_tiles(*bad)
            assert e.value.status == sim.SIM_EINVAL


def test_batch_rejects_mixed_loop2_lengths():
    cases = small_batch(n=2)
    cases[1] = cases[1].replace(iters=3)
    with pytest.raises(sim.SimError) as e:
        sim.Batch(cases)
    assert e.value.status == sim.SIM_EINVAL


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("plan", [(32, 8, 0, 0), (64, 4, 0, 0), (32, 4, 456, 0), (16, 16, 0, 0), (128, 2, 304, 0),
                                  (32, 1, 0, 0), (32, 4, 0, 1216), (32, 8, 0, 7)])
def test_single_problem_plans_give_the_same_bits(plan, precision):
    # sim_set_plan on one handle, on a ragged grid (37 x 29 positions) with
    # obstacles: every tile shape and CTA count, every precision, the implicit
    # upwind and explicit TVD schemes within one run
    rng = np.random.default_rng(4)
    nx, ny = 37, 29
    dx, dy = rng.uniform(0.2, 0.35, nx), rng.uniform(0.2, 0.35, ny)
    case = W.closed_box(implicit=True, tvd=False).replace(
        nx=nx, ny=ny, dx=dx, dy=dy, lx=float(dx.sum()), ly=float(dy.sum()),
        rects=[[5, 4, 12, 9], [20, 15, 24, 25]], perturb=1e-3, seed=21, precision=precision)
    with sim.Simulation(case) as a, sim.Simulation(case) as b:
        b.set_plan(*plan)
        for s in (a, b):
            s.step(3, sim.SIM_IMPLICIT)
            s.step(3, sim.SIM_EXPLICIT | sim.SIM_TVD)
        fa, fb = a.fields(), b.fields()
        ra, rb = a.residuals()[0], b.residuals()[0]
    for k in "uvpT":
        assert np.array_equal(fa[k], fb[k]), k
    np.testing.assert_array_equal(ra, rb)


def test_set_plan_rejects_other_shapes():
    with sim.Simulation(W.c1_small()) as s:
        for bad in [(32, 3, 0, 0), (8, 32, 0, 0), (512, 1, 0, 0), (32, 8, -1, 0), (32, 8, 0, -1)]:
            with pytest.raises(sim.SimError) as e:
                s.set_plan(*bad)
            assert e.value.status == sim.SIM_EINVAL


# ------------------------------------------------------- persistent step

@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("implicit,tvd", [(True, False), (False, True), (True, True)])
def test_persistent_step_equals_the_per_phase_launches(precision, implicit, tvd):
    # one cooperative kernel per step, phases separated by grid barriers, runs
    # the same phase bodies over the same tile list as the per-phase kernels
    cases = small_batch(precision=precision, implicit=implicit, tvd=tvd)
    with sim.Batch(cases) as a, sim.Batch(cases) as b:
        b.set_persistent(True)
        assert b.plan_info()[3] == 1
        a.step(6)
        b.step(6)
        assert b.plan_info()[3] == 1                # the step ran as a captured CUDA graph
        for q in range(len(cases)):
            fa, fb = a.fields(q), b.fields(q)
            ra, (rb, st) = a.residuals(q)[0], b.residuals(q)
            assert st == sim.SIM_OK
            for k in "uvpT":
                assert np.array_equal(fa[k], fb[k]), (q, k)
            np.testing.assert_array_equal(ra, rb)


def test_persistent_step_with_other_tiles_and_the_tuner():
    cases = small_batch(n=4, precision=W.FP64)
    with sim.Batch(cases) as a, sim.Batch(cases) as b:
        b.set_tiles(32, 4, 0)
        b.set_persistent(True)
        a.step(3)
        b.step(3)
        b.tune()                                   # may keep either mode; the state is restored
        a.step(3)
        b.step(3)
        for q in range(len(cases)):
            fa, fb = a.fields(q), b.fields(q)
            for k in "uvpT":
                assert np.array_equal(fa[k], fb[k]), (q, k)


def test_persistent_step_refused_with_symmetry_sides():
    cases = [W.uniform_flow(nx=48, ny=20).replace(rects=[[10, 6, 14, 12]], perturb=1e-3)]
    with sim.Batch(cases) as b:
        with pytest.raises(sim.SimError) as e:
            b.set_persistent(True)
        assert e.value.status == sim.SIM_EINVAL


def test_grid_barrier_completes_and_a_wait_that_cannot_complete_ends_with_an_error():
    # every resident CTA crosses 50 barriers; then a barrier that expects one
    # CTA more than were launched: each wait gives up after its limit, the
    # error word is set, the kernel ends, and the device stays usable
    err, ctas = sim.barrier_check(0, 50)
    assert err == 0 and ctas >= 152
    err, _ = sim.barrier_check(1, 3)
    assert err == 1
    cases = small_batch(n=2, precision=W.FP64)
    with sim.Batch(cases) as b:
        b.set_persistent(True)
        b.step(2)
        assert b.residuals(0)[1] == sim.SIM_OK
