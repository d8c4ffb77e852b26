"""Parity of the CUDA path (through the C ABI) with the FP64 reference oracle.

Error metric (per field): max |gpu - oracle| / max |oracle| over the logical
array, boundary values included.  The FP64 bar is 1e-9 after 100 steps, at
every full size (the 1024x256, 4096x1024 and 4864x1216 channels) and for
every scheme but implicit TVD.  Implicit TVD amplifies rounding differences
(see test_oracle_pins.test_rounding_sensitivity_per_scheme): it is held to
1e-9 over 20 steps, and over 100 steps to a bound set by the oracle's own
sensitivity to a 1e-14 change of its start state.  The full-size runs
compare with the oracle's row-parallel build, which gives the serial
build's bits (tests/test_oracle_rows.py).
"""
import numpy as np
import pytest

import oracle
import paper_1802_04243_gb300 as sim
import workloads as W
from discrete_checks import continuity_residual, fluid_mask
from paper_1802_04243_gb300 import build

pytestmark = pytest.mark.gpu

TOL = 1e-9
SCHEMES = [(False, False), (False, True), (True, False), (True, True)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    sim.load()


def rel_err(a, b):
    return {k: float(np.abs(a[k] - b[k]).max() / max(np.abs(b[k]).max(), 1e-300)) for k in b}


def steps_for(implicit, tvd, n):
    return min(n, 20) if (implicit and tvd) else n


def run_both(case, nsteps, start=None, rows=False):
    with sim.Simulation(case) as s:
        if start is not None:
            s.set_fields(start)
        s.step(nsteps)
        g = s.fields()
        gres, git, st = s.residuals()
        assert st == sim.SIM_OK
    o, ores, oit = oracle.run(case, start, nsteps=nsteps, rows=rows)
    return g, o, gres, ores, git, oit


def assert_parity(g, o, tol=TOL, what=""):
    e = rel_err(g, o)
    assert max(e.values()) <= tol, f"{what}: {e}"
    return e


# ------------------------------------------------------------ start state

@pytest.mark.parametrize("case", [W.c1_small(), W.closed_box(), W.uniform_flow(),
                                  W.c3_large().replace(nx=512, ny=128, rects=[[100, 40, 126, 66]])],
                         ids=["c1", "box", "uniform", "c3-like"])
def test_start_state_is_bitwise_identical(case):
    with sim.Simulation(case) as s:
        g = s.fields(("u", "v", "p", "T", "rho"))
        coef = s.coefficients()
    o = oracle.init(case)
    for k in "uvpT":
        assert np.array_equal(g[k], o[k]), k
    # rho = p/T (Eq. pl5) with the sweep's own reciprocal of T:
    # within two units in the last place of the IEEE quotient
    q = o["p"] / o["T"]
    assert np.all(np.abs(g["rho"] - q) <= 2 * np.spacing(np.abs(q)))
    oc = oracle.coefficients(case)
    for k in ("A", "B", "CT1f", "CT2f", "CT3f", "u_in", "dt"):
        assert coef[k] == pytest.approx(oc[k], rel=1e-15), k


# ------------------------------------------------------------ small cases

@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_parity_channel_128x32(implicit, tvd):
    case = W.c1_small().replace(implicit=implicit, tvd=tvd)
    n = steps_for(implicit, tvd, case.steps)
    g, o, gres, ores, git, oit = run_both(case, n)
    assert_parity(g, o, what=f"{n} steps")
    assert git == oit == case.iters
    np.testing.assert_allclose(gres, ores, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("precision", [W.FP64, W.DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_parity_box_nonuniform_moving_walls(implicit, tvd, precision):
    rng = np.random.default_rng(4)
    nx, ny = 37, 29                                  # ragged: not a multiple of the 32 x 8 tile
    dx, dy = rng.uniform(0.2, 0.35, nx), rng.uniform(0.2, 0.35, ny)
    case = W.closed_box(implicit=implicit, tvd=tvd).replace(
        nx=nx, ny=ny, dx=dx, dy=dy, lx=float(dx.sum()), ly=float(dy.sum()),
        rects=[[5, 4, 12, 9], [20, 15, 24, 25]], gx=0.01, gy=-0.02, iters=3, perturb=1e-3, seed=21,
        precision=precision)
    start = oracle.init(case)
    start["u"] += 0.03 * rng.standard_normal(start["u"].shape)
    start["v"] += 0.03 * rng.standard_normal(start["v"].shape)
    n = (df64_steps_for if precision == W.DF64 else steps_for)(implicit, tvd, 40)
    g, o, *_ = run_both(case, n, start=start)
    assert_parity(g, o)


@pytest.mark.parametrize("precision", [W.FP64, W.DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_parity_symmetry_sides_and_obstacle(implicit, tvd, precision):
    case = W.uniform_flow(nx=48, ny=20, implicit=implicit, tvd=tvd).replace(
        rects=[[10, 6, 14, 12]], perturb=1e-3, seed=8, precision=precision)
    n = (df64_steps_for if precision == W.DF64 else steps_for)(implicit, tvd, 60)
    g, o, *_ = run_both(case, n)
    assert_parity(g, o)


def test_parity_west_east_symmetry_box():
    case = W.closed_box(n=20, implicit=True, tvd=False).replace(
        side_kind=(W.SYMMETRY, W.SYMMETRY, W.WALL, W.WALL), perturb=1e-3, seed=3)
    rng = np.random.default_rng(5)
    start = oracle.init(case)
    start["v"] += 0.02 * rng.standard_normal(start["v"].shape)
    g, o, *_ = run_both(case, 50, start=start)
    assert_parity(g, o)


def test_parity_smallest_grid():
    case = W.Case(name="tiny", nx=4, ny=4, lx=1.0, ly=1.0, side_kind=(W.INFLOW, W.OUTFLOW, W.WALL, W.WALL),
                  mach_in=0.5, reynolds=20.0, perturb=1e-3)
    for implicit, tvd in SCHEMES:
        c = case.replace(implicit=implicit, tvd=tvd)
        g, o, *_ = run_both(c, 20)
        assert_parity(g, o, what=str((implicit, tvd)))


def test_parity_inflow_profile_body_force_and_hard_sphere_gas():
    ny = 24
    y = (np.arange(ny) + 0.5) / ny
    case = W.Case(name="hs", nx=40, ny=ny, lx=40 / 24, ly=1.0, gas_model=W.GAS_HARD_SPHERE_KN, kn=0.01,
                  mach_in=1.2, side_vel=(0, 0, 0.1, -0.2), side_T=(1, 1, 1.1, 0.9), gx=0.05,
                  inflow_u=0.8 * 4 * y * (1 - y), inflow_T=1 + 0.1 * y, inflow_p=np.ones(ny) * 1.05,
                  rects=[[10, 8, 14, 14]], implicit=True, tvd=False, perturb=1e-3, seed=17)
    g, o, *_ = run_both(case, 60)
    assert_parity(g, o)


def test_parity_loop2_tolerance_stop():
    case = W.c1_small().replace(implicit=True, tvd=False, iters=50, tol=1e-4)
    g, o, gres, ores, git, oit = run_both(case, 10)
    assert git == oit and 1 < git < 50
    assert_parity(g, o)


def test_restart_through_host_fields_is_bitwise():
    case = W.c1_small().replace(implicit=True, tvd=False)
    with sim.Simulation(case) as a:
        a.step(20)
        full = a.fields()
    with sim.Simulation(case) as b:
        b.step(10)
        mid = b.fields()
    with sim.Simulation(case) as c:
        c.set_fields(mid)
        c.step(10)
        again = c.fields()
    for k in "uvpT":
        assert np.array_equal(full[k], again[k]), k


def test_divergence_is_reported_and_blocks_the_handle():
    case = W.c1_small().replace(implicit=True, tvd=False, cfl=3.0)
    with sim.Simulation(case) as s:
        s.step(200)
        res, _, st = s.residuals()
        assert st == sim.SIM_EDIVERGED and not np.isfinite(res).all()
        with pytest.raises(sim.SimError) as e:
            s.step(1)
        assert e.value.status == sim.SIM_ESTATE
        start = oracle.init(case)
        s.set_fields(start)
        s.step(1)                                  # usable again after all four fields are set


def test_field_view_is_zero_copy_and_matches_host_copy():
    import torch
    case = W.c1_small()
    with sim.Simulation(case) as s:
        s.step(3)
        t = s.field_view("T")
        host = s.field("T")
        assert t.is_cuda and t.dtype == torch.float64
        assert np.array_equal(t[2:-2, 2:-2].cpu().numpy(), host)


# --------------------------------------- TVD with every Van Leer limiter zero

def _alternating_start(case, n):
    """A state in which every field alternates in sign about its mean from
    node to node, so every ratio of successive differences is negative and
    every Van Leer limiter (Eq. pl15_2) is 0."""
    s = oracle.init(case)
    jc, ic = np.mgrid[0:n, 0:n]
    ju, iu = np.mgrid[0:n, 0:n + 1]
    jv, iv = np.mgrid[0:n + 1, 0:n]
    s["T"] = 1.0 + 0.1 * (-1.0) ** (ic + jc)
    s["p"] = 1.0 + 0.05 * (-1.0) ** (ic + jc)
    s["u"][:, 1:n] = (0.2 + 0.05 * (-1.0) ** (iu + ju))[:, 1:n]
    s["v"][1:n, :] = (-0.1 + 0.05 * (-1.0) ** (iv + jv))[1:n, :]
    return s


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64], ids=["fp64", "mixed", "df64"])
@pytest.mark.parametrize("implicit", [False, True])
def test_tvd_with_every_limiter_zero_gives_the_upwind_bits(implicit, precision):
    # One loop-2 iteration of one step from the alternating state evaluates
    # every limiter (face densities, explicit terms of level n-1, coefficient
    # forms) on that state: the TVD kernels must give the upwind kernels' bits,
    # and the FP64 result the oracle's TVD result
    n = 8
    case = W.closed_box(n=n, implicit=implicit, tvd=True).replace(rects=[], iters=1, precision=precision)
    start = _alternating_start(case, n)
    out = {}
    for tvd in (True, False):
        with sim.Simulation(case.replace(tvd=tvd)) as s:
            s.set_fields(start)
            s.step(1)
            out[tvd] = s.fields()
    for k in "uvpT":
        assert np.array_equal(out[True][k], out[False][k]), k
    if precision == W.FP64:
        o, _, _ = oracle.run(case, start, nsteps=1)
        assert_parity(out[True], o, what="alternating start, TVD")


# ------------------------------------------------------------ full sizes

FULL_SIZE = {
    "c2-implicit-upwind": lambda: W.c2_medium(),
    "c2-explicit-upwind": lambda: W.c2_medium().replace(implicit=False, tvd=False),
    "c2-explicit-tvd": lambda: W.c2_medium().replace(implicit=False, tvd=True),
    "c3-implicit-upwind": lambda: W.c3_large(implicit=True),
    "c3-explicit-tvd": lambda: W.c3_large(implicit=False),
    "c4-implicit-upwind": W.c4_paper_scale,
}


@pytest.mark.parametrize("name", list(FULL_SIZE))
def test_parity_full_size_100_steps(name):
    # 100 time steps of the full-size channels (the paper-scale 4864x1216 one
    # included) from the seeded start, every field at the FP64 bar, residuals
    # of the last loop-2 iteration alike
    case = FULL_SIZE[name]()
    g, o, gres, ores, git, oit = run_both(case, 100, rows=True)
    e = assert_parity(g, o, what=f"{name}, 100 steps")
    print(name, e)
    assert git == oit == case.iters
    np.testing.assert_allclose(gres, ores, rtol=1e-6, atol=1e-12)


def _perturbed(state, rel, seed):
    rng = np.random.default_rng(seed)
    return {k: v * (1.0 + rel * rng.uniform(-1.0, 1.0, v.shape)) for k, v in state.items()}


@pytest.mark.parametrize("make", [lambda: W.c1_small(), lambda: W.c2_medium()], ids=["128x32", "1024x256"])
def test_parity_implicit_tvd_100_steps_within_the_oracles_own_sensitivity(make):
    # Implicit TVD amplifies any rounding difference (a limiter's branch flips
    # when the ratio of two near-zero differences changes sign).  Over 100
    # steps the GPU-oracle gap is bounded by how far the oracle itself moves
    # when its start state changes by 1e-14 (relative): the GPU may differ
    # from the oracle by no more than 10 times that, field by field.
    case = make().replace(implicit=True, tvd=True)
    start = oracle.init(case)
    n = 100
    g, o, *_ = run_both(case, n, start=start, rows=True)
    op, _, _ = oracle.run(case, _perturbed(start, 1e-14, 99), nsteps=n, rows=True)
    gap, sens = rel_err(g, o), rel_err(op, o)
    print("implicit TVD, 100 steps: GPU vs oracle", gap, "oracle vs perturbed oracle", sens)
    for k in "uvpT":
        assert gap[k] <= 10.0 * max(sens[k], 1e-13), (k, gap, sens)


@pytest.mark.parametrize("make", [W.c2_medium, W.c4_paper_scale], ids=["c2", "c4"])
def test_continuity_in_every_cell_at_the_loop2_fixed_point_full_size(make):
    # A property that holds at any size, checked on the GPU's own FP64 result
    # at the full sizes: with loop 2 iterated to its fixed point, every fluid
    # cell satisfies discrete continuity (what Eqs. pl23, pl24 with the
    # corrections of Eqs. pl18, pl19 solve, with the upwind fluxes of Eqs.
    # pl8-pl11), restated in numpy in tests/discrete_checks.py
    case = make()
    with sim.Simulation(case) as s:
        s.step(3)                                  # leave the start state
        start = s.fields()
    with sim.Simulation(case.replace(iters=1000, tol=1e-13)) as s:
        s.set_fields(start)
        rho0 = s.fields(("rho",))["rho"]
        s.step(1)
        g = s.fields(("u", "v", "p", "T", "rho"))
        res, it, st = s.residuals()
        coef = s.coefficients()
    assert st == sim.SIM_OK and it < 1000, (res, it)
    assert np.all(g["v"][0] == 0) and np.all(g["v"][-1] == 0)
    resid = continuity_residual(case, rho0, g["rho"], g["u"], g["v"], coef["dt"])
    scale = coef["u_in"] * case.ly / case.ny
    fluid = fluid_mask(case)
    assert np.abs(resid[fluid]).max() < 1e-10 * scale
    assert np.abs((g["rho"] - rho0)[fluid]).max() * case.lx / case.nx * case.ly / case.ny / coef["dt"] > 1e-6 * scale


# ------------------------------------------------------------ mixed precision

# Stated per-field bound of the FP32-assembly path against the FP64 oracle for
# the explicit schemes and implicit upwind (measured: <= 3e-6 after 100 steps).
# Implicit TVD amplifies rounding differences (the limiter's upwind switch in
# the coefficients depends on differences that are not small inside loop 2):
# FP32 rounding reaches ~4e-4 after 10 steps, so it has its own, looser bound.
MIXED_BOUND = 1e-5
MIXED_BOUND_IMPLICIT_TVD = 2e-3


@pytest.mark.parametrize("implicit,tvd,steps", [(False, True, 50), (False, False, 100), (True, False, 100),
                                                (True, True, 10)])
def test_mixed_precision_error_against_fp64_oracle(implicit, tvd, steps):
    case = W.c1_small().replace(implicit=implicit, tvd=tvd, precision=W.MIXED)
    with sim.Simulation(case) as s:
        start = s.fields()
        s.step(steps)
        g = s.fields()
        _, _, st = s.residuals()
    assert st == sim.SIM_OK
    o, _, _ = oracle.run(case.replace(precision=W.FP64), start, nsteps=steps)
    e = rel_err(g, o)
    print("mixed", implicit, tvd, steps, e)
    assert max(e.values()) <= (MIXED_BOUND_IMPLICIT_TVD if implicit and tvd else MIXED_BOUND), e
    assert max(e.values()) > 1e-12            # the FP32 assembly is really in use


def test_mixed_precision_1024x256_100_steps():
    case = W.c2_medium().replace(precision=W.MIXED)
    with sim.Simulation(case) as s:
        start = s.fields()
        s.step(100)
        g = s.fields()
    o, _, _ = oracle.run(case.replace(precision=W.FP64), start, nsteps=100)
    e = rel_err(g, o)
    print("mixed c2", e)
    assert max(e.values()) <= MIXED_BOUND, e


def test_mixed_and_df64_at_the_paper_scale_100_steps():
    # the bench workload (4864x1216 channel, 5.9 M cells): both added
    # precisions against the FP64 oracle after 100 steps, mixed within its
    # stated bound, double-float at the FP64 bar
    case = W.c4_paper_scale()
    o, _, _ = oracle.run(case, nsteps=100, rows=True)
    with sim.Simulation(case.replace(precision=W.MIXED)) as s:
        s.step(100)
        gm = s.fields()
    with sim.Simulation(case.replace(precision=W.DF64)) as s:
        s.step(100)
        gd = s.fields()
    em, ed = rel_err(gm, o), rel_err(gd, o)
    print("c4 mixed", em, "c4 df64", ed)
    assert max(em.values()) <= MIXED_BOUND, em
    assert max(ed.values()) <= TOL, ed


def test_mixed_start_state_matches_fp64_start_state():
    case = W.c1_small()
    with sim.Simulation(case) as a, sim.Simulation(case.replace(precision=W.MIXED)) as b:
        fa, fb = a.fields(), b.fields()
    for k in "uvpT":
        assert np.array_equal(fa[k], fb[k])


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64])
def test_step_graph_replay_matches_direct_launches(precision):
    # sim_step replays captured step graphs; with event timing on it launches
    # kernels one by one.  Both must give the same bits, for every start level
    # of the three-level rotation and when the scheme changes between calls.
    case = W.c1_small().replace(precision=precision)
    with sim.Simulation(case) as direct, sim.Simulation(case) as graph:
        direct.profile(True, timing=True)
        for scheme in (sim.SIM_IMPLICIT, sim.SIM_EXPLICIT | sim.SIM_TVD, sim.SIM_IMPLICIT):
            direct.step(4, scheme)
            graph.step(4, scheme)
        a, b = direct.fields(), graph.fields()
        n_direct = direct.profile_read()["assemble"][1]
    for k in "uvpT":
        assert np.array_equal(a[k], b[k]), k
    assert n_direct == 12 * case.iters


# ------------------------------------------------------------ double-float

# The DF64 path runs every kernel of the iteration in double-float arithmetic
# (pairs of floats, about 2^-48 relative precision per operation) and is held
# to the FP64 bar against the FP64 oracle.  Its start state is the FP64 start
# state rounded to double-float.

def df64_steps_for(implicit, tvd, n):
    # Implicit TVD amplifies rounding differences by about 1e4 over 10-20
    # steps (test_oracle_pins.test_rounding_sensitivity_per_scheme); the
    # double-float unit roundoff (2^-48) is 32 times FP64's, so its runs stop
    # at 10 steps where the FP64 runs stop at 20.
    return min(n, 10) if (implicit and tvd) else n


@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_df64_parity_channel_128x32(implicit, tvd):
    case = W.c1_small().replace(implicit=implicit, tvd=tvd, precision=W.DF64)
    n = df64_steps_for(implicit, tvd, case.steps)
    g, o, gres, ores, git, oit = run_both(case, n)
    e = assert_parity(g, o, what=f"df64 {n} steps")
    print("df64", implicit, tvd, n, e)
    assert git == oit == case.iters
    np.testing.assert_allclose(gres, ores, rtol=1e-6, atol=1e-12)


def test_df64_start_state_is_the_fp64_start_rounded():
    case = W.c1_small()
    with sim.Simulation(case) as a, sim.Simulation(case.replace(precision=W.DF64)) as b:
        fa, fb = a.fields(("u", "v", "p", "T", "rho")), b.fields(("u", "v", "p", "T", "rho"))
    for k in fa:
        rel = np.abs(fb[k] - fa[k]) / np.maximum(np.abs(fa[k]), 1e-300)
        assert rel.max() <= 2.0 ** -47, k


def test_df64_1024x256_implicit_100_steps():
    case = W.c2_medium().replace(precision=W.DF64)
    g, o, *_ = run_both(case, 100)
    e = assert_parity(g, o)
    print("df64 c2", e)


def test_df64_restart_through_host_fields_continues():
    # A DF64 state read out as FP64 and set again loses the bits beyond FP64's
    # reach only, so the continued run stays at the FP64 bar.
    case = W.c1_small().replace(implicit=True, tvd=False, precision=W.DF64)
    with sim.Simulation(case) as a:
        a.step(20)
        full = a.fields()
    with sim.Simulation(case) as b:
        b.step(10)
        mid = b.fields()
    with sim.Simulation(case) as c:
        c.set_fields(mid)
        c.step(10)
        again = c.fields()
    assert_parity(again, full, tol=1e-12)


# ------------------------------------------------- slip and jump walls (Eqs. pl38, pl39)

def slip_case(implicit, tvd, precision=W.FP64):
    # the paper's microchannel set-up (moving walls, square particle, hard-sphere
    # gas) at Kn = 0.05, where the slip velocity and the temperature jump are
    # large enough to matter at every wall and on the obstacle
    return W.paper_channel(ny=40, nx=160, kn=0.05, side=8, inlet=24, implicit=implicit, tvd=tvd).replace(
        perturb=1e-3, seed=13, precision=precision)


@pytest.mark.parametrize("precision", [W.FP64, W.DF64], ids=["fp64", "df64"])
@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_parity_slip_and_jump_walls(implicit, tvd, precision):
    case = slip_case(implicit, tvd, precision)
    n = (df64_steps_for if precision == W.DF64 else steps_for)(implicit, tvd, 40)
    g, o, gres, ores, *_ = run_both(case, n)
    e = assert_parity(g, o, what=f"slip {n} steps")
    print("slip", implicit, tvd, precision, e)
    np.testing.assert_allclose(gres, ores, rtol=1e-6, atol=1e-12)
    # the slip and jump terms are exercised: without them the fields differ
    o0, _, _ = oracle.run(case.replace(zeta_coef=0.0, tau_coef=0.0), None, nsteps=n)
    assert max(rel_err(o, o0).values()) > 1e-4


def test_mixed_precision_slip_walls_error():
    case = slip_case(True, False, W.MIXED)
    with sim.Simulation(case) as s:
        start = s.fields()
        s.step(40)
        g = s.fields()
    o, _, _ = oracle.run(case.replace(precision=W.FP64), start, nsteps=40)
    e = rel_err(g, o)
    print("mixed slip", e)
    assert max(e.values()) <= MIXED_BOUND, e


@pytest.mark.parametrize("ny", [200, 400], ids=["4032x200-1-particle", "4032x400-2-particles"])
@pytest.mark.parametrize("implicit,tvd", [(True, False), (False, True)], ids=["implicit-upwind", "explicit-tvd"])
def test_parity_paper_channel(implicit, tvd, ny):
    # the paper's own meshes (Section 4): 4032 x 200 and 4032 x 400 cells of
    # 0.05 a with one particle per 10 a of height, Kn 0.001, M 2.43
    case = W.paper_channel(ny=ny, implicit=implicit, tvd=tvd)
    g, o, *_ = run_both(case, 3)
    assert_parity(g, o)


# ------------------------------------------------- whole-state calls

def _page_locked(state, keep):
    # numpy views of page-locked copies (the library reads and writes these
    # directly from its kernels); `keep` holds the owning tensors
    import torch
    out = {}
    for k, v in state.items():
        t = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
        keep.append(t)
        out[k] = t.numpy()
    return out


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "page-locked"])
@pytest.mark.parametrize("precision", [W.FP64, W.MIXED, W.DF64], ids=["fp64", "mixed", "df64"])
def test_state_calls_match_field_calls(precision, pinned):
    # sim_set_state / sim_get_state (one synchronisation each) give the bits of
    # four sim_set_fields / sim_fields calls, from and into pageable arrays
    # (copies) and page-locked arrays (read and written by the kernels)
    case = W.c1_small().replace(precision=precision)
    keep = []
    with sim.Simulation(case) as a, sim.Simulation(case) as b:
        a.step(3)
        mid = a.fields()
        b.set_fields(mid)
        a.set_state(_page_locked(mid, keep) if pinned else mid)
        a.step(4)
        b.step(4)
        out = _page_locked({k: np.full(a.shape(k), np.nan) for k in "uvpT"}, keep) if pinned else None
        got, res, st = a.get_state(out)
        ref = b.fields()
        rres, _, _ = b.residuals()
    assert st == sim.SIM_OK
    for k in "uvpT":
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(res, rres)


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "page-locked"])
def test_set_state_rejects_inadmissible_values_and_changes_nothing(pinned):
    case = W.c1_small()
    keep = []
    with sim.Simulation(case) as s:
        s.step(2)
        before = s.fields()
        bad = {k: v.copy() for k, v in before.items()}
        bad["T"][3, 5] = -1.0
        with pytest.raises(sim.SimError) as e:
            s.set_state(_page_locked(bad, keep) if pinned else bad)
        assert e.value.status == sim.SIM_EINVAL
        bad = {k: v.copy() for k, v in before.items()}
        bad["u"][0, 0] = np.nan
        with pytest.raises(sim.SimError):
            s.set_state(_page_locked(bad, keep) if pinned else bad)
        bad = {k: v.copy() for k, v in before.items()}
        bad["p"][-1, -1] = 0.0                       # the last value of the staged state
        with pytest.raises(sim.SimError):
            s.set_state(_page_locked(bad, keep) if pinned else bad)
        after = s.fields()
    for k in "uvpT":
        assert np.array_equal(before[k], after[k]), k


def test_set_state_clears_a_diverged_handle():
    case = W.c1_small().replace(implicit=True, tvd=False, cfl=3.0)
    with sim.Simulation(case) as s:
        start = s.fields()
        s.step(200)
        _, _, st = s.residuals()
        assert st == sim.SIM_EDIVERGED
        s.set_state(start)
        s.step(1)
