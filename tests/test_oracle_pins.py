"""Pins of the reference oracle against facts that do not come from the
oracle itself: closed forms, exact invariants of the discrete equations,
analytic flows and the published splitmix64 test vector.

Each test names the part of the paper it pins.  None of these needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from discrete_checks import continuity_residual, fluid_mask

SCHEMES = [(False, False), (False, True), (True, False), (True, True)]   # (implicit, tvd)


# ------------------------------------------------------------ limiter (Eq. pl15_2)

@pytest.mark.parametrize("r", [-5.0, -1.5, -0.5, 0.0, 1e-3, 0.25, 1.0, 2.0, 7.5, 1e3])
def test_van_leer_matches_closed_form(r):
    # psi(r) = (r + |r|)/(1 + r), Van Leer's limiter as printed after Eq. pl15_2
    expected = (r + abs(r)) / (1.0 + r)
    assert oracle.van_leer(r, 1.0) == pytest.approx(expected, rel=1e-15, abs=0)
    # psi depends on the ratio only, whatever the sign of the denominator
    assert oracle.van_leer(3.0 * r, 3.0) == pytest.approx(expected, rel=1e-15, abs=0)
    assert oracle.van_leer(-2.0 * r, -2.0) == pytest.approx(expected, rel=1e-15, abs=0)


def test_van_leer_tvd_region_and_symmetry():
    # Sweby's second-order TVD region: 0 <= psi <= min(2, 2r), psi(1) = 1,
    # and the symmetry psi(r)/r = psi(1/r) of Van Leer's limiter.
    for r in np.geomspace(1e-4, 1e4, 57):
        psi = oracle.van_leer(r, 1.0)
        assert 0.0 <= psi <= min(2.0, 2.0 * r) + 1e-15
        assert psi / r == pytest.approx(oracle.van_leer(1.0 / r, 1.0), rel=1e-13)
    assert oracle.van_leer(1.0, 1.0) == 1.0
    # a vanishing downstream difference (r infinite) falls back to first order
    assert oracle.van_leer(1.0, 0.0) == 0.0


# ------------------------------------------ TVD weights on non-uniform grids (Eqs. pl15_1, pl15_2)

def _positions(d):
    """Cell-centre positions of four consecutive cells of sizes d."""
    x = [0.0]
    for k in range(3):
        x.append(x[-1] + 0.5 * (d[k] + d[k + 1]))
    return x


@pytest.mark.parametrize("seed", range(8))
def test_psi_s_reproduces_linear_data_on_nonuniform_cells(seed):
    # A second-order TVD face value is exact for linear data: r = 1, psi = 1,
    # and the face value must equal the linear interpolant at the cell face.
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.3, 2.0, 4)
    a, b = rng.normal(), rng.normal() + 3.0
    x = _positions(d)
    f = [a + b * xi for xi in x]
    x_face = x[1] + 0.5 * d[1]
    exact = a + b * x_face
    up = oracle.psi_s(*f, *d, 1.0)
    assert f[1] + up * (f[2] - f[1]) == pytest.approx(exact, rel=1e-13)
    dn = oracle.psi_s(*f, *d, -1.0)
    assert f[2] + dn * (f[2] - f[1]) == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("seed", range(8))
def test_psi_c_reproduces_linear_data_on_nonuniform_nodes(seed):
    # psi_c works on node distances; its face lies midway between nodes 2 and 3.
    rng = np.random.default_rng(100 + seed)
    dist = rng.uniform(0.3, 2.0, 3)
    a, b = rng.normal(), rng.normal() - 3.0
    x = np.concatenate([[0.0], np.cumsum(dist)])
    f = a + b * x
    exact = a + b * 0.5 * (x[1] + x[2])
    up = oracle.psi_c(*f, *dist, 1.0)
    assert f[1] + up * (f[2] - f[1]) == pytest.approx(exact, rel=1e-13)
    dn = oracle.psi_c(*f, *dist, -1.0)
    assert f[2] + dn * (f[2] - f[1]) == pytest.approx(exact, rel=1e-13)


def test_tvd_face_value_is_bounded_by_neighbours():
    # On uniform cells (weight 1/2, psi <= 2) monotone data stay monotone: the
    # face value lies between the two nodes.  (On stretched cells the printed
    # weights allow an overshoot, so the check is for uniform spacing.)
    rng = np.random.default_rng(3)
    for _ in range(200):
        f = np.sort(rng.uniform(-2, 2, 4))
        d = np.full(4, rng.uniform(0.5, 1.5))
        for vel in (1.0, -1.0):
            base = f[1] if vel > 0 else f[2]
            face = base + oracle.psi_s(*f, *d, vel) * (f[2] - f[1])
            assert f[1] - 1e-14 <= face <= f[2] + 1e-14


# ------------------------------------------------------- seeded perturbation

def test_splitmix64_published_first_outputs():
    # splitmix64 seeded with 0 outputs 0xE220A8397B1DCDAF, then 0x6E789E6AA1B965F4
    # (Vigna's reference generator).  The hash form adds the Weyl increment to
    # seed ^ key once, so key 0 with seeds 0 and 0x9E3779B97F4A7C15 gives them.
    for seed, z in ((0, 0xE220A8397B1DCDAF), (0x9E3779B97F4A7C15, 0x6E789E6AA1B965F4)):
        expected = (z >> 11) * 2.0 ** -53 * 2.0 - 1.0
        assert oracle.splitmix_uniform(seed, 0, 0, 0) == expected


def test_perturbation_is_small_and_deterministic():
    c = W.c1_small()
    a, b = oracle.init(c), oracle.init(c)
    for k in "uvpT":
        assert np.array_equal(a[k], b[k])
    coef = oracle.coefficients(c)
    fluid = a["T"] != 1.0
    assert np.abs(a["T"] - 1.0).max() <= 1e-3 and fluid.sum() > 0.9 * c.cells
    assert np.abs(a["v"]).max() <= 1e-3 * coef["u_in"] + 1e-15


# ------------------------------------------------------ gas constants (Eq. pl37)

def test_ideal_gas_mapping_reduces_to_hard_sphere_constants():
    # With gamma = 5/3, Pr = 2/3 and B = 5 sqrt(pi) Kn / 16 the ideal-gas
    # mapping must give the hard-sphere constants of Eq. pl37.
    kn, mach = 0.001, 2.43
    hs = oracle.coefficients(W.Case(name="hs", nx=8, ny=8, lx=1, ly=1, gas_model=W.GAS_HARD_SPHERE_KN,
                                    kn=kn, mach_in=mach))
    gam = 5.0 / 3.0
    u_in = mach * math.sqrt(gam / 2)
    re = u_in / (5 * math.sqrt(math.pi) * kn / 16)
    ig = oracle.coefficients(W.Case(name="ig", nx=8, ny=8, lx=1, ly=1, gamma=gam, prandtl=2.0 / 3.0,
                                    reynolds=re, mach_in=mach))
    for k in ("A", "B", "CT1f", "CT2f", "CT3f", "u_in"):
        assert ig[k] == pytest.approx(hs[k], rel=1e-12)
    # Eq. pl37 values, times gamma for the c_v form of the discrete energy equation
    assert hs["CT1f"] == pytest.approx(gam * kn * math.sqrt(math.pi * 225 / 1024), rel=1e-14)
    assert hs["CT2f"] == pytest.approx(gam * math.sqrt(math.pi) * kn / 4, rel=1e-14)
    assert hs["CT3f"] == pytest.approx(-(gam - 1.0), rel=1e-14)


# ------------------------------------------------- uniform flow is steady

@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_uniform_flow_is_preserved(implicit, tvd):
    c = W.uniform_flow(implicit=implicit, tvd=tvd)
    s0 = oracle.init(c)
    s, res, _ = oracle.run(c, s0, nsteps=25)
    u_in = oracle.coefficients(c)["u_in"]
    assert np.abs(s["u"] - u_in).max() < 1e-13
    assert np.abs(s["v"]).max() < 1e-13
    assert np.abs(s["p"] - 1).max() < 1e-13 and np.abs(s["T"] - 1).max() < 1e-13
    assert res.max() < 1e-13


# ------------------------------------------------- mirror symmetry in y

@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_mirror_symmetry_about_mid_height(implicit, tvd):
    # Implicit TVD amplifies rounding differences (see the test below), so its
    # mirror images drift apart after a few steps; it is checked over 2 steps.
    c = W.c1_small().replace(implicit=implicit, tvd=tvd, perturb=0.0)
    s, _, _ = oracle.run(c, nsteps=2 if (implicit and tvd) else 20)
    scale = {k: np.abs(s[k]).max() for k in "uvpT"}
    assert np.abs(s["u"] - s["u"][::-1]).max() <= 1e-12 * scale["u"]
    assert np.abs(s["p"] - s["p"][::-1]).max() <= 1e-12 * scale["p"]
    assert np.abs(s["T"] - s["T"][::-1]).max() <= 1e-12 * scale["T"]
    assert np.abs(s["v"] + s["v"][::-1]).max() <= 1e-12 * scale["u"]
    assert np.abs(s["v"]).max() > 1e-3          # the flow is two-dimensional


def _growth(case, steps, eps=1e-14):
    a = oracle.init(case)
    rng = np.random.default_rng(0)
    b = {k: v * (1 + eps * rng.standard_normal(v.shape)) for k, v in a.items()}
    a = oracle.run(case, a, nsteps=steps)[0]
    b = oracle.run(case, b, nsteps=steps)[0]
    return max(np.abs(a[k] - b[k]).max() / np.abs(a[k]).max() for k in "uvpT")


def test_rounding_sensitivity_per_scheme():
    # A 1e-14 relative perturbation of the start state decays under three of
    # the four schemes.  Under implicit TVD it grows by orders of magnitude:
    # the limiter ratio of two near-zero differences switches between
    # branches, and the coefficient form of Eqs. pl15/pl31 multiplies that
    # switch by (phi_P^new - phi_nb^old), which is not small inside loop 2.
    c = W.c1_small()
    for implicit, tvd in SCHEMES[:3]:
        assert _growth(c.replace(implicit=implicit, tvd=tvd), 40) < 1e-12
    assert _growth(c.replace(implicit=True, tvd=True), 40) > 1e-8


# ------------------------------ transpose symmetry (pins the unprinted u equation)

def _box_pair(implicit, tvd, zeta_coef=0.0, tau_coef=0.0):
    rng = np.random.default_rng(11)
    nx, ny = 12, 9
    dx = rng.uniform(0.2, 0.4, nx)
    dy = rng.uniform(0.2, 0.4, ny)
    a = W.closed_box(implicit=implicit, tvd=tvd).replace(
        nx=nx, ny=ny, dx=dx, dy=dy, lx=float(dx.sum()), ly=float(dy.sum()),
        rects=[[3, 2, 6, 5]], gx=0.02, gy=-0.03, dt=0.02, iters=3, zeta_coef=zeta_coef, tau_coef=tau_coef)
    # the transposed problem: x <-> y, u <-> v, W <-> S, E <-> N
    perm = [W.S, W.N, W.W, W.E]
    b = a.replace(nx=ny, ny=nx, dx=dy, dy=dx, lx=a.ly, ly=a.lx,
                  rects=[[r[1], r[0], r[3], r[2]] for r in a.rects],
                  side_vel=tuple(a.side_vel[perm[k]] for k in range(4)),
                  side_T=tuple(a.side_T[perm[k]] for k in range(4)),
                  gx=a.gy, gy=a.gx)
    sa = oracle.init(a)
    sa["u"] = sa["u"] + 0.05 * rng.standard_normal(sa["u"].shape)
    sa["v"] = sa["v"] + 0.05 * rng.standard_normal(sa["v"].shape)
    sa["p"] = 1.0 + 0.05 * rng.standard_normal(sa["p"].shape)
    sa["T"] = 1.0 + 0.05 * rng.standard_normal(sa["T"].shape)
    sb = {"u": sa["v"].T.copy(), "v": sa["u"].T.copy(), "p": sa["p"].T.copy(), "T": sa["T"].T.copy()}
    return a, b, sa, sb


@pytest.mark.parametrize("slip", [False, True], ids=["noslip", "slip"])
@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_transposed_problem_gives_transposed_fields(implicit, tvd, slip):
    # with slip and jump walls (Eqs. pl38, pl39): u slips across walls in y,
    # v across walls in x, and T jumps at every wall
    a, b, sa, sb = _box_pair(implicit, tvd, *((0.3, 0.5) if slip else (0.0, 0.0)))
    ra, _, _ = oracle.run(a, sa, nsteps=6)
    rb, _, _ = oracle.run(b, sb, nsteps=6)
    tol = 1e-12
    assert np.abs(ra["u"] - rb["v"].T).max() <= tol * np.abs(ra["u"]).max()
    assert np.abs(ra["v"] - rb["u"].T).max() <= tol * np.abs(ra["v"]).max()
    assert np.abs(ra["p"] - rb["p"].T).max() <= tol * np.abs(ra["p"]).max()
    assert np.abs(ra["T"] - rb["T"].T).max() <= tol * np.abs(ra["T"]).max()
    # the run moved the state a long way from the start
    assert np.abs(ra["u"] - sa["u"]).max() > 1e-2


# ------------------------------------------------- plane Couette flow

def test_couette_flow_profile():
    # Fully developed compressible Couette flow between isothermal walls at
    # T = 1 (energy equation with Phi = (du/dy)^2, Eq. pl7): u = U y/H and
    # T = 1 + Pr (gamma-1)/gamma U^2 (y/H)(1 - y/H) to leading order in U^2.
    ny, uw = 16, 0.05
    c = W.couette(ny=ny, u_wall=uw, reynolds=1.0)
    y = (np.arange(ny) + 0.5) / ny
    theta = c.prandtl * (c.gamma - 1) / c.gamma * uw ** 2 * y * (1 - y)
    c = c.replace(inflow_u=uw * y, inflow_T=1 + theta, inflow_p=np.ones(ny), dt=0.05)
    s = oracle.init(c)
    s["T"][:] = 1.0                       # start cold: the heating must build the profile
    s, res, _ = oracle.run(c, s, nsteps=1500)
    i = c.nx - 1
    assert np.abs(s["u"][:, i] - uw * y).max() < 2e-3 * uw
    assert np.abs(s["v"]).max() < 1e-3 * uw
    amp = theta.max()
    assert np.abs((s["T"][:, i] - 1) - theta).max() < 0.05 * amp
    assert res.max() < 1e-9


# ------------------------------------------------- plane Poiseuille flow

def test_poiseuille_flow_profile():
    # Body-force driven flow (rho g_x in Eq. pl2, added to b^u) between resting
    # walls: u = g y (H - y) / (2 B) with B = U_ref / Re (Section 4 scaling).
    ny, umax = 16, 0.05
    c = W.poiseuille(ny=ny, u_scale=umax, reynolds=1.0)
    B = oracle.coefficients(c)["B"]
    g = 8.0 * B * umax
    y = (np.arange(ny) + 0.5) / ny
    u_exact = g * y * (1 - y) / (2 * B)
    c = c.replace(gx=g, inflow_u=u_exact, inflow_T=np.ones(ny), inflow_p=np.ones(ny), dt=0.05)
    s = oracle.init(c)
    s["u"][:, 1:c.nx] = 0.0               # start at rest: the body force must build the profile
    s, res, _ = oracle.run(c, s, nsteps=1500)
    i = c.nx - 1
    assert np.abs(s["u"][:, i] - u_exact).max() < 5e-3 * umax
    assert np.abs(s["v"]).max() < 1e-3 * umax
    assert res.max() < 1e-6


# ------------------------------------------------- global mass conservation

@pytest.mark.parametrize("implicit,tvd", SCHEMES)
def test_mass_conservation_at_loop2_convergence(implicit, tvd):
    # Eqs. pl23, pl24 are continuity with rho = p/T: once loop 2 has converged,
    # the mass change over a step equals dt times (inflow - outflow).
    c = W.channel(48, 16, 4, mach_in=1.5, reynolds=50.0, implicit=implicit, tvd=tvd, seed=9)
    s, _, _ = oracle.run(c, nsteps=5)
    conv = c.replace(iters=400, tol=1e-14)
    s1, res, it = oracle.run(conv, s, nsteps=1)
    assert res.max() < 1e-12 and it < 400
    coef = oracle.coefficients(c)
    dx, dy = c.lx / c.nx, c.ly / c.ny
    mass0 = (s["p"] / s["T"]).sum() * dx * dy
    mass1 = (s1["p"] / s1["T"]).sum() * dx * dy
    f_in = coef["u_in"] * 1.0 * dy * c.ny
    rho_out = s1["p"][:, -1] / s1["T"][:, -1]
    f_out = (rho_out * s1["u"][:, -1] * dy).sum()
    dt = coef["dt"]
    assert abs((mass1 - mass0) - dt * (f_in - f_out)) < 1e-10 * dt * f_in


# ------------------------------- continuity cell by cell at the loop-2 fixed point

@pytest.mark.parametrize("implicit", [False, True])
def test_continuity_holds_in_every_cell_at_loop2_convergence(implicit):
    # What Eqs. pl23, pl24 with the corrections of Eqs. pl18, pl19 solve,
    # restated independently (tests/discrete_checks.py): at a fixed point of
    # loop 2 every fluid cell satisfies discrete continuity with the upwind
    # face densities of the converged iterate (the pressure equation takes them
    # from the previous iterate) and rho = p/T (Eq. pl5).
    # The global mass balance above is the sum of these; this sees every face.
    c = W.channel(48, 16, 4, mach_in=1.5, reynolds=50.0, implicit=implicit, tvd=False, seed=9)
    s, _, _ = oracle.run(c, nsteps=5)
    s1, res, it = oracle.run(c.replace(iters=400, tol=1e-14), s, nsteps=1)
    assert res.max() < 1e-12 and it < 400
    assert np.all(s1["v"][0] == 0) and np.all(s1["v"][-1] == 0)
    coef = oracle.coefficients(c)
    rho0, rho = s["p"] / s["T"], s1["p"] / s1["T"]
    resid = continuity_residual(c, rho0, rho, s1["u"], s1["v"], coef["dt"])
    scale = coef["u_in"] * c.ly / c.ny
    fluid = fluid_mask(c)
    assert np.abs(resid[fluid]).max() < 1e-10 * scale
    # and the check is not empty: the flow is unsteady and crosses the cells
    assert np.abs((rho - rho0)[fluid]).max() * (c.lx / c.nx) * (c.ly / c.ny) / coef["dt"] > 1e-4 * scale


# ------------------------- one cell's energy equation written out by hand

def _van_leer_face(f1, f2, f3, f4, vel):
    """Face value on a uniform grid between nodes f2 and f3 (f1, f4 their
    outer neighbours): the upwind node plus half Van Leer's psi(r) times the
    difference across the face, r the ratio of the upwind-side difference to
    the difference across the face (Eqs. pl10, pl15_1, pl15_2; psi = 0 unless
    both differences have one sign)."""
    def psi(num, den):
        return 2.0 * num / (num + den) if num * den > 0 else 0.0
    if vel > 0:
        return f2 + 0.5 * psi(f2 - f1, f3 - f2) * (f3 - f2)
    return f3 - 0.5 * psi(f4 - f3, f3 - f2) * (f3 - f2)


@pytest.mark.parametrize("tvd", [False, True], ids=["upwind", "van-leer"])
@pytest.mark.parametrize("implicit", [True, False], ids=["implicit", "explicit"])
def test_temperature_of_interior_cells_from_the_printed_equations(implicit, tvd):
    # Eqs. pl28-pl33 (and pl31_1 for the explicit scheme) on a uniform 10 x 8 box,
    # evaluated here term by term for every cell two or more cells from the
    # walls (no reflection in reach, every face stencil complete), after one
    # loop-2 iteration of one step from a random state (old = level n):
    #   F^x = rho^u u dy, rho^u the upwind density or its Van Leer face value
    #   (Eqs. pl8, pl10), F^y likewise;
    #   D = C^T1_f Gamma_h dy / dx, Gamma_h the harmonic mean (Eqs. pl32, pl33);
    #   a_W = max(0, F_w) - F_w psi_w + D_w, a_E = max(0, -F_e) - F_e psi_e + D_e,
    #   ... (Eq. pl31), psi the Van Leer weight of T's face value (0 upwind);
    #   a_0 = dt (sum a + F_e - F_w + F_n - F_s) + rho dV;
    #   S_c = (C^T2_f Gamma Phi + C^T3_f p div u) dV (Eq. pl29, C^T3_f = -(gamma - 1)),
    #   Phi of Eq. pl7 with dv/dx, du/dy from the corner means of four nodes;
    #   T = [dt (sum a T_nb + S_c) + rho^n T^n dV] / a_0 (Eq. pl30).
    # The explicit scheme (Eq. pl31_1) keeps a_k = D_k, drops the flux terms
    # from a_0 and adds T^exp = F_w T_w - F_e T_e + F_s T_s - F_n T_n with the
    # face values of level n-1 (here the start state) to the right-hand side.
    n_x, n_y = 10, 8
    c = W.closed_box(n=8).replace(nx=n_x, ny=n_y, lx=2.5, ly=1.6, rects=[], implicit=implicit, tvd=tvd,
                                  iters=1, perturb=0.0)
    rng = np.random.default_rng(11)
    s = oracle.init(c)
    s["u"][:, 1:n_x] = 0.3 * rng.standard_normal((n_y, n_x - 1))
    s["v"][1:n_y, :] = 0.3 * rng.standard_normal((n_y - 1, n_x))
    s["T"] = 1.0 + 0.3 * rng.random((n_y, n_x))
    s["p"] = 1.0 + 0.3 * rng.random((n_y, n_x))
    new, _, _ = oracle.run(c, s, nsteps=1)
    k = oracle.coefficients(c)
    dt, dx, dy = k["dt"], c.lx / n_x, c.ly / n_y
    u, v, T, p = s["u"], s["v"], s["T"], s["p"]
    rho, gam = p / T, T ** k["omega"]
    harm = lambda a, b: 2.0 * a * b / (a + b)

    def weight(f1, f2, f3, f4, vel):
        # psi of a face value written upwind + psi (f3 - f2)
        if not tvd or f3 == f2:
            return 0.0
        return (_van_leer_face(f1, f2, f3, f4, vel) - (f2 if vel > 0 else f3)) / (f3 - f2)

    def face_rho_x(i, j):
        if tvd:
            return _van_leer_face(rho[j, i - 2], rho[j, i - 1], rho[j, i], rho[j, i + 1], u[j, i])
        return rho[j, i - 1] if u[j, i] > 0 else rho[j, i]

    def face_rho_y(i, j):
        if tvd:
            return _van_leer_face(rho[j - 2, i], rho[j - 1, i], rho[j, i], rho[j + 1, i], v[j, i])
        return rho[j - 1, i] if v[j, i] > 0 else rho[j, i]

    checked = 0
    for j in range(2, n_y - 2):
        for i in range(2, n_x - 2):
            Fw, Fe = face_rho_x(i, j) * u[j, i] * dy, face_rho_x(i + 1, j) * u[j, i + 1] * dy
            Fs, Fn = face_rho_y(i, j) * v[j, i] * dx, face_rho_y(i, j + 1) * v[j + 1, i] * dx
            pw = weight(T[j, i - 2], T[j, i - 1], T[j, i], T[j, i + 1], u[j, i])
            pe = weight(T[j, i - 1], T[j, i], T[j, i + 1], T[j, i + 2], u[j, i + 1])
            ps = weight(T[j - 2, i], T[j - 1, i], T[j, i], T[j + 1, i], v[j, i])
            pn = weight(T[j - 1, i], T[j, i], T[j + 1, i], T[j + 2, i], v[j + 1, i])
            Dw = k["CT1f"] * harm(gam[j, i - 1], gam[j, i]) * dy / dx
            De = k["CT1f"] * harm(gam[j, i], gam[j, i + 1]) * dy / dx
            Ds = k["CT1f"] * harm(gam[j - 1, i], gam[j, i]) * dx / dy
            Dn = k["CT1f"] * harm(gam[j, i], gam[j + 1, i]) * dx / dy
            dV = dx * dy
            if implicit:
                aw, ae = max(0.0, Fw) - Fw * pw + Dw, max(0.0, -Fe) - Fe * pe + De
                as_, an = max(0.0, Fs) - Fs * ps + Ds, max(0.0, -Fn) - Fn * pn + Dn
                a0 = dt * (aw + ae + as_ + an + Fe - Fw + Fn - Fs) + rho[j, i] * dV
                Texp = 0.0
            else:
                aw, ae, as_, an = Dw, De, Ds, Dn
                a0 = dt * (aw + ae + as_ + an) + rho[j, i] * dV
                face = lambda f1, f2, f3, f4, vel: (_van_leer_face(f1, f2, f3, f4, vel) if tvd
                                                    else (f2 if vel > 0 else f3))
                Texp = (Fw * face(T[j, i - 2], T[j, i - 1], T[j, i], T[j, i + 1], u[j, i])
                        - Fe * face(T[j, i - 1], T[j, i], T[j, i + 1], T[j, i + 2], u[j, i + 1])
                        + Fs * face(T[j - 2, i], T[j - 1, i], T[j, i], T[j + 1, i], v[j, i])
                        - Fn * face(T[j - 1, i], T[j, i], T[j + 1, i], T[j + 2, i], v[j + 1, i]))
            ux = (u[j, i + 1] - u[j, i]) / dx
            vy = (v[j + 1, i] - v[j, i]) / dy
            v_w = 0.25 * (v[j, i - 1] + v[j, i] + v[j + 1, i - 1] + v[j + 1, i])
            v_e = 0.25 * (v[j, i] + v[j, i + 1] + v[j + 1, i] + v[j + 1, i + 1])
            u_s = 0.25 * (u[j - 1, i] + u[j, i] + u[j - 1, i + 1] + u[j, i + 1])
            u_n = 0.25 * (u[j, i] + u[j + 1, i] + u[j, i + 1] + u[j + 1, i + 1])
            vx, uy = (v_e - v_w) / dx, (u_n - u_s) / dy
            div = ux + vy
            phi = 2.0 * (ux * ux + vy * vy) + (vx + uy) ** 2 - 2.0 / 3.0 * div * div
            Sc = (k["CT2f"] * gam[j, i] * phi + k["CT3f"] * p[j, i] * div) * dV
            rhs = dt * (aw * T[j, i - 1] + ae * T[j, i + 1] + as_ * T[j - 1, i] + an * T[j + 1, i] + Sc + Texp) \
                + rho[j, i] * T[j, i] * dV
            assert new["T"][j, i] == pytest.approx(rhs / a0, rel=1e-12), (i, j)
            checked += 1
    assert checked == 24
    assert np.abs(new["T"] - T).max() > 1e-3          # the step did change T


# ------------- momentum, pressure and corrections of interior cells written out

def _uniform_box_step(seed, implicit, tvd):
    """One loop-2 iteration of one step on a uniform 12 x 10 box of
    0.25 x 0.2 cells from a random state; returns (case, start, result,
    coefficients)."""
    nx, ny = 12, 10
    c = W.closed_box(n=8).replace(nx=nx, ny=ny, lx=3.0, ly=2.0, rects=[], implicit=implicit, tvd=tvd,
                                  iters=1, perturb=0.0)
    rng = np.random.default_rng(seed)
    s = oracle.init(c)
    s["u"][:, 1:nx] = 0.3 * rng.standard_normal((ny, nx - 1))
    s["v"][1:ny, :] = 0.3 * rng.standard_normal((ny - 1, nx))
    s["T"] = 1.0 + 0.3 * rng.random((ny, nx))
    s["p"] = 1.0 + 0.3 * rng.random((ny, nx))
    new, _, _ = oracle.run(c, s, nsteps=1)
    return c, s, new, oracle.coefficients(c)


@pytest.mark.parametrize("tvd", [False, True], ids=["upwind", "van-leer"])
@pytest.mark.parametrize("implicit", [True, False], ids=["implicit", "explicit"])
def test_momentum_pressure_and_corrections_of_interior_cells_from_the_printed_equations(implicit, tvd):
    # Eqs. pl14-pl16 (implicit) or pl15_11 (explicit) with pl20, pl21 for the
    # v faces and their mirror image for the u faces, the pressure equation
    # Eqs. pl23, pl24 with the new T, and the corrections Eqs. pl18, pl19,
    # evaluated here term by term on a uniform grid for every cell two or more
    # cells from the walls, then compared with one loop-2 iteration of the
    # oracle.  Level n is the start state and the previous iterate.  The
    # Van Leer weight of a face applies only where all four nodes of its
    # stencil are unknowns; the v faces through cell centres take the mean
    # velocity of the cell (F^y bar = rho 0.5 (v_j + v_{j+1}) dx) to pick the
    # upwind side, the faces through corners the velocities of the two
    # neighbouring u faces, each for half of the face.
    c, s, new, k = _uniform_box_step(5, implicit, tvd)
    nx, ny = c.nx, c.ny
    dt, dx, dy, B, A = k["dt"], c.lx / nx, c.ly / ny, k["B"], k["A"]
    u, v, T, p = s["u"], s["v"], s["T"], s["p"]
    rho, gam = p / T, T ** k["omega"]

    fluid = lambda i, j: 0 <= i < nx and 0 <= j < ny
    ua = lambda i, j: 1 <= i <= nx - 1 and 0 <= j <= ny - 1      # u unknowns
    va = lambda i, j: 0 <= i <= nx - 1 and 1 <= j <= ny - 1      # v unknowns
    span = lambda ok, i, j, di, dj: tvd and all(ok(i + q * di, j + q * dj) for q in (-2, -1, 0, 1))

    def face(f1, f2, f3, f4, vel, complete):      # face value, upwind + psi (f3 - f2)
        if complete:
            return _van_leer_face(f1, f2, f3, f4, vel)
        return f2 if vel > 0 else f3

    def psi(f1, f2, f3, f4, vel, complete):       # the psi of that face value
        if not complete or f3 == f2:
            return 0.0
        return (face(f1, f2, f3, f4, vel, True) - (f2 if vel > 0 else f3)) / (f3 - f2)

    def Fx(i, j):                                  # Eqs. pl8, pl10
        r = face(rho[j, i - 2] if i >= 2 else 0, rho[j, i - 1], rho[j, i], rho[j, i + 1] if i + 1 < nx else 0,
                 u[j, i], span(fluid, i, j, 1, 0))
        return r * u[j, i] * dy, r

    def Fy(i, j):                                  # Eqs. pl9, pl11
        r = face(rho[j - 2, i] if j >= 2 else 0, rho[j - 1, i], rho[j, i], rho[j + 1, i] if j + 1 < ny else 0,
                 v[j, i], span(fluid, i, j, 0, 1))
        return r * v[j, i] * dx, r

    def gc(i, j):                                  # Gamma at the corner (x_i, y_j)
        return 0.25 * (gam[j - 1, i - 1] + gam[j - 1, i] + gam[j, i - 1] + gam[j, i])

    def v_face(i, j):                              # v^ and d^v, Eqs. pl14-pl16, pl15_11, pl21
        vP, vW, vE, vS, vN = v[j, i], v[j, i - 1], v[j, i + 1], v[j - 1, i], v[j + 1, i]
        vb_s, vb_n = 0.5 * (vS + vP), 0.5 * (vP + vN)
        Fbs, Fbn = vb_s * rho[j - 1, i] * dx, vb_n * rho[j, i] * dx
        (Fw1, _), (Fw2, _) = Fx(i, j - 1), Fx(i, j)
        (Fe1, _), (Fe2, _) = Fx(i + 1, j - 1), Fx(i + 1, j)
        uw1, uw2, ue1, ue2 = u[j - 1, i], u[j, i], u[j - 1, i + 1], u[j, i + 1]
        cw, ce = span(va, i, j, 1, 0), span(va, i + 1, j, 1, 0)
        cs, cn = span(va, i, j, 0, 1), span(va, i, j + 1, 0, 1)
        vWW = v[j, i - 2] if cw else 0.0
        vEE = v[j, i + 2] if ce else 0.0
        vSS = v[j - 2, i] if cs else 0.0
        vNN = v[j + 2, i] if cn else 0.0
        Dw, De = B * gc(i, j) * dy / dx, B * gc(i + 1, j) * dy / dx
        Ds, Dn = B * gam[j - 1, i] * dx / dy, B * gam[j, i] * dx / dy
        trans = (rho[j, i] + rho[j - 1, i]) * dy * dx / (2 * dt)
        b = trans * vP + B * (gc(i + 1, j) * (ue2 - ue1) - gc(i, j) * (uw2 - uw1)
                              - 2 / 3 * gam[j, i] * (ue2 - uw2) + 2 / 3 * gam[j - 1, i] * (ue1 - uw1))
        if implicit:
            pw1, pw2 = psi(vWW, vW, vP, vE, uw1, cw), psi(vWW, vW, vP, vE, uw2, cw)
            pe1, pe2 = psi(vW, vP, vE, vEE, ue1, ce), psi(vW, vP, vE, vEE, ue2, ce)
            ps, pn = psi(vSS, vS, vP, vN, vb_s, cs), psi(vS, vP, vN, vNN, vb_n, cn)
            a1 = 0.5 * (max(0.0, Fw2) - Fw2 * pw2 + max(0.0, Fw1) - Fw1 * pw1) + Dw
            a2 = 0.5 * (max(0.0, -Fe2) - Fe2 * pe2 + max(0.0, -Fe1) - Fe1 * pe1) + De
            a3 = max(0.0, Fbs) - Fbs * ps + 4 / 3 * Ds
            a4 = max(0.0, -Fbn) - Fbn * pn + 4 / 3 * Dn
            a0 = a1 + a2 + a3 + a4 + 0.5 * (Fe2 - Fw2 + Fe1 - Fw1) + Fbn - Fbs + trans
            vexp = 0.0
        else:
            a1, a2, a3, a4 = Dw, De, 4 / 3 * Ds, 4 / 3 * Dn
            a0 = a1 + a2 + a3 + a4 + trans
            vexp = (0.5 * (Fw1 * face(vWW, vW, vP, vE, uw1, cw) + Fw2 * face(vWW, vW, vP, vE, uw2, cw))
                    - 0.5 * (Fe1 * face(vW, vP, vE, vEE, ue1, ce) + Fe2 * face(vW, vP, vE, vEE, ue2, ce))
                    + Fbs * face(vSS, vS, vP, vN, vb_s, cs) - Fbn * face(vS, vP, vN, vNN, vb_n, cn))
        vh = (a1 * vW + a2 * vE + a3 * vS + a4 * vN + b + vexp) / a0
        return vh, A * dx / a0

    def u_face(i, j):                              # the mirror image: u^ and d^u, Eq. pl20
        uP, uW, uE, uS, uN = u[j, i], u[j, i - 1], u[j, i + 1], u[j - 1, i], u[j + 1, i]
        ub_w, ub_e = 0.5 * (uW + uP), 0.5 * (uP + uE)
        Fbw, Fbe = ub_w * rho[j, i - 1] * dy, ub_e * rho[j, i] * dy
        (Fs1, _), (Fs2, _) = Fy(i - 1, j), Fy(i, j)
        (Fn1, _), (Fn2, _) = Fy(i - 1, j + 1), Fy(i, j + 1)
        vs1, vs2, vn1, vn2 = v[j, i - 1], v[j, i], v[j + 1, i - 1], v[j + 1, i]
        cw, ce = span(ua, i, j, 1, 0), span(ua, i + 1, j, 1, 0)
        cs, cn = span(ua, i, j, 0, 1), span(ua, i, j + 1, 0, 1)
        uWW = u[j, i - 2] if cw else 0.0
        uEE = u[j, i + 2] if ce else 0.0
        uSS = u[j - 2, i] if cs else 0.0
        uNN = u[j + 2, i] if cn else 0.0
        Ds, Dn = B * gc(i, j) * dx / dy, B * gc(i, j + 1) * dx / dy
        Dw, De = B * gam[j, i - 1] * dy / dx, B * gam[j, i] * dy / dx
        trans = (rho[j, i] + rho[j, i - 1]) * dx * dy / (2 * dt)
        b = trans * uP + B * (gc(i, j + 1) * (vn2 - vn1) - gc(i, j) * (vs2 - vs1)
                              - 2 / 3 * gam[j, i] * (vn2 - vs2) + 2 / 3 * gam[j, i - 1] * (vn1 - vs1))
        if implicit:
            pw, pe = psi(uWW, uW, uP, uE, ub_w, cw), psi(uW, uP, uE, uEE, ub_e, ce)
            ps1, ps2 = psi(uSS, uS, uP, uN, vs1, cs), psi(uSS, uS, uP, uN, vs2, cs)
            pn1, pn2 = psi(uS, uP, uN, uNN, vn1, cn), psi(uS, uP, uN, uNN, vn2, cn)
            a1 = max(0.0, Fbw) - Fbw * pw + 4 / 3 * Dw
            a2 = max(0.0, -Fbe) - Fbe * pe + 4 / 3 * De
            a3 = 0.5 * (max(0.0, Fs2) - Fs2 * ps2 + max(0.0, Fs1) - Fs1 * ps1) + Ds
            a4 = 0.5 * (max(0.0, -Fn2) - Fn2 * pn2 + max(0.0, -Fn1) - Fn1 * pn1) + Dn
            a0 = a1 + a2 + a3 + a4 + 0.5 * (Fn2 - Fs2 + Fn1 - Fs1) + Fbe - Fbw + trans
            uexp = 0.0
        else:
            a1, a2, a3, a4 = 4 / 3 * Dw, 4 / 3 * De, Ds, Dn
            a0 = a1 + a2 + a3 + a4 + trans
            uexp = (0.5 * (Fs1 * face(uSS, uS, uP, uN, vs1, cs) + Fs2 * face(uSS, uS, uP, uN, vs2, cs))
                    - 0.5 * (Fn1 * face(uS, uP, uN, uNN, vn1, cn) + Fn2 * face(uS, uP, uN, uNN, vn2, cn))
                    + Fbw * face(uWW, uW, uP, uE, ub_w, cw) - Fbe * face(uW, uP, uE, uEE, ub_e, ce))
        uh = (a1 * uW + a2 * uE + a3 * uS + a4 * uN + b + uexp) / a0
        return uh, A * dy / a0

    checked = 0
    for j in range(2, ny - 2):
        for i in range(2, nx - 2):
            (uw, dw), (ue, de) = u_face(i, j), u_face(i + 1, j)
            (vs, ds), (vn, dn) = v_face(i, j), v_face(i, j + 1)
            rw, re_ = Fx(i, j)[1], Fx(i + 1, j)[1]
            rs, rn = Fy(i, j)[1], Fy(i, j + 1)[1]
            aw, ae, as_, an = rw * dw * dy, re_ * de * dy, rs * ds * dx, rn * dn * dx     # Eq. pl24
            ap0 = dx * dy / new["T"][j, i] + dt * (aw + ae + as_ + an)
            bp = rho[j, i] * dx * dy - dt * (re_ * ue * dy - rw * uw * dy + rn * vn * dx - rs * vs * dx)
            p_new = (dt * (aw * p[j, i - 1] + ae * p[j, i + 1] + as_ * p[j - 1, i] + an * p[j + 1, i]) + bp) / ap0
            assert new["p"][j, i] == pytest.approx(p_new, rel=1e-12), (i, j)
            # the corrections of the west and south faces, Eqs. pl18, pl19
            if i > 2:
                assert new["u"][j, i] == pytest.approx(uw - dw * (new["p"][j, i] - new["p"][j, i - 1]),
                                                       rel=1e-12, abs=1e-14), (i, j)
            if j > 2:
                assert new["v"][j, i] == pytest.approx(vs - ds * (new["p"][j, i] - new["p"][j - 1, i]),
                                                       rel=1e-12, abs=1e-14), (i, j)
            checked += 1
    assert checked == 48
    assert np.abs(new["p"] - p).max() > 1e-3


# ------------------------------------ observed order of the convection schemes

def _graded_channel(n, tvd, implicit, dt):
    """Channel of 2n x n cells, inflow profiles u = 1.5 U 4y(1-y),
    T = 1 + 0.2 sin(pi y), walls at T = 1, low Mach and Re 20; loop 2 is
    iterated to its fixed point every step."""
    ny = n
    y = (np.arange(ny) + 0.5) / ny
    mach = 0.3
    u_scale = mach * math.sqrt(1.4 / 2.0)
    return W.Case(name="graded", nx=2 * n, ny=ny, lx=2.0, ly=1.0, mach_in=mach, reynolds=20.0,
                  side_kind=(W.INFLOW, W.OUTFLOW, W.WALL, W.WALL), implicit=implicit, tvd=tvd,
                  inflow_u=1.5 * u_scale * 4 * y * (1 - y), inflow_T=1.0 + 0.2 * np.sin(math.pi * y),
                  inflow_p=np.ones(ny), perturb=0.0, iters=300, tol=1e-12, dt=dt)


def _smooth_start(c):
    """The inflow profiles carried through the channel, T modulated along x."""
    s = oracle.init(c)
    y = (np.arange(c.ny) + 0.5) / c.ny
    x = (np.arange(c.nx) + 0.5) * c.lx / c.nx
    s["u"] = np.repeat(c.inflow_u[:, None], c.nx + 1, axis=1)
    s["v"][:] = 0.0
    s["p"][:] = 1.0
    s["T"] = 1.0 + 0.2 * np.sin(math.pi * y)[:, None] * (1.0 + 0.5 * np.sin(2 * math.pi * x / c.lx))[None, :]
    return s


def _observed_order(tvd, implicit, dt_power, t_end=0.4):
    # T at t_end on 16x8, 32x16 and 64x32 cells with dt proportional to
    # h^dt_power; fine solutions averaged 2x2 onto the coarser cells; order
    # from the ratio of successive differences (L1 norm)
    sols = []
    for n in (8, 16, 32):
        nsteps = 8 * (n // 8) ** dt_power
        c = _graded_channel(n, tvd, implicit, t_end / nsteps)
        s, res, _ = oracle.run(c, _smooth_start(c), nsteps=nsteps)
        assert res.max() < 1e-11
        sols.append(s["T"])
    coarsen = lambda a: 0.25 * (a[0::2, 0::2] + a[1::2, 0::2] + a[0::2, 1::2] + a[1::2, 1::2])
    a, b, c = sols[0], coarsen(sols[1]), coarsen(coarsen(sols[2]))
    return math.log2(np.abs(a - b).mean() / np.abs(b - c).mean())


@pytest.mark.parametrize("implicit", [True, False])
def test_observed_order_of_upwind_and_tvd_convection(implicit):
    # Upwind faces (Eqs. pl15, pl31 with psi = 0; pl15_11, pl31_1) are first
    # order in space; Van Leer faces (Eqs. pl15_1, pl15_2) second order on
    # smooth data away from extrema and boundaries (a face whose four-node
    # stencil is not all unknowns stays upwind, so next to walls and the
    # inflow they are), so refined with dt ~ h^2 their observed order
    # is well above one.  Diffusion and sources are central in both.
    p_up = _observed_order(False, implicit, 1)
    p_tvd = _observed_order(True, implicit, 2)
    assert 0.6 < p_up < 1.3, p_up
    assert p_tvd > 1.4 and p_tvd > p_up + 0.4, (p_up, p_tvd)


# ------------------------------ TVD with every limiter zero is upwind

@pytest.mark.parametrize("implicit", [False, True])
def test_tvd_is_upwind_bit_for_bit_when_every_limiter_is_zero(implicit):
    # With every field alternating in sign from node to node (a checkerboard
    # about a mean), each ratio of successive differences is negative, so the
    # Van Leer limiter (Eq. pl15_2, 0 unless both differences have one sign)
    # is 0 on every face.  One loop-2 iteration of one step then evaluates
    # every limiter on that state
    # (the fluxes, the explicit terms of level n-1 and the coefficient forms),
    # and the TVD forms of Eqs. pl10, pl11, pl15, pl15_11, pl31, pl31_1 must
    # give the upwind scheme's bits.  From a smooth state they must not.
    n = 8

    def run(tvd, start):
        c = W.closed_box(n=n, implicit=implicit, tvd=tvd).replace(rects=[], iters=1)
        s = oracle.init(c)
        jc, ic = np.mgrid[0:n, 0:n]
        ju, iu = np.mgrid[0:n, 0:n + 1]
        jv, iv = np.mgrid[0:n + 1, 0:n]
        if start == "checkerboard":
            f = lambda j, i: (-1.0) ** (i + j)
        else:
            f = lambda j, i: np.sin(0.7 * i + 0.3) * np.cos(0.5 * j - 0.2)
        s["T"] = 1.0 + 0.1 * f(jc, ic)
        s["p"] = 1.0 + 0.05 * f(jc, ic)
        s["u"][:, 1:n] = 0.2 + 0.05 * f(ju, iu)[:, 1:n]
        s["v"][1:n, :] = -0.1 + 0.05 * f(jv, iv)[1:n, :]
        return oracle.run(c, s, nsteps=1)[0]

    a, b = run(True, "checkerboard"), run(False, "checkerboard")
    for k in "uvpT":
        assert np.array_equal(a[k], b[k]), k
    a, b = run(True, "smooth"), run(False, "smooth")
    assert max(np.abs(a[k] - b[k]).max() for k in "uvpT") > 1e-8


# ---------------- explicit and implicit convection agree to first order in dt

@pytest.mark.parametrize("tvd", [False, True])
def test_explicit_and_implicit_agree_to_first_order_in_dt(tvd):
    # The explicit terms (Eqs. pl15_11, pl31_1 and the u mirror) and the
    # implicit coefficients (Eqs. pl15, pl31) discretise the same convection;
    # with loop 2 converged their difference after a fixed time is O(dt).
    base = W.closed_box(n=12, tvd=tvd).replace(iters=300, tol=1e-14, reynolds=40.0)
    t_end, errs = 0.32, []
    s0 = oracle.init(base)
    rng = np.random.default_rng(2)
    s0["u"] += 0.02 * rng.standard_normal(s0["u"].shape)
    s0["v"] += 0.02 * rng.standard_normal(s0["v"].shape)
    s0 = oracle.run(base.replace(iters=1), s0, nsteps=0)[0]   # re-apply boundary values
    for nsteps in (8, 16, 32):
        dt = t_end / nsteps
        e = oracle.run(base.replace(implicit=False, dt=dt), s0, nsteps=nsteps)[0]
        i = oracle.run(base.replace(implicit=True, dt=dt), s0, nsteps=nsteps)[0]
        errs.append(max(np.abs(e[k] - i[k]).max() for k in "uvpT"))
    assert errs[0] > 1e-6
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.5, errs


# ------------------------- dissipation function Phi (Eq. pl7) and pressure work (Eq. pl29)

def _one_explicit_iteration(ux, uy, vx, vy, a=1.0):
    """Temperature increment of an interior cell after one loop-2 iteration of
    the explicit scheme, starting from T = p = rho = 1 and the linear velocity
    field u = a(ux (x-x0) + uy (y-y0)), v = a(vx (x-x0) + vy (y-y0))."""
    n = 16
    c = W.closed_box(n=n).replace(rects=[], side_vel=(0, 0, 0, 0), side_T=(1, 1, 1, 1),
                                  implicit=False, tvd=False, iters=1, dt=0.01)
    d = c.lx / n
    x0 = y0 = c.lx / 2
    s = oracle.init(c)
    i = np.arange(n + 1)[None, :]
    j = np.arange(n)[:, None]
    s["u"] = a * (ux * (i * d - x0) + uy * ((j + 0.5) * d - y0)) + 0.0 * s["u"]
    i = np.arange(n)[None, :]
    j = np.arange(n + 1)[:, None]
    s["v"] = a * (vx * ((i + 0.5) * d - x0) + vy * (j * d - y0)) + 0.0 * s["v"]
    r, _, _ = oracle.run(c, s, nsteps=1)
    return r["T"][n // 2, n // 2] - 1.0, oracle.coefficients(c)


def test_dissipation_is_rotation_invariant_and_zero_for_rigid_rotation():
    # Phi is frame invariant: pure shear (du/dy = dv/dx = a) and the same
    # strain rotated by 45 degrees (du/dx = -dv/dy = a) dissipate 4 a^2 each;
    # a rigid rotation dissipates nothing.  With T uniform the explicit energy
    # update is T - 1 = dt dV (C^T2_f Phi + (C^T3_f - 1) div u) / a0 with the
    # same a0 for every field, so the increments must match these ratios.
    shear, _ = _one_explicit_iteration(0, 1, 1, 0)
    ext, _ = _one_explicit_iteration(1, 0, 0, -1)
    rot, _ = _one_explicit_iteration(0, -1, 1, 0)
    assert shear > 1e-6
    assert ext == pytest.approx(shear, rel=1e-9)
    assert abs(rot) < 1e-10 * shear


def test_dilatation_heating_and_pressure_work():
    # Uniform dilatation du/dx = dv/dy = a: Phi = 4a^2 - (2/3)(2a)^2 = 4a^2/3 and
    # div u = 2a; the compression work C^T3_f p div u (C^T3_f = -(gamma-1)) and
    # the convective term -T div(rho u) enter linearly in a.
    shear, k = _one_explicit_iteration(0, 1, 1, 0, a=0.5)
    d1, _ = _one_explicit_iteration(1, 0, 0, 1, a=0.5)
    d2, _ = _one_explicit_iteration(1, 0, 0, 1, a=1.0)
    a = 0.5
    scale = shear / (k["CT2f"] * 4 * a * a)          # dt dV / a0
    quad = (d2 - 2 * d1) / 2                          # c1 a^2
    lin = 2 * d1 - d2 / 2                             # c2 a
    assert quad == pytest.approx(scale * k["CT2f"] * 4 / 3 * a * a, rel=1e-7)
    assert lin == pytest.approx(scale * (k["CT3f"] - 1.0) * 2 * a, rel=1e-7)


# ------------------------- velocity slip and temperature jump (Eqs. pl38, pl39)

def test_slip_couette_flow_profile():
    # Couette flow with Maxwell slip u_s - u_w = zeta du/dn at both walls,
    # zeta = zeta_coef / rho: the profile stays linear with a slip velocity
    # zeta dU/(H + 2 zeta) at each wall, u = U (y + zeta) / (H + 2 zeta).  At
    # p = 2 and T = 1 the density is 2, so zeta is half of zeta_coef.
    ny, uw, zc, rho = 16, 0.05, 0.3, 2.0
    zeta = zc / rho
    y = (np.arange(ny) + 0.5) / ny
    exact = uw * (y + zeta) / (1 + 2 * zeta)
    c = W.couette(ny=ny, u_wall=uw, reynolds=1.0).replace(
        inflow_u=exact, inflow_T=np.ones(ny), inflow_p=rho * np.ones(ny), dt=0.05, zeta_coef=zc)
    s, res, _ = oracle.run(c, oracle.init(c), nsteps=1500)
    i = c.nx - 1
    assert np.abs(s["u"][:, i] - exact).max() < 1e-4 * uw
    assert np.abs(exact - uw * y).max() > 0.1 * uw          # the slip is large against that bound
    assert res.max() < 1e-9


def _jump_conduction(ny, tc=0.2, t_top=1.02, omega=0.5):
    # Gas at rest between walls at T = 1 and t_top with the temperature jump
    # T_s - T_w = tau dT/dn, tau = tc / rho = tc T / p.  Steady state: the
    # Kirchhoff variable K(T) = T^(omega+1)/(omega+1) is linear in y,
    # K(T(y)) = K(T_0) + q y with Gamma dT/dy = q; T_0, T_H, q solve the two
    # jump conditions and K(T_H) - K(T_0) = q H.
    from scipy.optimize import fsolve
    c = W.Case(name="cond", nx=4, ny=ny, lx=1.0, ly=1.0,
               side_kind=(W.SYMMETRY, W.SYMMETRY, W.WALL, W.WALL), side_T=(1, 1, 1, t_top),
               mach_in=0.3, reynolds=2.0, visc_exp=omega, implicit=True, perturb=0.0,
               iters=4, dt=0.02, tau_coef=tc)
    s, res, _ = oracle.run(c, oracle.init(c), nsteps=6000)
    p = s["p"][:, 1].mean()
    K = lambda T: T ** (omega + 1) / (omega + 1)

    def eqs(x):
        T0, TH, q = x
        return [K(TH) - K(T0) - q, T0 - 1 - tc * T0 / p * q / T0 ** omega,
                TH - t_top + tc * TH / p * q / TH ** omega]

    T0, TH, q = fsolve(eqs, [1.0, t_top, t_top - 1.0], xtol=1e-14)
    yc = (np.arange(ny) + 0.5) / ny
    exact = ((K(T0) + q * yc) * (omega + 1)) ** (1 / (omega + 1))
    return np.abs(s["T"][:, 1] - exact).max() / (t_top - 1), res.max(), (T0 - 1) / (t_top - 1)


def test_temperature_jump_conduction_profile():
    pytest.importorskip("scipy")
    err, res, jump = _jump_conduction(16)
    assert res < 1e-12
    assert jump > 0.1                                       # a jump of 14 % of the wall difference
    assert err < 1e-3


# ----------------------- heat conduction with T-dependent Gamma^lambda (Eqs. pl32, pl33)

def _steady_conduction(ny, ratio=4.0, omega=2.0, t_top=3.0):
    n1 = ny // 2
    h = 1.0 / (n1 + (ny - n1) * ratio)
    dy = np.array([h] * n1 + [h * ratio] * (ny - n1))
    c = W.Case(name="cond", nx=4, ny=ny, lx=1.0, ly=float(dy.sum()), dy=dy,
               side_kind=(W.SYMMETRY, W.SYMMETRY, W.WALL, W.WALL), side_T=(1, 1, 1, t_top),
               mach_in=0.3, reynolds=2.0, visc_exp=omega, implicit=True, perturb=0.0,
               iters=4, dt=0.02)
    s, res, _ = oracle.run(c, oracle.init(c), nsteps=6000)
    yc = np.cumsum(dy) - dy / 2
    # Kirchhoff transform of d/dy(T^omega dT/dy) = 0: T^(omega+1) is linear in y
    exact = (1 + (t_top ** (omega + 1) - 1) * yc / dy.sum()) ** (1 / (omega + 1))
    return np.abs(s["T"][:, 1] - exact).max(), res.max()


def test_face_conductance_is_two_half_cells_in_series():
    # Eq. pl32 divides the face value of Gamma (Eq. pl33) by the centre
    # distance 0.5 (da + db).  Between two cells of sizes da, db and
    # conductivities ga, gb that must be the conductance of the two half-cells
    # in series, 1 / (da / (2 ga) + db / (2 gb)), which fixes which size
    # weights which Gamma in the harmonic mean.
    rng = np.random.default_rng(3)
    for _ in range(2000):
        ga, gb = 10.0 ** rng.uniform(-2, 2, 2)
        da, db = 10.0 ** rng.uniform(-2, 1, 2)
        got = oracle.gam_harmonic(ga, gb, da, db) / (0.5 * (da + db))
        want = 1.0 / (da / (2.0 * ga) + db / (2.0 * gb))
        assert got == pytest.approx(want, rel=1e-13)
    # equal sizes: the plain harmonic mean; equal conductivities: that value
    assert oracle.gam_harmonic(2.0, 6.0, 0.3, 0.3) == pytest.approx(3.0, rel=1e-15)
    assert oracle.gam_harmonic(1.7, 1.7, 0.1, 0.9) == pytest.approx(1.7, rel=1e-15)


def test_steady_conduction_converges_to_kirchhoff_solution():
    # Gas at rest between walls at T = 1 and 3, Gamma^lambda = T^2, and a grid
    # whose spacing jumps by 4x at mid height.
    e16, r16 = _steady_conduction(16)
    e32, r32 = _steady_conduction(32)
    assert r16 < 1e-12 and r32 < 1e-12
    assert e32 < 2e-3
    assert math.log2(e16 / e32) > 1.5
