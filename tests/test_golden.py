"""Checks against the stored values of tests/golden/, each printed in a cited
source: the paper's test case and gas constants (Section 5, Eqs. pl35-pl39)
and the published first outputs of splitmix64.  None of these needs a GPU."""
import math
import os

import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_table(name):
    """key -> list of numbers; the last column(s) of a line, after the
    numbers, say where the value is printed."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals = []
            for tok in rest:
                try:
                    vals.append(int(tok, 0) if tok.lower().startswith("0x") else float(tok))
                except ValueError:
                    break                       # the citation starts here
            out[key] = vals
    return out


PAPER = read_table("paper_test_case.txt")


def hard_sphere_case(kn):
    return W.Case(name="hs", nx=8, ny=8, lx=1.0, ly=1.0, gas_model=W.GAS_HARD_SPHERE_KN, kn=kn,
                  mach_in=PAPER["Mach"][0])


@pytest.mark.parametrize("kn", [PAPER["Kn"][0], 0.05])
def test_hard_sphere_coefficients_are_the_printed_ones(kn):
    # Eq. pl37 as printed; the discrete energy equation takes C^T1..3 in the
    # c_v form (times gamma, the C^T3 work term with its sign, -(gamma - 1))
    k = oracle.coefficients(hard_sphere_case(kn))
    gam = PAPER["gamma"][0]
    assert k["A"] == PAPER["A"][0]
    assert k["B"] == pytest.approx(PAPER["B_per_Kn"][0] * kn, rel=1e-15)
    assert k["CT1f"] == pytest.approx(gam * PAPER["CT1_per_Kn"][0] * kn, rel=1e-15)
    assert k["CT2f"] == pytest.approx(gam * PAPER["CT2_per_Kn"][0] * kn, rel=1e-15)
    assert k["CT3f"] == pytest.approx(-gam * PAPER["CT3"][0], rel=1e-15)
    # the inlet speed in units of V0 = sqrt(2 R T0): M sqrt(gamma / 2)
    assert k["u_in"] == pytest.approx(PAPER["Mach"][0] * math.sqrt(gam / 2.0), rel=1e-15)


def test_paper_workloads_use_the_printed_test_case():
    delta, side = PAPER["Delta"][0], 20
    assert 1.0 / side == pytest.approx(delta)
    for ny, h, n in zip(PAPER["mesh_ny"], PAPER["H_channel"], PAPER["particles"]):
        c = W.paper_channel(ny=int(ny))
        assert c.nx == int(PAPER["mesh_nx"][0]) and c.ny == int(ny)
        assert c.lx == pytest.approx(PAPER["L_channel"][0]) and c.ly == pytest.approx(h)
        assert c.lx / c.nx == pytest.approx(delta) and c.ly / c.ny == pytest.approx(delta)
        assert len(c.rects) == int(n)
        for i0, j0, i1, j1 in c.rects:
            assert i1 - i0 == side and j1 - j0 == side                   # squares of side a
            assert i0 * delta == pytest.approx(PAPER["L_inlet"][0])      # 5.5 a from the inlet
        assert c.kn == PAPER["Kn"][0] and c.mach_in == PAPER["Mach"][0]
        assert c.gas_model == W.GAS_HARD_SPHERE_KN
        assert c.zeta_coef == pytest.approx(PAPER["zeta_per_Kn"][0] * c.kn, rel=1e-15)
        assert c.tau_coef == pytest.approx(PAPER["tau_per_Kn"][0] * c.kn, rel=1e-15)
        # seen from the particle the channel walls move with the gas at the
        # inlet (Section 4): both wall speeds are the inlet speed the oracle
        # derives from the case itself, M sqrt(gamma / 2) in units of V0
        u_in = oracle.coefficients(c)["u_in"]
        assert c.side_kind[W.S] == W.WALL and c.side_kind[W.N] == W.WALL
        assert c.side_vel[W.S] == u_in and c.side_vel[W.N] == u_in
        assert c.side_vel[W.W] == 0.0 and c.side_vel[W.E] == 0.0


def test_splitmix64_first_outputs():
    # The oracle's counter-based form hashes state + increment once per key, so
    # key 0 with seed k * increment gives output k + 1 of the sequential
    # generator seeded with 0; the oracle maps the top 53 bits to [-1, 1).
    inc = 0x9E3779B97F4A7C15
    ref = read_table("splitmix64_seed0.txt")
    for idx, (z,) in ((int(k), v) for k, v in ref.items()):
        seed = ((idx - 1) * inc) % 2 ** 64
        expected = (z >> 11) * 2.0 ** -53 * 2.0 - 1.0
        assert oracle.splitmix_uniform(seed, 0, 0, 0) == expected, idx
