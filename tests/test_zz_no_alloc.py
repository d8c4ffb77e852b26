"""sim_step_noalloc (include/simplets_noalloc.h) against the existing entry
points.

sim_step_noalloc is for callers that cannot allocate device memory when they
run the solver (under a fixed memory budget, inside a host framework that owns
the device memory, or where the synchronisation of cudaMalloc is
unacceptable).  It advances state
that lives in the caller's own device arrays and keeps all its working
memory in a static array of the library.  These tests give it device arrays
(allocated here by the test, as such a caller would beforehand), call it
twice in a row, and compare each result with sim_create + sim_step +
sim_fields on the same problem, within the parity tolerance of the other
GPU tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import paper_1802_04243_gb300 as sim
import workloads as W
from paper_1802_04243_gb300 import build

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    sim.load()


def noalloc(case, dev, nsteps, stream):
    d = sim._Desc(case)
    res = np.zeros(4)
    st = sim.load().sim_step_noalloc(ctypes.byref(d.grid), ctypes.byref(d.gas), ctypes.byref(d.bc), int(nsteps),
                                     sim.scheme_of(case.implicit, case.tvd),
                                     *(ctypes.c_void_p(dev[k].data_ptr()) for k in "uvpT"),
                                     ctypes.c_void_p(stream), res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, res


def rel(a, b):
    return max(float(np.abs(a[k] - b[k]).max() / max(np.abs(b[k]).max(), 1e-300)) for k in b)


CASES = {
    "channel-implicit-upwind": lambda: W.c1_small().replace(implicit=True, tvd=False),
    "channel-explicit-tvd": lambda: W.c1_small(),
    "box-ragged-nonuniform-implicit-tvd": lambda: W.closed_box(n=21, tvd=True).replace(
        nx=27, ny=21, dx=np.linspace(0.2, 0.3, 27), dy=np.linspace(0.3, 0.2, 21), lx=float(np.linspace(0.2, 0.3, 27).sum()),
        ly=float(np.linspace(0.3, 0.2, 21).sum()), perturb=1e-3, seed=31),
    "symmetry-sides": lambda: W.uniform_flow(nx=40, ny=18).replace(rects=[[9, 6, 13, 11]], perturb=1e-3),
    "slip-jump-walls": lambda: W.paper_channel(ny=40, nx=160, kn=0.05, side=8, inlet=24).replace(perturb=1e-3),
    "inflow-profile-body-force-hard-sphere": lambda: _profile_case(),
}


def _profile_case():
    # inflow u, T and p profiles (the start state's inflow rows and the inflow
    # ghosts come from them), moving and heated walls, a body force
    ny = 24
    y = (np.arange(ny) + 0.5) / ny
    return W.Case(name="hs", nx=40, ny=ny, lx=40 / 24, ly=1.0, gas_model=W.GAS_HARD_SPHERE_KN, kn=0.01,
                  mach_in=1.2, side_vel=(0, 0, 0.1, -0.2), side_T=(1, 1, 1.1, 0.9), gx=0.05,
                  inflow_u=0.8 * 4 * y * (1 - y), inflow_T=1 + 0.1 * y, inflow_p=np.ones(ny) * 1.05,
                  rects=[[10, 8, 14, 14]], implicit=True, tvd=False, perturb=1e-3, seed=17)


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_matches_sim_step_on_two_calls_in_a_row(name):
    import torch
    case = CASES[name]()
    stream = torch.cuda.current_stream().cuda_stream
    with sim.Simulation(case, stream=stream) as s:
        start = s.fields()
        s.step(6)
        ref1, (r1, _, _) = s.fields(), s.residuals()
        s.step(5)
        ref2, (r2, _, _) = s.fields(), s.residuals()
    dev = {k: torch.from_numpy(start[k]).to("cuda") for k in "uvpT"}
    torch.cuda.synchronize()

    st, res = noalloc(case, dev, 6, stream)
    assert st == sim.SIM_OK
    out1 = {k: dev[k].cpu().numpy() for k in "uvpT"}
    assert rel(out1, ref1) <= TOL
    np.testing.assert_allclose(res, r1, rtol=1e-6, atol=1e-14)

    st, res = noalloc(case, dev, 5, stream)          # second call continues from the first call's output
    assert st == sim.SIM_OK
    out2 = {k: dev[k].cpu().numpy() for k in "uvpT"}
    assert rel(out2, ref2) <= TOL
    np.testing.assert_allclose(res, r2, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("nx,ny", [(1000, 240), (490, 490)])
def test_noalloc_accepts_the_sizes_its_header_names(nx, ny):
    # the header's examples of problems that fit the static scratch
    import torch
    case = W.channel(nx, ny, max(2, ny // 4), name="fits", mach_in=2.0, reynolds=200.0, seed=3)
    with sim.Simulation(case) as s:
        start = s.fields()
    dev = {k: torch.from_numpy(start[k]).to("cuda") for k in "uvpT"}
    torch.cuda.synchronize()
    st, res = noalloc(case, dev, 1, torch.cuda.current_stream().cuda_stream)
    assert st == sim.SIM_OK
    assert np.all(np.isfinite(res))


def test_noalloc_rejects_problems_larger_than_its_static_scratch():
    import torch
    case = W.c3_large()
    dev = {k: torch.zeros(1, dtype=torch.float64, device="cuda") for k in "uvpT"}
    st, _ = noalloc(case, dev, 1, torch.cuda.current_stream().cuda_stream)
    assert st == sim.SIM_ENOMEM


def test_noalloc_rejects_unsupported_descriptions():
    import torch
    dev = {k: torch.zeros(1, dtype=torch.float64, device="cuda") for k in "uvpT"}
    for bad in (dict(tol=1e-6), dict(precision=W.MIXED), dict(nx=3)):
        st, _ = noalloc(W.c1_small().replace(**bad), dev, 1, torch.cuda.current_stream().cuda_stream)
        assert st == sim.SIM_EINVAL, bad
