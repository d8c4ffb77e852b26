"""The C-ABI library loads and exports every symbol include/simplets.h
declares, and rejects invalid problem descriptions before touching the GPU.
No compute calls: these tests run without a GPU."""
import ctypes
import os
import re

import pytest

import paper_1802_04243_gb300 as sim
import workloads as W
from paper_1802_04243_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sim.load()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            with open(os.path.join(inc, f)) as fh:
                text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
            names |= set(re.findall(r"\b((?:sim|simplets)_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "sim_create" in names and "sim_step" in names and len(names) >= 9
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/simplets.h but not exported"
        assert n in sim._SIGNATURES, f"{n} has no binding signature"


def test_no_undeclared_sim_symbols(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", sim.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b((?:sim|simplets)_[a-z0-9_]+)\b", out))
    assert exported <= set(declared_functions())


def _create(case):
    d = sim._Desc(case)
    h = ctypes.c_void_p()
    st = sim.load().sim_create(ctypes.byref(d.grid), ctypes.byref(d.gas), ctypes.byref(d.bc), None, ctypes.byref(h))
    if h.value:
        sim.load().sim_destroy(h)
    return st


@pytest.mark.parametrize("bad", [
    dict(nx=3),
    dict(ny=2),
    dict(nx=60000, ny=60000),                # padded grid beyond 32-bit indexing
    dict(rects=[[1, 10, 9, 18]]),            # touches the inflow ghost band
    dict(rects=[[30, 10, 31, 20]]),          # one cell wide
    dict(rects=[[30, 10, 40, 31]]),          # reaches the north wall
    dict(side_kind=(W.OUTFLOW, W.OUTFLOW, W.WALL, W.WALL)),
    dict(side_kind=(W.INFLOW, W.OUTFLOW, W.INFLOW, W.WALL)),
    dict(iters=0),
    dict(reynolds=0.0),
    dict(gamma=1.0),
    dict(tol=-1.0),
    dict(precision=7),
    dict(side_T=(1.0, 1.0, 0.0, 1.0)),
    dict(zeta_coef=-0.1),
    dict(tau_coef=float("nan")),
])
def test_invalid_descriptions_are_rejected_on_the_host(lib, bad):
    case = W.c1_small().replace(**bad)
    assert _create(case) == sim.SIM_EINVAL


def test_batch_rejects_inconsistent_descriptions_on_the_host(lib):
    import ctypes
    cases = [W.c1_small(), W.c1_small().replace(precision=W.MIXED)]
    descs = [sim._Desc(c) for c in cases]
    grids, gases, bcs = (sim.sim_grid * 2)(), (sim.sim_gas * 2)(), (sim.sim_bc * 2)()
    for q, d in enumerate(descs):
        grids[q], gases[q], bcs[q] = d.grid, d.gas, d.bc
    h = ctypes.c_void_p()
    assert lib.sim_batch_create(2, grids, gases, bcs, None, ctypes.byref(h)) == sim.SIM_EINVAL
    assert lib.sim_batch_create(0, grids, gases, bcs, None, ctypes.byref(h)) == sim.SIM_EINVAL
    lib.sim_batch_destroy(None)


def test_null_arguments(lib):
    assert lib.sim_create(None, None, None, None, None) == sim.SIM_EINVAL
    assert lib.sim_set_state(None, None, None, None, None) == sim.SIM_EINVAL
    assert lib.sim_get_state(None, None, None, None, None, None) == sim.SIM_EINVAL
    assert lib.sim_batch_set_tiles(None, 32, 8, 0) == sim.SIM_EINVAL
    lib.sim_destroy(None)
    assert lib.sim_last_error(None) == b"null handle"


def test_every_translation_unit_is_built_and_the_fp32_units_keep_their_rounding():
    # every .cu file of csrc/ goes into libsimplets.so; the FP32 and
    # double-float units (per-phase and persistent kernels) are compiled
    # without multiply-add contraction, so each compiled form of a body rounds
    # the same way, and the FP64 units with it
    import os
    from paper_1802_04243_gb300 import build as B
    on_disk = sorted(f for f in os.listdir(B.CSRC) if f.endswith(".cu"))
    assert sorted(B.SOURCES) == on_disk
    nofma = {f for f, flags in B.EXTRA_FLAGS.items() if "--fmad=false" in flags}
    assert nofma == {"phase_mixed.cu", "step_mixed.cu", "phase_df64.cu", "step_df64.cu"}
