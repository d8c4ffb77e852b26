"""The row-parallel build of the oracle (the same source compiled with OpenMP,
used only as a multi-core CPU baseline) must give the serial build's bits:
every row loop it splits writes disjoint elements with the same arithmetic.
Covers the four schemes on obstacles, moving walls, symmetry planes,
slip/jump walls (Eqs. pl38, pl39) and stretched cells, with ragged row counts
that do not divide evenly among the threads."""
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def rows_threads():
    try:
        oracle.build(rows=True)
    except (OSError, subprocess.CalledProcessError) as e:
        pytest.skip(f"gcc without OpenMP: {e}")
    n = oracle.threads(rows=True)
    if n < 2:
        pytest.skip("one host thread: the row-parallel build runs serially")
    return n


def _stretched(case):
    dx = np.linspace(0.2, 0.32, case.nx)
    dy = np.linspace(0.3, 0.18, case.ny)
    return case.replace(dx=dx, dy=dy, lx=float(dx.sum()), ly=float(dy.sum()))


CASES = {
    "channel-obstacle": lambda: W.c1_small(),
    "box-moving-walls-stretched": lambda: _stretched(W.closed_box(n=19)),
    "uniform-symmetry": lambda: W.uniform_flow(nx=30, ny=13),
    "paper-slip-jump": lambda: W.paper_channel(ny=45, nx=150, side=10, inlet=30),
}


@pytest.mark.parametrize("implicit,tvd", [(True, False), (True, True), (False, True), (False, False)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_row_parallel_build_gives_the_serial_bits(rows_threads, name, implicit, tvd):
    case = CASES[name]().replace(implicit=implicit, tvd=tvd)
    a, ra, ia = oracle.run(case, nsteps=6)
    b, rb, ib = oracle.run(case, nsteps=6, rows=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(ra, rb) and ia == ib
