"""Seeded, synthetic workload descriptions shared by the tests, the benchmark
and the smoke check.

This module holds no arithmetic of the method.  It only describes problems:
grid sizes, obstacle rectangles in cell indices, gas and flow parameters,
boundary kinds, scheme switches and seeds.  Both the CUDA library and the
reference oracle turn a description into their own initial state and
coefficients.

The channel cases stand in for the paper's test case (Section 4: flow past
squares in a channel at supersonic speed, uniform grid, 4032 x {200 .. 4000}
cells).  Lengths are in units of the obstacle side, so the cell size is
1 / (obstacle side in cells).
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

# side indices and kinds (same meaning on both sides of the parity tests)
W, E, S, N = 0, 1, 2, 3
WALL, SYMMETRY, INFLOW, OUTFLOW = 0, 1, 2, 3
GAS_IDEAL_RE, GAS_HARD_SPHERE_KN = 0, 1
FP64, MIXED, DF64 = 0, 1, 2


@dataclass
class Case:
    """One flow problem.  Arrays are row-major with x fastest."""

    name: str
    nx: int
    ny: int
    lx: float
    ly: float
    dx: Optional[np.ndarray] = None
    dy: Optional[np.ndarray] = None
    gas_model: int = GAS_IDEAL_RE
    gamma: float = 1.4
    prandtl: float = 0.72
    visc_exp: float = 0.5
    mach_in: float = 2.0
    reynolds: float = 100.0
    kn: float = 0.0
    gx: float = 0.0
    gy: float = 0.0
    side_kind: Sequence[int] = (INFLOW, OUTFLOW, WALL, WALL)
    side_vel: Sequence[float] = (0.0, 0.0, 0.0, 0.0)
    side_T: Sequence[float] = (1.0, 1.0, 1.0, 1.0)
    body_T: float = 1.0
    rects: List[Sequence[int]] = field(default_factory=list)   # [i0, j0, i1, j1)
    inflow_u: Optional[np.ndarray] = None
    inflow_T: Optional[np.ndarray] = None
    inflow_p: Optional[np.ndarray] = None
    dt: float = 0.0          # 0: from cfl
    cfl: float = 0.2
    implicit: bool = True
    tvd: bool = False
    iters: int = 2           # loop-2 iterations per time step
    tol: float = 0.0
    seed: int = 1
    perturb: float = 1e-3
    precision: int = FP64
    # velocity-slip / temperature-jump walls (Eqs. pl38, pl39): zeta = zeta_coef
    # / rho_local, tau = tau_coef / rho_local; 0 = no slip / no jump
    zeta_coef: float = 0.0
    tau_coef: float = 0.0
    steps: int = 1           # length of the run the case is quoted on

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


def _square(cx: float, cy: float, side: int) -> List[int]:
    i0 = int(math.floor(cx - side / 2.0 + 0.5))
    j0 = int(math.floor(cy - side / 2.0 + 0.5))
    return [i0, j0, i0 + side, j0 + side]


def channel(nx: int, ny: int, side: int, n_squares: int = 1, first_at_quarter: bool = True,
            **kw) -> Case:
    """Channel of nx x ny uniform cells with a row of square obstacles of
    `side` cells centred on the mid-height.  One square sits at a quarter of
    the length; several squares are equispaced at k L/(n+1)."""
    if n_squares == 1 and first_at_quarter:
        centres = [nx / 4.0]
    else:
        centres = [k * nx / (n_squares + 1.0) for k in range(1, n_squares + 1)]
    rects = [_square(cx, ny / 2.0, side) for cx in centres]
    name = kw.pop("name", f"channel_{nx}x{ny}")
    return Case(name=name, nx=nx, ny=ny, lx=nx / side, ly=ny / side, rects=rects, **kw)


# ----------------------------------------------------------------- named cases

def c1_small() -> Case:
    """128x32 channel, one square (side H/4) at L/4, explicit TVD, Mach 2, Re 100, 50 steps."""
    return channel(128, 32, 8, name="c1_128x32_explicit_tvd", mach_in=2.0, reynolds=100.0,
                   implicit=False, tvd=True, seed=1, steps=50)


def c2_medium() -> Case:
    """1024x256 channel, one square (side H/4) at L/4, implicit upwind, Mach 2.5, Re 200, 500 steps."""
    return channel(1024, 256, 64, name="c2_1024x256_implicit_upwind", mach_in=2.5, reynolds=200.0,
                   implicit=True, tvd=False, seed=2, steps=500)


def c3_large(implicit: bool = True) -> Case:
    """4096x1024 channel, row of 4 equispaced squares (side H/5), Mach 3, Re 400, 1000 steps."""
    tag = "implicit_upwind" if implicit else "explicit_tvd"
    return channel(4096, 1024, 205, n_squares=4, first_at_quarter=False,
                   name=f"c3_4096x1024_{tag}", mach_in=3.0, reynolds=400.0, cfl=0.15,
                   implicit=implicit, tvd=not implicit, seed=3, steps=1000)


def c4_paper_scale() -> Case:
    """4864x1216 channel (about 5.9M cells), one square (side H/4), implicit, Mach 2, Re 300, 2000 steps."""
    return channel(4864, 1216, 304, name="c4_4864x1216_implicit_upwind", mach_in=2.0, reynolds=300.0,
                   implicit=True, tvd=False, seed=4, steps=2000)


def profile_channel() -> Case:
    """2048x512 channel (the 1024x256 case refined 2x): large enough that the
    state (about 230 MB) does not fit in L2, small enough for a detailed
    profiler capture."""
    return channel(2048, 512, 128, name="profile_2048x512_implicit_upwind", mach_in=2.5, reynolds=200.0,
                   implicit=True, tvd=False, seed=2, steps=500)


def c5_batch(n: int = 64, precision: int = MIXED) -> List[Case]:
    """64 independent channels with seeded uneven grids from 256x64 to 2048x512,
    Mach in [1.5, 3], Re in [50, 400], 1-4 squares of side H/5, 500 steps each."""
    cases = []
    for k in range(n):
        rng = np.random.default_rng(1000 + k)
        nx = int(rng.integers(256 // 32, 2048 // 32 + 1)) * 32
        ny = nx // 4
        mach = float(rng.uniform(1.5, 3.0))
        re = float(rng.uniform(50.0, 400.0))
        nsq = int(rng.integers(1, 5))
        side = int(round(ny / 5.0))
        cases.append(channel(nx, ny, side, n_squares=nsq, first_at_quarter=False,
                             name=f"c5_{k:02d}_{nx}x{ny}", mach_in=mach, reynolds=re,
                             implicit=True, tvd=False, seed=1000 + k, steps=500,
                             precision=precision))
    return cases


def paper_channel(ny: int = 200, nx: int = 4032, kn: float = 0.001, mach: float = 2.43,
                  side: int = 20, inlet: int = 110, implicit: bool = True, tvd: bool = False,
                  seed: int = 9, n_squares: Optional[int] = None) -> Case:
    """The paper's test case (Section 4): square particles of side a in a
    microchannel, seen from the particles, so the gas enters at Mach 2.43 and
    the channel walls move with the inflow speed; hard-sphere gas at Kn = 0.001
    (Eqs. pl35-pl37) with velocity-slip and temperature-jump walls (Eqs. pl38,
    pl39: zeta = 1.1466 Kn / rho, tau = 2.1904 Kn / rho).  Uniform cells of
    0.05 a (side = 20 cells); channel length 201.6 a (4032 cells), inlet length
    5.5 a (110 cells); the paper's heights are 10, 20, 100 and 200 a (200 to
    4000 cells) with 1, 2, 10 and 20 particles, i.e. one per 10 a of height
    (n_squares None); each sits at the centre of its 10 a band, all at the same
    distance from the inlet."""
    u_in = mach * math.sqrt((5.0 / 3.0) / 2.0)
    n = max(1, ny // (10 * side)) if n_squares is None else n_squares
    rects = []
    for k in range(n):
        j0 = int(math.floor((k + 0.5) * ny / n - side / 2.0 + 0.5))
        rects.append([inlet, j0, inlet + side, j0 + side])
    return Case(name=f"paper_{nx}x{ny}", nx=nx, ny=ny, lx=nx / side, ly=ny / side,
                side_kind=(INFLOW, OUTFLOW, WALL, WALL), side_vel=(0.0, 0.0, u_in, u_in),
                rects=rects,
                gas_model=GAS_HARD_SPHERE_KN, kn=kn, mach_in=mach,
                zeta_coef=1.1466 * kn, tau_coef=2.1904 * kn,
                implicit=implicit, tvd=tvd, seed=seed, steps=1000)


# ------------------------------------------------------------ analytic set-ups

def uniform_flow(nx: int = 24, ny: int = 12, implicit: bool = True, tvd: bool = False,
                 mach: float = 1.5) -> Case:
    """Obstacle-free channel with symmetry planes top and bottom and an inflow
    equal to the initial state: the uniform state is a steady solution."""
    return Case(name="uniform", nx=nx, ny=ny, lx=nx / 4.0, ly=ny / 4.0,
                side_kind=(INFLOW, OUTFLOW, SYMMETRY, SYMMETRY), mach_in=mach,
                reynolds=50.0, implicit=implicit, tvd=tvd, perturb=0.0, seed=5)


def closed_box(n: int = 16, implicit: bool = True, tvd: bool = True, seed: int = 7) -> Case:
    """Square box with four walls of different speeds and temperatures and an
    off-centre obstacle; used for the transpose-symmetry check."""
    return Case(name="box", nx=n, ny=n, lx=n / 4.0, ly=n / 4.0,
                side_kind=(WALL, WALL, WALL, WALL),
                side_vel=(0.15, -0.1, 0.2, 0.35), side_T=(1.05, 0.97, 1.1, 1.0),
                body_T=1.2, rects=[[3, 5, 6, 9]], mach_in=0.3, reynolds=20.0,
                implicit=implicit, tvd=tvd, perturb=0.0, seed=seed)


def couette(ny: int = 16, nx: int = 4, u_wall: float = 0.05, reynolds: float = 1.0,
            aspect: float = 32.0) -> Case:
    """Plane Couette channel of height 1: the north wall moves at u_wall, both
    walls at T = 1.  Cells are `aspect` times longer in x than in y so the
    columns are nearly independent.  The test supplies the inflow profiles."""
    return Case(name="couette", nx=nx, ny=ny, lx=nx * aspect / ny, ly=1.0,
                side_kind=(INFLOW, OUTFLOW, WALL, WALL), side_vel=(0.0, 0.0, 0.0, u_wall),
                mach_in=u_wall / math.sqrt(1.4 / 2.0), reynolds=reynolds,
                implicit=True, tvd=False, perturb=0.0, iters=4)


def poiseuille(ny: int = 16, nx: int = 4, u_scale: float = 0.05, reynolds: float = 1.0,
               aspect: float = 32.0) -> Case:
    """Body-force driven channel of height 1 between resting walls at T = 1;
    the test supplies the body force and the inflow profiles."""
    return Case(name="poiseuille", nx=nx, ny=ny, lx=nx * aspect / ny, ly=1.0,
                side_kind=(INFLOW, OUTFLOW, WALL, WALL),
                mach_in=u_scale / math.sqrt(1.4 / 2.0), reynolds=reynolds,
                implicit=True, tvd=False, perturb=0.0, iters=4)
