"""Independent numpy restatements of discrete balances the sweep must satisfy,
shared by the oracle pins and the GPU property tests.  Test infrastructure:
nothing here is used by the product or by the oracle."""
import numpy as np


def fluid_mask(case):
    """True for fluid cells, [j, i]; the obstacles are [i0, j0, i1, j1)."""
    fluid = np.ones((case.ny, case.nx), dtype=bool)
    for i0, j0, i1, j1 in case.rects:
        fluid[j0:j1, i0:i1] = False
    return fluid


def continuity_residual(case, rho0, rho, u, v, dt):
    """Discrete continuity of every cell of a channel (inflow west with
    p = T = 1, outflow east, walls south and north) with upwind face
    densities: mass change over dt plus net outflow of F^x = rho^u u dy and
    F^y = rho^v v dx (Eqs. pl8-pl11 with psi = 0).  Arrays are [j, i]; at a
    fixed point of loop 2 this is what Eqs. pl23, pl24 with the corrections of
    Eqs. pl18, pl19 solve, so it vanishes in every fluid cell."""
    dx = np.asarray(case.dx) if case.dx is not None else np.full(case.nx, case.lx / case.nx)
    dy = np.asarray(case.dy) if case.dy is not None else np.full(case.ny, case.ly / case.ny)
    rx = np.concatenate([np.ones((case.ny, 1)), rho, rho[:, -1:]], axis=1)
    ry = np.concatenate([rho[:1], rho, rho[-1:]], axis=0)        # wall faces carry v = 0
    Fx = np.where(u > 0, rx[:, :-1], rx[:, 1:]) * u * dy[:, None]
    Fy = np.where(v > 0, ry[:-1], ry[1:]) * v * dx[None, :]
    return ((rho - rho0) * dx[None, :] * dy[:, None] / dt
            + (Fx[:, 1:] - Fx[:, :-1]) + (Fy[1:] - Fy[:-1]))
