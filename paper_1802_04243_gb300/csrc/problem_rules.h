// problem_rules.h -- host-side rules that turn a problem description
// (include/simplets.h) into the non-dimensional coefficients and the time
// step.  Shared by sim_create and sim_step_noalloc, so that both derive the
// same values from the same description.  Nothing here allocates.
#pragma once

#include <cmath>

#include "simplets.h"
#include "stg_common.cuh"

namespace stg {

// Non-dimensional parameters (Section 4 scaling; Eq. pl37 for the hard-sphere
// gas).  The energy constants are the c_v-form C^Tk_f = gamma C^Tk (C^T3_f
// with a minus sign), the form Eq. pl29 uses.  Fills A, B, C^T1_f..C^T3_f,
// omega, gx, gy of k, the inflow speed u_in and gamma; false for an unknown
// model or an ideal gas without reynolds > 0, gamma > 1, prandtl > 0.
inline bool gas_coefficients(const sim_gas *gas, Coef &k, double &u_in, double &gm)
{
    double ct1, ct2, ct3;
    k.A = 0.5;                 // for every gas model; the FP64 kernels take A dy as the tabulated half height
    if (gas->model == SIM_GAS_HARD_SPHERE_KN) {
        const double pi = 3.14159265358979323846;
        gm = 5.0 / 3.0;
        k.omega = 0.5;
        u_in = gas->mach_in * std::sqrt(gm / 2.0);
        k.B = 5.0 * std::sqrt(pi) * gas->kn / 16.0;
        ct1 = gas->kn * std::sqrt(pi * 225.0 / 1024.0);
        ct2 = std::sqrt(pi) * gas->kn / 4.0;
        ct3 = 2.0 / 5.0;
    } else if (gas->model == SIM_GAS_IDEAL_RE) {
        if (!(gas->reynolds > 0.0) || !(gas->gamma > 1.0) || !(gas->prandtl > 0.0)) return false;
        gm = gas->gamma;
        k.omega = gas->visc_exp;
        u_in = gas->mach_in * std::sqrt(gm / 2.0);
        k.B = u_in / gas->reynolds;
        ct1 = k.B / gas->prandtl;
        ct2 = 2.0 * k.B * (gm - 1.0) / gm;
        ct3 = (gm - 1.0) / gm;
    } else {
        return false;
    }
    k.CT1f = gm * ct1;
    k.CT2f = gm * ct2;
    k.CT3f = -gm * ct3;
    k.B23 = (2.0 / 3.0) * k.B;
    k.gx = gas->gx;
    k.gy = gas->gy;
    return true;
}

// Time step: bc->dt when positive, else cfl * (smallest cell size) /
// (U_ref + sqrt(gamma/2)), with cfl = bc->cfl (0.2 when <= 0) and U_ref the
// largest of |u_in|, the side speeds and the inflow profile.  Cell sizes come
// from grid->dx / dy, or lx/nx, ly/ny when those are NULL.
inline double time_step(const sim_grid *grid, const sim_bc *bc, double u_in, double gm)
{
    if (bc->dt > 0.0) return bc->dt;
    const int nx = grid->nx, ny = grid->ny;
    double cfl = bc->cfl > 0.0 ? bc->cfl : 0.2, dmin = 1e300, uref = std::fabs(u_in);
    for (int i = 0; i < nx; i++) dmin = std::fmin(dmin, grid->dx ? grid->dx[i] : grid->lx / nx);
    for (int j = 0; j < ny; j++) dmin = std::fmin(dmin, grid->dy ? grid->dy[j] : grid->ly / ny);
    for (int s = 0; s < 4; s++) uref = std::fmax(uref, std::fabs(bc->side_vel[s]));
    if (bc->inflow_u)
        for (int j = 0; j < ny; j++) uref = std::fmax(uref, std::fabs(bc->inflow_u[j]));
    return cfl * dmin / (uref + std::sqrt(gm / 2.0));
}

}  // namespace stg
