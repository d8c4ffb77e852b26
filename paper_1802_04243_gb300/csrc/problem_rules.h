// problem_rules.h -- host-side rules that turn a problem description
// (include/simplets.h) into the non-dimensional coefficients and the time
// step.  Shared by sim_create and sim_step_noalloc, so that both derive the
// same values from the same description.  Nothing here allocates.
#pragma once

#include <cmath>
#include <cstdio>

#include "simplets.h"
#include "stg_common.cuh"

namespace stg {

// The checks of a problem description (include/simplets.h) that every entry
// point applies: grid size and cell sizes, side kinds, wall, obstacle and
// inflow temperatures, obstacle placement, loop-2 control, precision, slip
// and jump coefficients (the gas is checked by gas_coefficients).  Returns
// SIM_OK, or SIM_EINVAL with the reason written to msg (n bytes; msg may be
// NULL).  Host only; nothing is allocated.
inline sim_status check_description(const sim_grid *gr, const sim_bc *bc, char *msg, size_t n)
{
#define STG_BAD(...)                                       \
    do {                                                   \
        if (msg && n) std::snprintf(msg, n, __VA_ARGS__);  \
        return SIM_EINVAL;                                 \
    } while (0)
    if (!gr || !bc) STG_BAD("null description");
    if (gr->nx < 4 || gr->ny < 4 || gr->nx >= (1 << 20) || gr->ny >= (1 << 20))
        STG_BAD("grid %d x %d outside [4, 2^20)", gr->nx, gr->ny);
    // the kernels index the padded grid with 32-bit integers
    const long long padded = ((long long)(gr->nx + 2 * G + 1) + 7) / 8 * 8 * (gr->ny + 2 * G + 1);
    if (padded > 0x7FFFFFFFLL)
        STG_BAD("grid %d x %d: %lld padded elements exceed 32-bit indexing", gr->nx, gr->ny, padded);
    for (int i = 0; i < gr->nx; i++) {
        const double d = gr->dx ? gr->dx[i] : gr->lx / gr->nx;
        if (!(d > 0.0) || !std::isfinite(d)) STG_BAD("cell widths must be positive");
    }
    for (int j = 0; j < gr->ny; j++) {
        const double d = gr->dy ? gr->dy[j] : gr->ly / gr->ny;
        if (!(d > 0.0) || !std::isfinite(d)) STG_BAD("cell heights must be positive");
    }
    for (int s = 0; s < 4; s++) {
        const int kd = bc->side_kind[s];
        if (kd < 0 || kd > 3) STG_BAD("side %d: unknown kind %d", s, kd);
        if (kd == SIM_BC_INFLOW && s != SIM_W) STG_BAD("inflow only on the west side");
        if (kd == SIM_BC_OUTFLOW && s != SIM_E) STG_BAD("outflow only on the east side");
        if (kd == SIM_BC_WALL && !(bc->side_T[s] > 0.0)) STG_BAD("wall temperature must be positive");
    }
    if (bc->n_rect < 0 || (bc->n_rect > 0 && !bc->rect)) STG_BAD("bad obstacle list");
    if (bc->n_rect > 0 && !(bc->body_T > 0.0)) STG_BAD("obstacle temperature must be positive");
    for (int r = 0; r < bc->n_rect; r++) {
        const int *q = bc->rect + 4 * r;
        if (q[0] < 2 || q[1] < 2 || q[2] > gr->nx - 2 || q[3] > gr->ny - 2 || q[2] - q[0] < 2 || q[3] - q[1] < 2)
            STG_BAD("obstacle %d [%d,%d,%d,%d) must be >= 2 cells wide and >= 2 cells from the sides", r, q[0], q[1],
                    q[2], q[3]);
    }
    if (bc->iters < 1) STG_BAD("iters must be >= 1");
    if (!(bc->tol >= 0.0)) STG_BAD("tol must be >= 0");
    if (bc->precision != SIM_FP64 && bc->precision != SIM_MIXED && bc->precision != SIM_DF64)
        STG_BAD("unknown precision");
    if (!(bc->zeta_coef >= 0.0) || !(bc->tau_coef >= 0.0) || !std::isfinite(bc->zeta_coef) ||
        !std::isfinite(bc->tau_coef))
        STG_BAD("slip and jump coefficients must be finite and >= 0");
    if (bc->inflow_T)
        for (int j = 0; j < gr->ny; j++)
            if (!(bc->inflow_T[j] > 0.0)) STG_BAD("inflow temperature must be positive");
#undef STG_BAD
    return SIM_OK;
}

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
