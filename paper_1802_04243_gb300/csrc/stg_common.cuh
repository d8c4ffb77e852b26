// stg_common.cuh -- data layout shared by the host driver and the sweep
// kernels of the SIMPLE-TS time step (arXiv:1802.04243, Section 3).
//
// Every field lives in one device array of (ny + 5) rows x pitch doubles.
// Element (i, j) of any field -- cell centre, u face (x^f_i, y^v_j) or v face
// (x^v_i, y^f_j) -- sits at IX(i, j) = (j + G) * pitch + (i + G), with two
// ghost layers (G = 2) on every side.  Cells use i in [-2, nx+1], u faces
// i in [-2, nx+2], v faces j in [-2, ny+2].
#pragma once

#include <cstddef>
#include <cstdint>

namespace stg {

constexpr int G = 2;

// Per-node geometry flags, one uint16 per extended grid position (i, j).
enum : uint32_t {
    F_FLUID = 1u << 0,    // cell (i,j) is fluid (an unknown of T and p)
    F_WALL = 1u << 1,     // cell (i,j) is a wall ghost or obstacle cell
    F_UACT = 1u << 2,     // u face (i,j) lies between two fluid cells
    F_UWALL = 1u << 3,    // u face (i,j) lies inside a wall or obstacle
    F_VACT = 1u << 4,     // v face (i,j) lies between two fluid cells
    F_VWALL = 1u << 5,    // v face (i,j) lies inside a wall or obstacle
    F_TCX = 1u << 6,      // cells i-2..i+1 of row j are fluid (TVD on x face i)
    F_TCY = 1u << 7,      // cells j-2..j+1 of column i are fluid (TVD on y face j)
    F_TUX = 1u << 8,      // u faces i-2..i+1 of row j are unknowns
    F_TUY = 1u << 9,      // u faces j-2..j+1 of column i are unknowns
    F_TVX = 1u << 10,     // v faces i-2..i+1 of row j are unknowns
    F_TVY = 1u << 11,     // v faces j-2..j+1 of column i are unknowns
};

// Per-index grid factors, each array indexed by i + G (x) or j + G (y) over
// the extended range [-2, n + 2].
struct Axis {
    const double *d;      // cell size
    const double *rd;     // 1 / d
    const double *wlo;    // d_i / (d_{i-1} + d_i): weight of index i-1 at face i
    const double *whi;    // d_{i-1} / (d_{i-1} + d_i): weight of index i at face i
    const double *rc;     // 1 / (0.5 (d_{i-1} + d_i)): inverse centre distance across face i
};

struct Geo {
    int nx, ny;
    int pitch;
    const uint16_t *flag;
    Axis x, y;
};

struct Coef {
    double A, B, CT1f, CT2f, CT3f, omega, dt, gx, gy;
};

struct Level {
    double *u, *v, *p, *T, *rho, *gam;
};

// Boundary description used by the ghost refresh.
struct Sides {
    int kind[4];          // W, E, S, N
};

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { BC_WALL = 0, BC_SYMMETRY = 1, BC_INFLOW = 2, BC_OUTFLOW = 3 };

// Scratch of one loop-2 iteration (all extended-indexed).
struct Work {
    double *rho_u, *rho_v;        // face densities (Eqs. pl10, pl11)
    double *uhat, *du, *vhat, *dv; // pseudo velocities and d (Eqs. pl14, pl20, pl21)
    double *uexp, *vexp, *Texp;   // explicit convective terms (Eqs. pl15_11, pl31_1)
    unsigned long long *res;      // 4 residual maxima as ordered bit patterns
};

// Launch wrappers (sweep_kernels.cu).  All are asynchronous on `stream`.
void launch_face_densities(const Geo &g, const Level &lv, const Work &w, bool tvd, void *stream);
void launch_explicit_terms(const Geo &g, const Level &prev, const Work &w, bool tvd, void *stream);
void launch_assemble(const Geo &g, const Coef &c, const Level &prev, const Level &old,
                     const Level &nw, const Work &w, bool implicit, bool tvd, void *stream);
void launch_pressure(const Geo &g, const Coef &c, const Level &prev, const Level &old,
                     const Level &nw, const Work &w, void *stream);
void launch_velocity(const Geo &g, const Level &old, const Level &nw, const Work &w, void *stream);
void launch_ghosts(const Geo &g, const Sides &s, const Level &lv, void *stream);
void launch_derive(const Geo &g, const Coef &c, const Level &lv, void *stream);
void launch_scatter(const Geo &g, int field, const double *src, const Level &lv, void *stream);
void launch_gather(const Geo &g, int field, const Level &lv, double *dst, void *stream);

}  // namespace stg
