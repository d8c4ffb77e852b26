/*
 * simplets_oracle.h -- interface of the serial FP64 reference implementation
 * of SIMPLE-TS (Shterev, arXiv:1802.04243).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Array layouts (logical, no ghost cells), row-major with x fastest:
 *   u : (nx+1) * ny   u[j*(nx+1) + i], face i between cells i-1 and i
 *   v : nx * (ny+1)   v[j*nx + i],     face j between cells j-1 and j
 *   p, T : nx * ny    p[j*nx + i]
 */
#ifndef SIMPLETS_ORACLE_H
#define SIMPLETS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_W = 0, ORC_E = 1, ORC_S = 2, ORC_N = 3 };
enum { ORC_BC_WALL = 0, ORC_BC_SYMMETRY = 1, ORC_BC_INFLOW = 2, ORC_BC_OUTFLOW = 3 };
enum { ORC_GAS_IDEAL_RE = 0, ORC_GAS_HARD_SPHERE_KN = 1 };

typedef struct {
    /* grid */
    int nx, ny;
    double lx, ly;              /* used when dx/dy are NULL (uniform grid) */
    const double *dx, *dy;      /* optional cell sizes, nx and ny entries */
    /* gas (Section 2 and Section 4) */
    int gas_model;
    double gamma, prandtl, visc_exp, mach_in, reynolds, kn;
    double gx, gy;              /* body force per unit mass */
    /* boundaries */
    int side_kind[4];           /* W, E, S, N */
    double side_vel[4];         /* tangential wall velocity */
    double side_T[4];           /* wall temperature */
    double body_T;              /* obstacle temperature */
    int n_rect;
    const int *rect;            /* [i0, j0, i1, j1) per obstacle, cell indices */
    const double *inflow_u, *inflow_T, *inflow_p;  /* optional, ny entries */
    /* time stepping */
    double dt, cfl;
    int implicit, tvd;
    int iters;                  /* loop-2 iterations per step (maximum if tol > 0) */
    double tol;                 /* stop loop 2 when every residual <= tol (0: fixed iters) */
    uint64_t seed;
    double perturb;
    /* velocity-slip and temperature-jump walls (Eqs. pl38, pl39):
     * zeta = zeta_coef / rho_local, tau = tau_coef / rho_local (the paper's
     * hard-sphere values: 1.1466 Kn and 2.1904 Kn); 0 = no slip / no jump */
    double zeta_coef, tau_coef;
} orc_problem;

/* Non-dimensional coefficients derived from the gas description. */
typedef struct {
    double A, B, CT1f, CT2f, CT3f, omega, u_in, dt;
} orc_coeffs;

int orc_coefficients(const orc_problem *P, orc_coeffs *out);

/* Initial state: uniform inflow state plus the seeded perturbation. */
int orc_init(const orc_problem *P, double *u, double *v, double *p, double *T);

/* Advance nsteps time steps from the given state (in/out).
 * res[4] receives max |new - old| of u, v, p, T in the last loop-2 iteration;
 * iters_last receives the number of loop-2 iterations of the last step. */
int orc_run(const orc_problem *P, double *u, double *v, double *p, double *T,
            int nsteps, double *res, int *iters_last);

/* Building blocks exposed for closed-form checks. */
double orc_van_leer(double num, double den);
double orc_psi_s(double f1, double f2, double f3, double f4,
                 double d1, double d2, double d3, double d4, double vel);
double orc_psi_c(double f1, double f2, double f3, double f4,
                 double d1, double d2, double d3, double vel);
double orc_splitmix_uniform(uint64_t seed, int field, int i, int j);
double orc_gam_harmonic(double ga, double gb, double da, double db);

/* Threads the row loops of orc_run use: 1 in the plain build, the OpenMP
 * thread count in the row-parallel build (-fopenmp). */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
