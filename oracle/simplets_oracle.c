/*
 * simplets_oracle.c -- serial FP64 reference implementation of the SIMPLE-TS
 * time step (Shterev, "GPU implementation of algorithm SIMPLE-TS ...",
 * arXiv:1802.04243).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares nothing
 * with the CUDA path and must never be called by the product.
 *
 * Shape of the computation (Section 3.1, the GPU column of Figs. 1 and 2, in
 * which the CPU "loop 3" is one energy pass followed by one pressure pass):
 *
 *   loop 1 (time steps):
 *     explicit scheme only: explicit convective terms from level n-1
 *                           (Eqs. pl15_11 for v, its mirror for u, pl31_1 for T)
 *     loop 2 (Jacobi iterations, every right-hand side from the previous iterate):
 *       face densities rho^u, rho^v and mass fluxes F^x, F^y   (Eqs. pl8-pl11)
 *       temperature T                                           (Eqs. pl30-pl33, pl28, pl29)
 *       pseudo velocities u^, v^ and d^u, d^v                   (Eqs. pl20, pl21, pl14-pl16)
 *       pressure p, using the T just computed                   (Eqs. pl23, pl24)
 *       velocities u, v from the new p                          (Eqs. pl18, pl19)
 *       density rho = p/T and diffusion coefficient Gamma = T^omega (Eq. pl5, Section 3.4)
 *       maximum residuals |new - old| of u, v, p, T
 *
 * Everything is plain double arithmetic in the order the formulas are printed.
 * The paper prints only the v-momentum coefficients; the u-momentum
 * coefficients here are their mirror image under x<->y, u<->v, i<->j.
 *
 * Boundary treatment (the paper gives only the slip/jump forms Eqs. pl38,
 * pl39 for walls):
 *   - every field lives on an extended grid with two ghost layers;
 *   - ghost cells of an inflow side hold the inflow state, of an outflow side
 *     a zero-gradient copy, of a symmetry side a mirror copy (refreshed after
 *     every iteration);
 *   - wall ghost cells and obstacle cells hold the wall state (wall T, wall
 *     tangential velocity) and are never updated; a temperature or a
 *     tangential velocity read across a wall is reflected about the value at
 *     the wall surface, phi = 2 phi_s - phi_reader, which puts phi_s half a
 *     cell from the reader.  phi_s follows Eqs. pl38, pl39,
 *     phi_s - phi_wall = s dphi/dn with dphi/dn = (phi_reader - phi_s)/h, h half
 *     the reader's size normal to the wall and s = zeta or tau (coefficient
 *     over the local density, the reader's); s = 0 gives phi_s = phi_wall;
 *   - a face between a fluid cell and a wall carries zero normal velocity;
 *   - the TVD correction of a face is applied only when all four nodes of its
 *     stencil are unknowns of the equation, otherwise the face is upwind;
 *   - faces that are not unknowns enter the pressure equation with d = 0 and
 *     their stored velocity as the pseudo velocity.
 */
#include "simplets_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define G 2                  /* ghost layers on each side */

/* Row loops whose iterations write disjoint elements and read only what an
 * earlier pass wrote.  The plain build runs them serially.  The row-parallel
 * build (-fopenmp, the multi-core CPU baseline) splits the rows across
 * threads; each element takes the same arithmetic in the same order in both
 * builds, so they give the same bits.  The residual maxima stay serial. */
#ifdef _OPENMP
#define ROWS _Pragma("omp parallel for private(i) schedule(static)")
#else
#define ROWS
#endif

enum { C_FLUID = 0, C_SOLID, C_WALL, C_SYMM, C_INFLOW, C_OUTFLOW };

typedef struct {
    double *u, *v, *p, *T, *rho, *gam;
} level;

typedef struct {
    const orc_problem *P;
    orc_coeffs k;
    int nx, ny;
    int cw;                  /* extended cell / v row width: nx + 2G */
    int uw;                  /* extended u row width: nx + 1 + 2G */
    int ncell, nu, nv;       /* extended array sizes */
    double *dxe, *dye;       /* cell sizes on the extended grid, index i + G */
    unsigned char *ctype;    /* extended cell type */
    unsigned char *cside;    /* wall side of a C_WALL cell */
    level lv[3];
    /* work arrays on the logical faces */
    double *rho_u, *rho_v, *Fx, *Fy;
    double *uhat, *du, *vhat, *dv;
    double *Fx_prev, *Fy_prev;
    double *Uexp, *Vexp, *Texp;
} orc;

/* ------------------------------------------------------------------ indexing */

static int CI(const orc *o, int i, int j) { return (j + G) * o->cw + (i + G); }
static int UI(const orc *o, int i, int j) { return (j + G) * o->uw + (i + G); }
static int VI(const orc *o, int i, int j) { return (j + G) * o->cw + (i + G); }
static int FU(const orc *o, int i, int j) { return j * (o->nx + 1) + i; }   /* logical u face */
static int FV(const orc *o, int i, int j) { return j * o->nx + i; }         /* logical v face */
static int FC(const orc *o, int i, int j) { return j * o->nx + i; }         /* logical cell */

static double DX(const orc *o, int i) { return o->dxe[i + G]; }
static double DY(const orc *o, int j) { return o->dye[j + G]; }

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

static int ctype(const orc *o, int i, int j)
{
    i = clampi(i, -G, o->nx + G - 1);
    j = clampi(j, -G, o->ny + G - 1);
    return o->ctype[CI(o, i, j)];
}
static int cside(const orc *o, int i, int j)
{
    i = clampi(i, -G, o->nx + G - 1);
    j = clampi(j, -G, o->ny + G - 1);
    return o->cside[CI(o, i, j)];
}
static int fluid(const orc *o, int i, int j) { return ctype(o, i, j) == C_FLUID; }
static int wallish(const orc *o, int i, int j)
{
    int t = ctype(o, i, j);
    return t == C_SOLID || t == C_WALL;
}

/* u node (i,j) sits on the face between cells (i-1,j) and (i,j). */
static int u_active(const orc *o, int i, int j) { return fluid(o, i - 1, j) && fluid(o, i, j); }
static int u_inwall(const orc *o, int i, int j) { return wallish(o, i - 1, j) && wallish(o, i, j); }
/* v node (i,j) sits on the face between cells (i,j-1) and (i,j). */
static int v_active(const orc *o, int i, int j) { return fluid(o, i, j - 1) && fluid(o, i, j); }
static int v_inwall(const orc *o, int i, int j) { return wallish(o, i, j - 1) && wallish(o, i, j); }

/* ------------------------------------------------------- limiter and TVD */

/* Van Leer limiter psi(r) = (r + |r|)/(1 + r) (Eq. pl15_2 text), written for
 * r = num/den: 2 num/(num + den) when num and den have the same sign, else 0
 * (den = 0 gives 0, the first-order fallback). */
double orc_van_leer(double num, double den)
{
    if (num * den > 0.0)
        return 2.0 * num / (num + den);
    return 0.0;
}

/* Surface TVD correction, Eq. pl15_2: the face lies between nodes 2 and 3,
 * d1..d4 are the cell sizes of the four nodes, vel the velocity whose sign
 * picks the upwind side. */
double orc_psi_s(double f1, double f2, double f3, double f4,
                 double d1, double d2, double d3, double d4, double vel)
{
    if (vel > 0.0)
        return d2 / (d2 + d3) * orc_van_leer((d2 + d3) * (f2 - f1), (d1 + d2) * (f3 - f2));
    return -d3 / (d2 + d3) * orc_van_leer((d2 + d3) * (f4 - f3), (d3 + d4) * (f3 - f2));
}

/* Centre TVD correction, Eq. pl15_1: the face lies midway between nodes 2 and
 * 3, d1..d3 are the node distances 1-2, 2-3, 3-4. */
double orc_psi_c(double f1, double f2, double f3, double f4,
                 double d1, double d2, double d3, double vel)
{
    if (vel > 0.0)
        return 0.5 * orc_van_leer(d2 * (f2 - f1), d1 * (f3 - f2));
    return -0.5 * orc_van_leer(d2 * (f4 - f3), d3 * (f3 - f2));
}

/* upwind(phi1, phi2, v), Eq. pl15_12 */
static double upwind(double f1, double f2, double vel) { return vel > 0.0 ? f1 : f2; }

static double maxd(double a, double b) { return a > b ? a : b; }

/* ------------------------------------------------------ seeded perturbation */

/* splitmix64 (Steele, Lea, Flood 2014; constants as published by Vigna)
 * used as a counter-based hash of (seed, field, j, i); result in [-1, 1). */
double orc_splitmix_uniform(uint64_t seed, int field, int i, int j)
{
    uint64_t key = ((uint64_t)field << 40) + ((uint64_t)j << 20) + (uint64_t)i;
    uint64_t z = (seed ^ key) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* ------------------------------------------------------------ coefficients */

/* Non-dimensional parameters.  Reference scales as in Section 4: velocity
 * V0 = sqrt(2 R T0), length = obstacle side, p0 and T0 the inflow/wall state,
 * so p = rho T (Eq. pl5) and the speed of sound is sqrt(gamma/2).
 * Hard-sphere gas: Eq. pl37.  Ideal gas with Reynolds number Re on the
 * obstacle side: A = 1/2, B = U_in/Re, C^T1 = B/Pr, C^T2 = 2B(gamma-1)/gamma,
 * C^T3 = (gamma-1)/gamma (these reduce to Eq. pl37 for the hard-sphere
 * values).  The energy equation Eq. pl6 is written with Dp/Dt; the discrete
 * Eqs. pl29, pl32 use C^Tk_f, the constants after eliminating Dp/Dt with
 * continuity and p = rho T: C^T1_f = gamma C^T1, C^T2_f = gamma C^T2,
 * C^T3_f = -gamma C^T3. */
int orc_coefficients(const orc_problem *P, orc_coeffs *k)
{
    double gam, ct1, ct2, ct3;
    if (P->gas_model == ORC_GAS_HARD_SPHERE_KN) {
        const double pi = 3.14159265358979323846;
        gam = 5.0 / 3.0;
        k->omega = 0.5;
        k->u_in = P->mach_in * sqrt(gam / 2.0);
        k->A = 0.5;
        k->B = 5.0 * sqrt(pi) * P->kn / 16.0;
        ct1 = P->kn * sqrt(pi * 225.0 / 1024.0);
        ct2 = sqrt(pi) * P->kn / 4.0;
        ct3 = 2.0 / 5.0;
    } else if (P->gas_model == ORC_GAS_IDEAL_RE) {
        if (!(P->reynolds > 0.0) || !(P->gamma > 1.0) || !(P->prandtl > 0.0))
            return 1;
        gam = P->gamma;
        k->omega = P->visc_exp;
        k->u_in = P->mach_in * sqrt(gam / 2.0);
        k->A = 0.5;
        k->B = k->u_in / P->reynolds;
        ct1 = k->B / P->prandtl;
        ct2 = 2.0 * k->B * (gam - 1.0) / gam;
        ct3 = (gam - 1.0) / gam;
    } else {
        return 1;
    }
    k->CT1f = gam * ct1;
    k->CT2f = gam * ct2;
    k->CT3f = -gam * ct3;

    if (P->dt > 0.0) {
        k->dt = P->dt;
    } else {
        double cfl = P->cfl > 0.0 ? P->cfl : 0.2;
        double dmin = 1e300, uref = fabs(k->u_in);
        int i;
        for (i = 0; i < P->nx; i++) {
            double d = P->dx ? P->dx[i] : P->lx / P->nx;
            if (d < dmin) dmin = d;
        }
        for (i = 0; i < P->ny; i++) {
            double d = P->dy ? P->dy[i] : P->ly / P->ny;
            if (d < dmin) dmin = d;
        }
        for (i = 0; i < 4; i++)
            if (fabs(P->side_vel[i]) > uref) uref = fabs(P->side_vel[i]);
        if (P->inflow_u)
            for (i = 0; i < P->ny; i++)
                if (fabs(P->inflow_u[i]) > uref) uref = fabs(P->inflow_u[i]);
        k->dt = cfl * dmin / (uref + sqrt(gam / 2.0));
    }
    return 0;
}

static double gamma_of_T(const orc *o, double T)
{
    if (o->k.omega == 0.5)
        return sqrt(T);
    return pow(T, o->k.omega);
}

/* ------------------------------------------------------------- set-up */

static int validate(const orc_problem *P)
{
    int r, s;
    if (P->nx < 4 || P->ny < 4 || P->nx >= (1 << 20) || P->ny >= (1 << 20))
        return 1;
    if (!P->dx && !(P->lx > 0.0)) return 1;
    if (!P->dy && !(P->ly > 0.0)) return 1;
    for (s = 0; s < 4; s++) {
        int kd = P->side_kind[s];
        if (kd == ORC_BC_INFLOW && s != ORC_W) return 1;
        if (kd == ORC_BC_OUTFLOW && s != ORC_E) return 1;
        if (kd < 0 || kd > 3) return 1;
    }
    if (P->side_kind[ORC_S] > ORC_BC_SYMMETRY || P->side_kind[ORC_N] > ORC_BC_SYMMETRY)
        return 1;
    if (!(P->iters >= 1)) return 1;
    for (r = 0; r < P->n_rect; r++) {
        const int *q = P->rect + 4 * r;
        if (q[0] < 2 || q[1] < 2 || q[2] > P->nx - 2 || q[3] > P->ny - 2) return 1;
        if (q[2] - q[0] < 2 || q[3] - q[1] < 2) return 1;
    }
    return 0;
}

static void orc_free(orc *o)
{
    int l;
    free(o->dxe); free(o->dye); free(o->ctype); free(o->cside);
    for (l = 0; l < 3; l++) {
        free(o->lv[l].u); free(o->lv[l].v); free(o->lv[l].p);
        free(o->lv[l].T); free(o->lv[l].rho); free(o->lv[l].gam);
    }
    free(o->rho_u); free(o->rho_v); free(o->Fx); free(o->Fy);
    free(o->uhat); free(o->du); free(o->vhat); free(o->dv);
    free(o->Fx_prev); free(o->Fy_prev);
    free(o->Uexp); free(o->Vexp); free(o->Texp);
}

static int orc_alloc(orc *o, const orc_problem *P)
{
    int l, i, j, nfu, nfv, nfc;
    memset(o, 0, sizeof *o);
    o->P = P;
    if (validate(P) || orc_coefficients(P, &o->k))
        return 1;
    o->nx = P->nx;
    o->ny = P->ny;
    o->cw = P->nx + 2 * G;
    o->uw = P->nx + 1 + 2 * G;
    o->ncell = o->cw * (P->ny + 2 * G);
    o->nu = o->uw * (P->ny + 2 * G);
    o->nv = o->cw * (P->ny + 1 + 2 * G);
    nfu = (P->nx + 1) * P->ny;
    nfv = P->nx * (P->ny + 1);
    nfc = P->nx * P->ny;

    o->dxe = calloc(P->nx + 2 * G, sizeof(double));
    o->dye = calloc(P->ny + 2 * G, sizeof(double));
    o->ctype = calloc(o->ncell, 1);
    o->cside = calloc(o->ncell, 1);
    for (l = 0; l < 3; l++) {
        o->lv[l].u = calloc(o->nu, sizeof(double));
        o->lv[l].v = calloc(o->nv, sizeof(double));
        o->lv[l].p = calloc(o->ncell, sizeof(double));
        o->lv[l].T = calloc(o->ncell, sizeof(double));
        o->lv[l].rho = calloc(o->ncell, sizeof(double));
        o->lv[l].gam = calloc(o->ncell, sizeof(double));
    }
    o->rho_u = calloc(nfu, sizeof(double)); o->Fx = calloc(nfu, sizeof(double));
    o->rho_v = calloc(nfv, sizeof(double)); o->Fy = calloc(nfv, sizeof(double));
    o->uhat = calloc(nfu, sizeof(double)); o->du = calloc(nfu, sizeof(double));
    o->vhat = calloc(nfv, sizeof(double)); o->dv = calloc(nfv, sizeof(double));
    o->Fx_prev = calloc(nfu, sizeof(double)); o->Fy_prev = calloc(nfv, sizeof(double));
    o->Uexp = calloc(nfu, sizeof(double)); o->Vexp = calloc(nfv, sizeof(double));
    o->Texp = calloc(nfc, sizeof(double));
    if (!o->dxe || !o->dye || !o->ctype || !o->cside || !o->Texp || !o->Vexp || !o->Uexp)
        return 2;
    for (l = 0; l < 3; l++)
        if (!o->lv[l].u || !o->lv[l].v || !o->lv[l].p || !o->lv[l].T || !o->lv[l].rho || !o->lv[l].gam)
            return 2;

    /* cell sizes, ghost sizes mirrored from the boundary cells */
    for (i = 0; i < P->nx; i++) o->dxe[i + G] = P->dx ? P->dx[i] : P->lx / P->nx;
    for (j = 0; j < P->ny; j++) o->dye[j + G] = P->dy ? P->dy[j] : P->ly / P->ny;
    for (i = 1; i <= G; i++) {
        o->dxe[G - i] = o->dxe[G + i - 1];
        o->dxe[G + P->nx - 1 + i] = o->dxe[G + P->nx - i];
    }
    for (j = 1; j <= G; j++) {
        o->dye[G - j] = o->dye[G + j - 1];
        o->dye[G + P->ny - 1 + j] = o->dye[G + P->ny - j];
    }

    /* cell types: S/N ghost rows own the corners */
    for (j = -G; j < P->ny + G; j++) {
        for (i = -G; i < P->nx + G; i++) {
            int side = -1, t = C_FLUID, c = CI(o, i, j);
            if (j < 0) side = ORC_S;
            else if (j >= P->ny) side = ORC_N;
            else if (i < 0) side = ORC_W;
            else if (i >= P->nx) side = ORC_E;
            if (side >= 0) {
                int kd = P->side_kind[side];
                t = kd == ORC_BC_WALL ? C_WALL : kd == ORC_BC_SYMMETRY ? C_SYMM
                  : kd == ORC_BC_INFLOW ? C_INFLOW : C_OUTFLOW;
            }
            o->ctype[c] = (unsigned char)t;
            o->cside[c] = (unsigned char)(side < 0 ? 0 : side);
        }
    }
    for (l = 0; l < P->n_rect; l++) {
        const int *q = P->rect + 4 * l;
        for (j = q[1]; j < q[3]; j++)
            for (i = q[0]; i < q[2]; i++)
                o->ctype[CI(o, i, j)] = C_SOLID;
    }
    return 0;
}

static double inflow_u(const orc *o, int j)
{
    j = clampi(j, 0, o->ny - 1);
    return o->P->inflow_u ? o->P->inflow_u[j] : o->k.u_in;
}
static double inflow_T(const orc *o, int j)
{
    j = clampi(j, 0, o->ny - 1);
    return o->P->inflow_T ? o->P->inflow_T[j] : 1.0;
}
static double inflow_p(const orc *o, int j)
{
    j = clampi(j, 0, o->ny - 1);
    return o->P->inflow_p ? o->P->inflow_p[j] : 1.0;
}

/* Mirror / zero-gradient ghost values of symmetry and outflow sides,
 * recomputed from the interior after every update of a level. */
static void ghost_fill(const orc *o, level *L)
{
    const orc_problem *P = o->P;
    int nx = o->nx, ny = o->ny, i, j, k;
    double *sc[4];
    sc[0] = L->p; sc[1] = L->T; sc[2] = L->rho; sc[3] = L->gam;

    if (P->side_kind[ORC_E] == ORC_BC_OUTFLOW) {
        for (j = 0; j < ny; j++) {
            for (k = 0; k < 4; k++) {
                sc[k][CI(o, nx, j)] = sc[k][CI(o, nx - 1, j)];
                sc[k][CI(o, nx + 1, j)] = sc[k][CI(o, nx - 1, j)];
            }
            L->u[UI(o, nx, j)] = L->u[UI(o, nx - 1, j)];
            L->u[UI(o, nx + 1, j)] = L->u[UI(o, nx - 1, j)];
            L->u[UI(o, nx + 2, j)] = L->u[UI(o, nx - 1, j)];
        }
        for (j = 0; j <= ny; j++) {
            L->v[VI(o, nx, j)] = L->v[VI(o, nx - 1, j)];
            L->v[VI(o, nx + 1, j)] = L->v[VI(o, nx - 1, j)];
        }
    }
    if (P->side_kind[ORC_W] == ORC_BC_SYMMETRY) {
        for (j = 0; j < ny; j++) {
            for (k = 0; k < 4; k++) {
                sc[k][CI(o, -1, j)] = sc[k][CI(o, 0, j)];
                sc[k][CI(o, -2, j)] = sc[k][CI(o, 1, j)];
            }
            L->u[UI(o, -1, j)] = -L->u[UI(o, 1, j)];
            L->u[UI(o, -2, j)] = -L->u[UI(o, 2, j)];
        }
        for (j = 0; j <= ny; j++) {
            L->v[VI(o, -1, j)] = L->v[VI(o, 0, j)];
            L->v[VI(o, -2, j)] = L->v[VI(o, 1, j)];
        }
    }
    if (P->side_kind[ORC_E] == ORC_BC_SYMMETRY) {
        for (j = 0; j < ny; j++) {
            for (k = 0; k < 4; k++) {
                sc[k][CI(o, nx, j)] = sc[k][CI(o, nx - 1, j)];
                sc[k][CI(o, nx + 1, j)] = sc[k][CI(o, nx - 2, j)];
            }
            L->u[UI(o, nx + 1, j)] = -L->u[UI(o, nx - 1, j)];
            L->u[UI(o, nx + 2, j)] = -L->u[UI(o, nx - 2, j)];
        }
        for (j = 0; j <= ny; j++) {
            L->v[VI(o, nx, j)] = L->v[VI(o, nx - 1, j)];
            L->v[VI(o, nx + 1, j)] = L->v[VI(o, nx - 2, j)];
        }
    }
    if (P->side_kind[ORC_S] == ORC_BC_SYMMETRY) {
        for (i = -G; i < nx + G; i++)
            for (k = 0; k < 4; k++) {
                sc[k][CI(o, i, -1)] = sc[k][CI(o, i, 0)];
                sc[k][CI(o, i, -2)] = sc[k][CI(o, i, 1)];
            }
        for (i = -G; i <= nx + G; i++) {
            L->u[UI(o, i, -1)] = L->u[UI(o, i, 0)];
            L->u[UI(o, i, -2)] = L->u[UI(o, i, 1)];
        }
        for (i = -G; i < nx + G; i++) {
            L->v[VI(o, i, -1)] = -L->v[VI(o, i, 1)];
            L->v[VI(o, i, -2)] = -L->v[VI(o, i, 2)];
        }
    }
    if (P->side_kind[ORC_N] == ORC_BC_SYMMETRY) {
        for (i = -G; i < nx + G; i++)
            for (k = 0; k < 4; k++) {
                sc[k][CI(o, i, ny)] = sc[k][CI(o, i, ny - 1)];
                sc[k][CI(o, i, ny + 1)] = sc[k][CI(o, i, ny - 2)];
            }
        for (i = -G; i <= nx + G; i++) {
            L->u[UI(o, i, ny)] = L->u[UI(o, i, ny - 1)];
            L->u[UI(o, i, ny + 1)] = L->u[UI(o, i, ny - 2)];
        }
        for (i = -G; i < nx + G; i++) {
            L->v[VI(o, i, ny + 1)] = -L->v[VI(o, i, ny - 1)];
            L->v[VI(o, i, ny + 2)] = -L->v[VI(o, i, ny - 2)];
        }
    }
}

/* Fill a level from logical state arrays: unknowns from the arrays, every
 * other node from the boundary rules, then the ghost copies. */
static void load_level(const orc *o, level *L, const double *u, const double *v,
                       const double *p, const double *T)
{
    const orc_problem *P = o->P;
    int nx = o->nx, ny = o->ny, i, j;

    for (j = -G; j < ny + G; j++) {
        for (i = -G; i < nx + G; i++) {
            int c = CI(o, i, j), t = o->ctype[c];
            double pc = 1.0, Tc = 1.0;
            if (t == C_FLUID) { pc = p[FC(o, i, j)]; Tc = T[FC(o, i, j)]; }
            else if (t == C_SOLID) Tc = P->body_T;
            else if (t == C_WALL) Tc = P->side_T[o->cside[c]];
            else if (t == C_INFLOW) { pc = inflow_p(o, j); Tc = inflow_T(o, j); }
            L->p[c] = pc;
            L->T[c] = Tc;
            L->rho[c] = pc / Tc;
            L->gam[c] = gamma_of_T(o, Tc);
        }
    }
    for (j = -G; j < ny + G; j++) {
        for (i = -G; i <= nx + G; i++) {
            int m = UI(o, i, j);
            int tl = ctype(o, i - 1, j), tr = ctype(o, i, j);
            double val = 0.0;
            if (tl == C_FLUID && tr == C_FLUID) {
                val = u[FU(o, i, j)];
            } else if (tl == C_FLUID || tr == C_FLUID) {
                int other = tl == C_FLUID ? tr : tl;
                if (other == C_INFLOW) val = inflow_u(o, j);
                else val = 0.0;                   /* wall / symmetry face; outflow set by ghost_fill */
            } else if (u_inwall(o, i, j)) {
                int sl = cside(o, i - 1, j), sr = cside(o, i, j);
                if (tl == C_WALL && (sl == ORC_S || sl == ORC_N)) val = P->side_vel[sl];
                else if (tr == C_WALL && (sr == ORC_S || sr == ORC_N)) val = P->side_vel[sr];
                else val = 0.0;                   /* obstacle, or normal to a W/E wall */
            } else if (tl == C_INFLOW || tr == C_INFLOW) {
                val = inflow_u(o, j);
            }
            L->u[m] = val;
        }
    }
    for (j = -G; j <= ny + G; j++) {
        for (i = -G; i < nx + G; i++) {
            int m = VI(o, i, j);
            int tb = ctype(o, i, j - 1), tt = ctype(o, i, j);
            double val = 0.0;
            if (tb == C_FLUID && tt == C_FLUID) {
                val = v[FV(o, i, j)];
            } else if (tb == C_FLUID || tt == C_FLUID) {
                val = 0.0;
            } else if (v_inwall(o, i, j)) {
                int sb = cside(o, i, j - 1), st = cside(o, i, j);
                if (tb == C_WALL && (sb == ORC_W || sb == ORC_E)) val = P->side_vel[sb];
                else if (tt == C_WALL && (st == ORC_W || st == ORC_E)) val = P->side_vel[st];
                else val = 0.0;
            } else {
                val = 0.0;                        /* inflow ghosts carry v = 0 */
            }
            L->v[m] = val;
        }
    }
    ghost_fill(o, L);
}

static void store_level(const orc *o, const level *L, double *u, double *v, double *p, double *T)
{
    int nx = o->nx, ny = o->ny, i, j;
    for (j = 0; j < ny; j++)
        for (i = 0; i <= nx; i++)
            u[FU(o, i, j)] = L->u[UI(o, i, j)];
    for (j = 0; j <= ny; j++)
        for (i = 0; i < nx; i++)
            v[FV(o, i, j)] = L->v[VI(o, i, j)];
    for (j = 0; j < ny; j++)
        for (i = 0; i < nx; i++) {
            p[FC(o, i, j)] = L->p[CI(o, i, j)];
            T[FC(o, i, j)] = L->T[CI(o, i, j)];
        }
}

static void copy_level(const orc *o, level *dst, const level *src)
{
    memcpy(dst->u, src->u, sizeof(double) * o->nu);
    memcpy(dst->v, src->v, sizeof(double) * o->nv);
    memcpy(dst->p, src->p, sizeof(double) * o->ncell);
    memcpy(dst->T, src->T, sizeof(double) * o->ncell);
    memcpy(dst->rho, src->rho, sizeof(double) * o->ncell);
    memcpy(dst->gam, src->gam, sizeof(double) * o->ncell);
}

/* ----------------------------------------------------------- node access */

static double Tc(const orc *o, const level *L, int i, int j) { return L->T[CI(o, i, j)]; }
static double Uc(const orc *o, const level *L, int i, int j) { return L->u[UI(o, i, j)]; }
static double Vc(const orc *o, const level *L, int i, int j) { return L->v[VI(o, i, j)]; }
static double RHOc(const orc *o, const level *L, int i, int j) { return L->rho[CI(o, i, j)]; }
static double GAMc(const orc *o, const level *L, int i, int j) { return L->gam[CI(o, i, j)]; }
static double Pc(const orc *o, const level *L, int i, int j) { return L->p[CI(o, i, j)]; }

/* Value at the wall surface between a reader node (value phi_r, distance h
 * from the surface, local density rho) and a wall (value phi_w): Eqs. pl38,
 * pl39 with the normal derivative (phi_r - phi_s)/h solved for phi_s,
 * phi_s = (h phi_w + s phi_r)/(h + s), s = coef/rho. */
static double wall_surface(double phi_w, double phi_r, double h, double coef, double rho)
{
    double s = coef / rho;
    return (h * phi_w + s * phi_r) / (h + s);
}

/* Temperature of cell (ni,nj) as read from cell (ci,cj): reflected about the
 * surface temperature when (ni,nj) is a wall or obstacle cell (temperature
 * jump, Eq. pl39, tau = tau_coef / rho of the reader cell). */
static double T_at(const orc *o, const level *L, int ci, int cj, int ni, int nj)
{
    double Tn = L->T[CI(o, ni, nj)];
    if (wallish(o, ni, nj)) {
        double Tr = L->T[CI(o, ci, cj)];
        if (o->P->tau_coef > 0.0) {
            double h = 0.5 * (ni != ci ? DX(o, ci) : DY(o, cj));
            return 2.0 * wall_surface(Tn, Tr, h, o->P->tau_coef, RHOc(o, L, ci, cj)) - Tr;
        }
        return 2.0 * Tn - Tr;
    }
    return Tn;
}

/* u of node (mi,mj) as read from node (ai,aj): reflected about the surface
 * velocity when (mi,mj) lies inside a wall or obstacle.  Across a wall in y,
 * u is tangential and slips (Eq. pl38, zeta = zeta_coef / rho of the reader's
 * u control volume, the mean of its two cells); across a wall in x it is the
 * normal component and is reflected about the wall value. */
static double u_at(const orc *o, const level *L, int ai, int aj, int mi, int mj)
{
    double um = L->u[UI(o, mi, mj)];
    if (u_inwall(o, mi, mj)) {
        double ur = L->u[UI(o, ai, aj)];
        if (mj != aj && o->P->zeta_coef > 0.0) {
            double rho = 0.5 * (RHOc(o, L, ai - 1, aj) + RHOc(o, L, ai, aj));
            return 2.0 * wall_surface(um, ur, 0.5 * DY(o, aj), o->P->zeta_coef, rho) - ur;
        }
        return 2.0 * um - ur;
    }
    return um;
}

/* v of node (mi,mj) as read from node (ai,aj): as u_at with x and y swapped. */
static double v_at(const orc *o, const level *L, int ai, int aj, int mi, int mj)
{
    double vm = L->v[VI(o, mi, mj)];
    if (v_inwall(o, mi, mj)) {
        double vr = L->v[VI(o, ai, aj)];
        if (mi != ai && o->P->zeta_coef > 0.0) {
            double rho = 0.5 * (RHOc(o, L, ai, aj - 1) + RHOc(o, L, ai, aj));
            return 2.0 * wall_surface(vm, vr, 0.5 * DX(o, ai), o->P->zeta_coef, rho) - vr;
        }
        return 2.0 * vm - vr;
    }
    return vm;
}


/* TVD applies on a face only when the four stencil nodes are all unknowns. */
static int tvd_cells_x(const orc *o, int i, int j)   /* cells i-2..i+1 (face i) */
{
    return o->P->tvd && fluid(o, i - 2, j) && fluid(o, i - 1, j) && fluid(o, i, j) && fluid(o, i + 1, j);
}
static int tvd_cells_y(const orc *o, int i, int j)   /* cells j-2..j+1 (face j) */
{
    return o->P->tvd && fluid(o, i, j - 2) && fluid(o, i, j - 1) && fluid(o, i, j) && fluid(o, i, j + 1);
}
static int tvd_u_x(const orc *o, int i, int j)       /* u nodes i-2..i+1 */
{
    return o->P->tvd && u_active(o, i - 2, j) && u_active(o, i - 1, j) && u_active(o, i, j) && u_active(o, i + 1, j);
}
static int tvd_u_y(const orc *o, int i, int j)       /* u nodes j-2..j+1 */
{
    return o->P->tvd && u_active(o, i, j - 2) && u_active(o, i, j - 1) && u_active(o, i, j) && u_active(o, i, j + 1);
}
static int tvd_v_x(const orc *o, int i, int j)       /* v nodes i-2..i+1 */
{
    return o->P->tvd && v_active(o, i - 2, j) && v_active(o, i - 1, j) && v_active(o, i, j) && v_active(o, i + 1, j);
}
static int tvd_v_y(const orc *o, int i, int j)       /* v nodes j-2..j+1 */
{
    return o->P->tvd && v_active(o, i, j - 2) && v_active(o, i, j - 1) && v_active(o, i, j) && v_active(o, i, j + 1);
}

/* Gamma at the cell corner (x^f_i, y^f_j): bilinear interpolation between the
 * four surrounding cell centres (Section 3.2, text after Eq. pl15). */
static double gam_corner(const orc *o, const level *L, int i, int j)
{
    double wxm = DX(o, i) / (DX(o, i - 1) + DX(o, i));       /* weight of column i-1 */
    double wxp = DX(o, i - 1) / (DX(o, i - 1) + DX(o, i));   /* weight of column i */
    double wym = DY(o, j) / (DY(o, j - 1) + DY(o, j));
    double wyp = DY(o, j - 1) / (DY(o, j - 1) + DY(o, j));
    double lo = wxm * GAMc(o, L, i - 1, j - 1) + wxp * GAMc(o, L, i, j - 1);
    double hi = wxm * GAMc(o, L, i - 1, j) + wxp * GAMc(o, L, i, j);
    return wym * lo + wyp * hi;
}

/* Harmonic mean of Gamma^lambda at the face between cells a (size da) and b
 * (size db), Eq. pl33 (exported for the closed-form check). */
double orc_gam_harmonic(double ga, double gb, double da, double db)
{
    return (da + db) * ga * gb / (da * gb + db * ga);
}

/* ------------------------------------------------ face densities, fluxes */

/* rho^u at u face (i,j), Eq. pl10 with the TVD term as a correction of the
 * upwind value: rho_up + psi_s (rho_i - rho_{i-1}). */
static double face_rho_u(const orc *o, const level *L, int i, int j)
{
    double vel = Uc(o, L, i, j);
    double rl = RHOc(o, L, i - 1, j), rr = RHOc(o, L, i, j);
    double val = upwind(rl, rr, vel);
    if (tvd_cells_x(o, i, j))
        val += orc_psi_s(RHOc(o, L, i - 2, j), rl, rr, RHOc(o, L, i + 1, j),
                         DX(o, i - 2), DX(o, i - 1), DX(o, i), DX(o, i + 1), vel) * (rr - rl);
    return val;
}

/* rho^v at v face (i,j), Eq. pl11. */
static double face_rho_v(const orc *o, const level *L, int i, int j)
{
    double vel = Vc(o, L, i, j);
    double rb = RHOc(o, L, i, j - 1), rt = RHOc(o, L, i, j);
    double val = upwind(rb, rt, vel);
    if (tvd_cells_y(o, i, j))
        val += orc_psi_s(RHOc(o, L, i, j - 2), rb, rt, RHOc(o, L, i, j + 1),
                         DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vel) * (rt - rb);
    return val;
}

/* F^x = rho^u u dy (Eq. pl8) and F^y = rho^v v dx (Eq. pl9) on every face of
 * the domain, from level L.  rho_u/rho_v may be NULL. */
static void compute_fluxes(const orc *o, const level *L, double *rho_u, double *rho_v,
                           double *Fx, double *Fy)
{
    int i, j;
    ROWS
    for (j = 0; j < o->ny; j++)
        for (i = 0; i <= o->nx; i++) {
            double r = face_rho_u(o, L, i, j);
            if (rho_u) rho_u[FU(o, i, j)] = r;
            Fx[FU(o, i, j)] = r * Uc(o, L, i, j) * DY(o, j);
        }
    ROWS
    for (j = 0; j <= o->ny; j++)
        for (i = 0; i < o->nx; i++) {
            double r = face_rho_v(o, L, i, j);
            if (rho_v) rho_v[FV(o, i, j)] = r;
            Fy[FV(o, i, j)] = r * Vc(o, L, i, j) * DX(o, i);
        }
}

/* ----------------------------------------------------- explicit terms */

/* T^explicit of fluid cell (i,j), Eq. pl31_1, from level n-1 (L) with the
 * level n-1 fluxes. */
static double T_explicit(const orc *o, const level *L, const double *Fx, const double *Fy, int i, int j)
{
    double Tp = Tc(o, L, i, j);
    double Tw = T_at(o, L, i, j, i - 1, j), Te = T_at(o, L, i, j, i + 1, j);
    double Ts = T_at(o, L, i, j, i, j - 1), Tn = T_at(o, L, i, j, i, j + 1);
    double Fw = Fx[FU(o, i, j)], Fe = Fx[FU(o, i + 1, j)];
    double Fs = Fy[FV(o, i, j)], Fn = Fy[FV(o, i, j + 1)];
    double uw = Uc(o, L, i, j), ue = Uc(o, L, i + 1, j);
    double vs = Vc(o, L, i, j), vn = Vc(o, L, i, j + 1);
    double pe = 0, pw = 0, pn = 0, ps = 0;
    if (tvd_cells_x(o, i + 1, j))
        pe = orc_psi_s(Tc(o, L, i - 1, j), Tp, Te, Tc(o, L, i + 2, j),
                       DX(o, i - 1), DX(o, i), DX(o, i + 1), DX(o, i + 2), ue);
    if (tvd_cells_x(o, i, j))
        pw = orc_psi_s(Tc(o, L, i - 2, j), Tw, Tp, Te,
                       DX(o, i - 2), DX(o, i - 1), DX(o, i), DX(o, i + 1), uw);
    if (tvd_cells_y(o, i, j + 1))
        pn = orc_psi_s(Tc(o, L, i, j - 1), Tp, Tn, Tc(o, L, i, j + 2),
                       DY(o, j - 1), DY(o, j), DY(o, j + 1), DY(o, j + 2), vn);
    if (tvd_cells_y(o, i, j))
        ps = orc_psi_s(Tc(o, L, i, j - 2), Ts, Tp, Tn,
                       DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vs);
    return -Fe * (upwind(Tp, Te, ue) + (Te - Tp) * pe)
           + Fw * (upwind(Tw, Tp, uw) + (Tp - Tw) * pw)
           - Fn * (upwind(Tp, Tn, vn) + (Tn - Tp) * pn)
           + Fs * (upwind(Ts, Tp, vs) + (Tp - Ts) * ps);
}

/* v^explicit of v node (i,j), Eq. pl15_11, level n-1. */
static double v_explicit(const orc *o, const level *L, const double *Fx, int i, int j)
{
    double vP = Vc(o, L, i, j);
    double vW = v_at(o, L, i, j, i - 1, j), vE = v_at(o, L, i, j, i + 1, j);
    double vS = Vc(o, L, i, j - 1), vN = Vc(o, L, i, j + 1);
    double Fw1 = Fx[FU(o, i, j - 1)], Fw2 = Fx[FU(o, i, j)];
    double Fe1 = Fx[FU(o, i + 1, j - 1)], Fe2 = Fx[FU(o, i + 1, j)];
    double uw1 = Uc(o, L, i, j - 1), uw2 = Uc(o, L, i, j);
    double ue1 = Uc(o, L, i + 1, j - 1), ue2 = Uc(o, L, i + 1, j);
    double vbar_s = 0.5 * (vS + vP), vbar_n = 0.5 * (vP + vN);
    double pe1 = 0, pe2 = 0, pw1 = 0, pw2 = 0, pn = 0, ps = 0;
    if (tvd_v_x(o, i + 1, j)) {
        double f1 = Vc(o, L, i - 1, j), f4 = Vc(o, L, i + 2, j);
        pe1 = orc_psi_s(f1, vP, vE, f4, DX(o, i - 1), DX(o, i), DX(o, i + 1), DX(o, i + 2), ue1);
        pe2 = orc_psi_s(f1, vP, vE, f4, DX(o, i - 1), DX(o, i), DX(o, i + 1), DX(o, i + 2), ue2);
    }
    if (tvd_v_x(o, i, j)) {
        double f1 = Vc(o, L, i - 2, j);
        pw1 = orc_psi_s(f1, vW, vP, vE, DX(o, i - 2), DX(o, i - 1), DX(o, i), DX(o, i + 1), uw1);
        pw2 = orc_psi_s(f1, vW, vP, vE, DX(o, i - 2), DX(o, i - 1), DX(o, i), DX(o, i + 1), uw2);
    }
    if (tvd_v_y(o, i, j + 1))
        pn = orc_psi_c(vS, vP, vN, Vc(o, L, i, j + 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vbar_n);
    if (tvd_v_y(o, i, j))
        ps = orc_psi_c(Vc(o, L, i, j - 2), vS, vP, vN, DY(o, j - 2), DY(o, j - 1), DY(o, j), vbar_s);
    return -0.5 * (Fe1 * (upwind(vP, vE, ue1) + (vE - vP) * pe1)
                   + Fe2 * (upwind(vP, vE, ue2) + (vE - vP) * pe2))
           + 0.5 * (Fw1 * (upwind(vW, vP, uw1) + (vP - vW) * pw1)
                    + Fw2 * (upwind(vW, vP, uw2) + (vP - vW) * pw2))
           - DX(o, i) * RHOc(o, L, i, j) * vbar_n * (upwind(vP, vN, vbar_n) + (vN - vP) * pn)
           + DX(o, i) * RHOc(o, L, i, j - 1) * vbar_s * (upwind(vS, vP, vbar_s) + (vP - vS) * ps);
}

/* u^explicit of u node (i,j): the mirror of Eq. pl15_11, level n-1. */
static double u_explicit(const orc *o, const level *L, const double *Fy, int i, int j)
{
    double uP = Uc(o, L, i, j);
    double uS = u_at(o, L, i, j, i, j - 1), uN = u_at(o, L, i, j, i, j + 1);
    double uW = Uc(o, L, i - 1, j), uE = Uc(o, L, i + 1, j);
    double Fs1 = Fy[FV(o, i - 1, j)], Fs2 = Fy[FV(o, i, j)];
    double Fn1 = Fy[FV(o, i - 1, j + 1)], Fn2 = Fy[FV(o, i, j + 1)];
    double vs1 = Vc(o, L, i - 1, j), vs2 = Vc(o, L, i, j);
    double vn1 = Vc(o, L, i - 1, j + 1), vn2 = Vc(o, L, i, j + 1);
    double ubar_w = 0.5 * (uW + uP), ubar_e = 0.5 * (uP + uE);
    double pn1 = 0, pn2 = 0, ps1 = 0, ps2 = 0, pe = 0, pw = 0;
    if (tvd_u_y(o, i, j + 1)) {
        double f1 = Uc(o, L, i, j - 1), f4 = Uc(o, L, i, j + 2);
        pn1 = orc_psi_s(f1, uP, uN, f4, DY(o, j - 1), DY(o, j), DY(o, j + 1), DY(o, j + 2), vn1);
        pn2 = orc_psi_s(f1, uP, uN, f4, DY(o, j - 1), DY(o, j), DY(o, j + 1), DY(o, j + 2), vn2);
    }
    if (tvd_u_y(o, i, j)) {
        double f1 = Uc(o, L, i, j - 2);
        ps1 = orc_psi_s(f1, uS, uP, uN, DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vs1);
        ps2 = orc_psi_s(f1, uS, uP, uN, DY(o, j - 2), DY(o, j - 1), DY(o, j), DY(o, j + 1), vs2);
    }
    if (tvd_u_x(o, i + 1, j))
        pe = orc_psi_c(uW, uP, uE, Uc(o, L, i + 2, j), DX(o, i - 1), DX(o, i), DX(o, i + 1), ubar_e);
    if (tvd_u_x(o, i, j))
        pw = orc_psi_c(Uc(o, L, i - 2, j), uW, uP, uE, DX(o, i - 2), DX(o, i - 1), DX(o, i), ubar_w);
    return -0.5 * (Fn1 * (upwind(uP, uN, vn1) + (uN - uP) * pn1)
                   + Fn2 * (upwind(uP, uN, vn2) + (uN - uP) * pn2))
           + 0.5 * (Fs1 * (upwind(uS, uP, vs1) + (uP - uS) * ps1)
                    + Fs2 * (upwind(uS, uP, vs2) + (uP - uS) * ps2))
           - DY(o, j) * RHOc(o, L, i, j) * ubar_e * (upwind(uP, uE, ubar_e) + (uE - uP) * pe)
           + DY(o, j) * RHOc(o, L, i - 1, j) * ubar_w * (upwind(uW, uP, ubar_w) + (uP - uW) * pw);
}

static void explicit_terms(orc *o, const level *prev)
{
    int i, j;
    compute_fluxes(o, prev, NULL, NULL, o->Fx_prev, o->Fy_prev);
    ROWS
    for (j = 0; j < o->ny; j++)
        for (i = 0; i < o->nx; i++)
            o->Texp[FC(o, i, j)] = fluid(o, i, j) ? T_explicit(o, prev, o->Fx_prev, o->Fy_prev, i, j) : 0.0;
    ROWS
    for (j = 0; j < o->ny; j++)
        for (i = 0; i <= o->nx; i++)
            o->Uexp[FU(o, i, j)] = u_active(o, i, j) ? u_explicit(o, prev, o->Fy_prev, i, j) : 0.0;
    ROWS
    for (j = 0; j <= o->ny; j++)
        for (i = 0; i < o->nx; i++)
            o->Vexp[FV(o, i, j)] = v_active(o, i, j) ? v_explicit(o, prev, o->Fx_prev, i, j) : 0.0;
}

/* ------------------------------------------------------------ temperature */

/* Energy source S^T_c of cell (i,j), Eq. pl29 (S^T_p = 0, Eq. pl28), from
 * level L. Velocities off their nodes are bilinear interpolations. */
static double energy_source(const orc *o, const level *L, int i, int j)
{
    const orc_coeffs *k = &o->k;
    double dxi = DX(o, i), dyj = DY(o, j);
    double dudx = (Uc(o, L, i + 1, j) - Uc(o, L, i, j)) / dxi;
    double dvdy = (Vc(o, L, i, j + 1) - Vc(o, L, i, j)) / dyj;
    /* v at (x^f_i, y^v_j) and (x^f_{i+1}, y^v_j) */
    double wl = DX(o, i) / (DX(o, i - 1) + DX(o, i)), wr = DX(o, i - 1) / (DX(o, i - 1) + DX(o, i));
    double vw = 0.5 * ((wl * v_at(o, L, i, j, i - 1, j) + wr * Vc(o, L, i, j))
                       + (wl * v_at(o, L, i, j + 1, i - 1, j + 1) + wr * Vc(o, L, i, j + 1)));
    double wl2 = DX(o, i + 1) / (DX(o, i) + DX(o, i + 1)), wr2 = DX(o, i) / (DX(o, i) + DX(o, i + 1));
    double ve = 0.5 * ((wl2 * Vc(o, L, i, j) + wr2 * v_at(o, L, i, j, i + 1, j))
                       + (wl2 * Vc(o, L, i, j + 1) + wr2 * v_at(o, L, i, j + 1, i + 1, j + 1)));
    /* u at (x^v_i, y^f_j) and (x^v_i, y^f_{j+1}) */
    double wb = DY(o, j) / (DY(o, j - 1) + DY(o, j)), wt = DY(o, j - 1) / (DY(o, j - 1) + DY(o, j));
    double us = 0.5 * ((wb * u_at(o, L, i, j, i, j - 1) + wt * Uc(o, L, i, j))
                       + (wb * u_at(o, L, i + 1, j, i + 1, j - 1) + wt * Uc(o, L, i + 1, j)));
    double wb2 = DY(o, j + 1) / (DY(o, j) + DY(o, j + 1)), wt2 = DY(o, j) / (DY(o, j) + DY(o, j + 1));
    double un = 0.5 * ((wb2 * Uc(o, L, i, j) + wt2 * u_at(o, L, i, j, i, j + 1))
                       + (wb2 * Uc(o, L, i + 1, j) + wt2 * u_at(o, L, i + 1, j, i + 1, j + 1)));
    double dvdx = (ve - vw) / dxi;
    double dudy = (un - us) / dyj;
    double div = dudx + dvdy;
    double phi = 2.0 * (dudx * dudx + dvdy * dvdy) + (dvdx + dudy) * (dvdx + dudy)
                 - 2.0 / 3.0 * div * div;
    return k->CT2f * GAMc(o, L, i, j) * phi * dxi * dyj + k->CT3f * Pc(o, L, i, j) * div * dxi * dyj;
}

/* New temperature of fluid cell (i,j), Eqs. pl30-pl33 (implicit) or pl30,
 * pl31_1, pl32, pl33 (explicit). */
static double temperature(const orc *o, const level *prev, const level *old, int i, int j)
{
    const orc_coeffs *k = &o->k;
    double dt = k->dt, dxi = DX(o, i), dyj = DY(o, j);
    double Tp = Tc(o, old, i, j);
    double Tw = T_at(o, old, i, j, i - 1, j), Te = T_at(o, old, i, j, i + 1, j);
    double Ts = T_at(o, old, i, j, i, j - 1), Tn = T_at(o, old, i, j, i, j + 1);
    double Fw = o->Fx[FU(o, i, j)], Fe = o->Fx[FU(o, i + 1, j)];
    double Fs = o->Fy[FV(o, i, j)], Fn = o->Fy[FV(o, i, j + 1)];
    double gp = GAMc(o, old, i, j);
    double gw = orc_gam_harmonic(GAMc(o, old, i - 1, j), gp, DX(o, i - 1), dxi);
    double ge = orc_gam_harmonic(gp, GAMc(o, old, i + 1, j), dxi, DX(o, i + 1));
    double gs = orc_gam_harmonic(GAMc(o, old, i, j - 1), gp, DY(o, j - 1), dyj);
    double gn = orc_gam_harmonic(gp, GAMc(o, old, i, j + 1), dyj, DY(o, j + 1));
    double Dw = k->CT1f * gw * dyj / (0.5 * (dxi + DX(o, i - 1)));
    double De = k->CT1f * ge * dyj / (0.5 * (DX(o, i + 1) + dxi));
    double Ds = k->CT1f * gs * dxi / (0.5 * (dyj + DY(o, j - 1)));
    double Dn = k->CT1f * gn * dxi / (0.5 * (DY(o, j + 1) + dyj));
    double a1, a2, a3, a4, a0, Texp, Sc, rhs;

    if (o->P->implicit) {
        double pw = 0, pe = 0, ps = 0, pn = 0;
        if (tvd_cells_x(o, i, j))
            pw = orc_psi_s(Tc(o, old, i - 2, j), Tw, Tp, Te,
                           DX(o, i - 2), DX(o, i - 1), dxi, DX(o, i + 1), Uc(o, old, i, j));
        if (tvd_cells_x(o, i + 1, j))
            pe = orc_psi_s(Tw, Tp, Te, Tc(o, old, i + 2, j),
                           DX(o, i - 1), dxi, DX(o, i + 1), DX(o, i + 2), Uc(o, old, i + 1, j));
        if (tvd_cells_y(o, i, j))
            ps = orc_psi_s(Tc(o, old, i, j - 2), Ts, Tp, Tn,
                           DY(o, j - 2), DY(o, j - 1), dyj, DY(o, j + 1), Vc(o, old, i, j));
        if (tvd_cells_y(o, i, j + 1))
            pn = orc_psi_s(Ts, Tp, Tn, Tc(o, old, i, j + 2),
                           DY(o, j - 1), dyj, DY(o, j + 1), DY(o, j + 2), Vc(o, old, i, j + 1));
        a1 = maxd(0.0, Fw) - Fw * pw + Dw;
        a2 = maxd(0.0, -Fe) - Fe * pe + De;
        a3 = maxd(0.0, Fs) - Fs * ps + Ds;
        a4 = maxd(0.0, -Fn) - Fn * pn + Dn;
        a0 = dt * (a1 + a2 + a3 + a4 + Fe - Fw + Fn - Fs) + RHOc(o, old, i, j) * dxi * dyj;
        Texp = 0.0;
    } else {
        a1 = Dw; a2 = De; a3 = Ds; a4 = Dn;
        a0 = dt * (a1 + a2 + a3 + a4) + RHOc(o, old, i, j) * dxi * dyj;
        Texp = o->Texp[FC(o, i, j)];
    }
    Sc = energy_source(o, old, i, j);
    rhs = dt * (a1 * Tw + a2 * Te + a3 * Ts + a4 * Tn + Sc + Texp)
          + RHOc(o, prev, i, j) * Tc(o, prev, i, j) * dxi * dyj;
    return rhs / a0;
}

/* ------------------------------------------------------- pseudo velocities */

/* u^ and d^u of active u node (i,j): the mirror image of Eqs. pl14-pl16, pl20
 * (and of pl15_11 for the explicit coefficients). */
static void pseudo_u(const orc *o, const level *prev, const level *old, int i, int j,
                     double *uhat, double *du)
{
    const orc_coeffs *k = &o->k;
    double dt = k->dt, B = k->B;
    double dxw = DX(o, i - 1), dxp = DX(o, i), dyj = DY(o, j);
    double uP = Uc(o, old, i, j);
    double uW = u_at(o, old, i, j, i - 1, j), uE = u_at(o, old, i, j, i + 1, j);
    double uS = u_at(o, old, i, j, i, j - 1), uN = u_at(o, old, i, j, i, j + 1);
    double ubar_w = 0.5 * (uW + uP), ubar_e = 0.5 * (uP + uE);
    double Fbar_w = ubar_w * RHOc(o, old, i - 1, j) * dyj;
    double Fbar_e = ubar_e * RHOc(o, old, i, j) * dyj;
    double Fs1 = o->Fy[FV(o, i - 1, j)], Fs2 = o->Fy[FV(o, i, j)];
    double Fn1 = o->Fy[FV(o, i - 1, j + 1)], Fn2 = o->Fy[FV(o, i, j + 1)];
    double Dx_w = B * GAMc(o, old, i - 1, j) * dyj / dxw;
    double Dx_e = B * GAMc(o, old, i, j) * dyj / dxp;
    double Dy_s = B * gam_corner(o, old, i, j) * (dxp + dxw) / (dyj + DY(o, j - 1));
    double Dy_n = B * gam_corner(o, old, i, j + 1) * (dxp + dxw) / (DY(o, j + 1) + dyj);
    double trans = (RHOc(o, old, i, j) * dxp + RHOc(o, old, i - 1, j) * dxw) * dyj / (2.0 * dt);
    double b = (RHOc(o, prev, i, j) * dxp + RHOc(o, prev, i - 1, j) * dxw) * dyj / (2.0 * dt) * Uc(o, prev, i, j)
             + B * (gam_corner(o, old, i, j + 1) * (Vc(o, old, i, j + 1) - Vc(o, old, i - 1, j + 1))
                    - gam_corner(o, old, i, j) * (Vc(o, old, i, j) - Vc(o, old, i - 1, j))
                    - 2.0 / 3.0 * GAMc(o, old, i, j) * (Vc(o, old, i, j + 1) - Vc(o, old, i, j))
                    + 2.0 / 3.0 * GAMc(o, old, i - 1, j) * (Vc(o, old, i - 1, j + 1) - Vc(o, old, i - 1, j)))
             + o->P->gx * (RHOc(o, old, i, j) * dxp + RHOc(o, old, i - 1, j) * dxw) * dyj / 2.0;
    double a1, a2, a3, a4, a0, uexp;

    if (o->P->implicit) {
        double pw = 0, pe = 0, ps1 = 0, ps2 = 0, pn1 = 0, pn2 = 0;
        if (tvd_u_x(o, i, j))
            pw = orc_psi_c(Uc(o, old, i - 2, j), uW, uP, uE, DX(o, i - 2), dxw, dxp, ubar_w);
        if (tvd_u_x(o, i + 1, j))
            pe = orc_psi_c(uW, uP, uE, Uc(o, old, i + 2, j), dxw, dxp, DX(o, i + 1), ubar_e);
        if (tvd_u_y(o, i, j)) {
            double f1 = Uc(o, old, i, j - 2);
            ps1 = orc_psi_s(f1, uS, uP, uN, DY(o, j - 2), DY(o, j - 1), dyj, DY(o, j + 1), Vc(o, old, i - 1, j));
            ps2 = orc_psi_s(f1, uS, uP, uN, DY(o, j - 2), DY(o, j - 1), dyj, DY(o, j + 1), Vc(o, old, i, j));
        }
        if (tvd_u_y(o, i, j + 1)) {
            double f4 = Uc(o, old, i, j + 2);
            pn1 = orc_psi_s(uS, uP, uN, f4, DY(o, j - 1), dyj, DY(o, j + 1), DY(o, j + 2), Vc(o, old, i - 1, j + 1));
            pn2 = orc_psi_s(uS, uP, uN, f4, DY(o, j - 1), dyj, DY(o, j + 1), DY(o, j + 2), Vc(o, old, i, j + 1));
        }
        a1 = maxd(0.0, Fbar_w) - Fbar_w * pw + 4.0 / 3.0 * Dx_w;
        a2 = maxd(0.0, -Fbar_e) - Fbar_e * pe + 4.0 / 3.0 * Dx_e;
        a3 = 0.5 * (maxd(0.0, Fs1) - Fs1 * ps1 + maxd(0.0, Fs2) - Fs2 * ps2) + Dy_s;
        a4 = 0.5 * (maxd(0.0, -Fn1) - Fn1 * pn1 + maxd(0.0, -Fn2) - Fn2 * pn2) + Dy_n;
        a0 = a1 + a2 + a3 + a4 + 0.5 * (Fn2 - Fs2 + Fn1 - Fs1) + Fbar_e - Fbar_w + trans;
        uexp = 0.0;
    } else {
        a1 = 4.0 / 3.0 * Dx_w; a2 = 4.0 / 3.0 * Dx_e; a3 = Dy_s; a4 = Dy_n;
        a0 = a1 + a2 + a3 + a4 + trans;
        uexp = o->Uexp[FU(o, i, j)];
    }
    *uhat = (a1 * uW + a2 * uE + a3 * uS + a4 * uN + b + uexp) / a0;
    *du = k->A * dyj / a0;
}

/* v^ and d^v of active v node (i,j), Eqs. pl14-pl16, pl21 (implicit) and
 * pl15_11 (explicit). */
static void pseudo_v(const orc *o, const level *prev, const level *old, int i, int j,
                     double *vhat, double *dv)
{
    const orc_coeffs *k = &o->k;
    double dt = k->dt, B = k->B;
    double dys = DY(o, j - 1), dyp = DY(o, j), dxi = DX(o, i);
    double vP = Vc(o, old, i, j);
    double vW = v_at(o, old, i, j, i - 1, j), vE = v_at(o, old, i, j, i + 1, j);
    double vS = v_at(o, old, i, j, i, j - 1), vN = v_at(o, old, i, j, i, j + 1);
    double vbar_s = 0.5 * (vS + vP), vbar_n = 0.5 * (vP + vN);
    double Fbar_s = vbar_s * RHOc(o, old, i, j - 1) * dxi;
    double Fbar_n = vbar_n * RHOc(o, old, i, j) * dxi;
    double Fw1 = o->Fx[FU(o, i, j - 1)], Fw2 = o->Fx[FU(o, i, j)];
    double Fe1 = o->Fx[FU(o, i + 1, j - 1)], Fe2 = o->Fx[FU(o, i + 1, j)];
    double Dx_w = B * gam_corner(o, old, i, j) * (dyp + dys) / (dxi + DX(o, i - 1));
    double Dx_e = B * gam_corner(o, old, i + 1, j) * (dyp + dys) / (DX(o, i + 1) + dxi);
    double Dy_s = B * GAMc(o, old, i, j - 1) * dxi / dys;
    double Dy_n = B * GAMc(o, old, i, j) * dxi / dyp;
    double trans = (RHOc(o, old, i, j) * dyp + RHOc(o, old, i, j - 1) * dys) * dxi / (2.0 * dt);
    double b = (RHOc(o, prev, i, j) * dyp + RHOc(o, prev, i, j - 1) * dys) * dxi / (2.0 * dt) * Vc(o, prev, i, j)
             + B * (gam_corner(o, old, i + 1, j) * (Uc(o, old, i + 1, j) - Uc(o, old, i + 1, j - 1))
                    - gam_corner(o, old, i, j) * (Uc(o, old, i, j) - Uc(o, old, i, j - 1))
                    - 2.0 / 3.0 * GAMc(o, old, i, j) * (Uc(o, old, i + 1, j) - Uc(o, old, i, j))
                    + 2.0 / 3.0 * GAMc(o, old, i, j - 1) * (Uc(o, old, i + 1, j - 1) - Uc(o, old, i, j - 1)))
             + o->P->gy * (RHOc(o, old, i, j) * dyp + RHOc(o, old, i, j - 1) * dys) * dxi / 2.0;
    double a1, a2, a3, a4, a0, vexp;

    if (o->P->implicit) {
        double pw1 = 0, pw2 = 0, pe1 = 0, pe2 = 0, ps = 0, pn = 0;
        if (tvd_v_x(o, i, j)) {
            double f1 = Vc(o, old, i - 2, j);
            pw1 = orc_psi_s(f1, vW, vP, vE, DX(o, i - 2), DX(o, i - 1), dxi, DX(o, i + 1), Uc(o, old, i, j - 1));
            pw2 = orc_psi_s(f1, vW, vP, vE, DX(o, i - 2), DX(o, i - 1), dxi, DX(o, i + 1), Uc(o, old, i, j));
        }
        if (tvd_v_x(o, i + 1, j)) {
            double f4 = Vc(o, old, i + 2, j);
            pe1 = orc_psi_s(vW, vP, vE, f4, DX(o, i - 1), dxi, DX(o, i + 1), DX(o, i + 2), Uc(o, old, i + 1, j - 1));
            pe2 = orc_psi_s(vW, vP, vE, f4, DX(o, i - 1), dxi, DX(o, i + 1), DX(o, i + 2), Uc(o, old, i + 1, j));
        }
        if (tvd_v_y(o, i, j))
            ps = orc_psi_c(Vc(o, old, i, j - 2), vS, vP, vN, DY(o, j - 2), dys, dyp, vbar_s);
        if (tvd_v_y(o, i, j + 1))
            pn = orc_psi_c(vS, vP, vN, Vc(o, old, i, j + 2), dys, dyp, DY(o, j + 1), vbar_n);
        a1 = 0.5 * (maxd(0.0, Fw2) - Fw2 * pw2 + maxd(0.0, Fw1) - Fw1 * pw1) + Dx_w;
        a2 = 0.5 * (maxd(0.0, -Fe2) - Fe2 * pe2 + maxd(0.0, -Fe1) - Fe1 * pe1) + Dx_e;
        a3 = maxd(0.0, Fbar_s) - Fbar_s * ps + 4.0 / 3.0 * Dy_s;
        a4 = maxd(0.0, -Fbar_n) - Fbar_n * pn + 4.0 / 3.0 * Dy_n;
        a0 = a1 + a2 + a3 + a4 + 0.5 * (Fe2 - Fw2 + Fe1 - Fw1) + Fbar_n - Fbar_s + trans;
        vexp = 0.0;
    } else {
        a1 = Dx_w; a2 = Dx_e; a3 = 4.0 / 3.0 * Dy_s; a4 = 4.0 / 3.0 * Dy_n;
        a0 = a1 + a2 + a3 + a4 + trans;
        vexp = o->Vexp[FV(o, i, j)];
    }
    *vhat = (a1 * vW + a2 * vE + a3 * vS + a4 * vN + b + vexp) / a0;
    *dv = k->A * dxi / a0;
}

/* ---------------------------------------------------------------- pressure */

/* New pressure of fluid cell (i,j), Eqs. pl23, pl24, with the new T. */
static double pressure(const orc *o, const level *prev, const level *old, double Tnew, int i, int j)
{
    double dt = o->k.dt, dxi = DX(o, i), dyj = DY(o, j);
    int fw = FU(o, i, j), fe = FU(o, i + 1, j), fs = FV(o, i, j), fn = FV(o, i, j + 1);
    double apx_w = o->rho_u[fw] * o->du[fw] * dyj, apx_e = o->rho_u[fe] * o->du[fe] * dyj;
    double apy_s = o->rho_v[fs] * o->dv[fs] * dxi, apy_n = o->rho_v[fn] * o->dv[fn] * dxi;
    double bpx_w = o->rho_u[fw] * o->uhat[fw] * dyj, bpx_e = o->rho_u[fe] * o->uhat[fe] * dyj;
    double bpy_s = o->rho_v[fs] * o->vhat[fs] * dxi, bpy_n = o->rho_v[fn] * o->vhat[fn] * dxi;
    double ap0 = 1.0 / Tnew * dxi * dyj + (apx_w + apx_e + apy_s + apy_n) * dt;
    double bp = RHOc(o, prev, i, j) * dxi * dyj - (bpx_e - bpx_w + bpy_n - bpy_s) * dt;
    return ((apx_w * Pc(o, old, i - 1, j) + apx_e * Pc(o, old, i + 1, j)
             + apy_s * Pc(o, old, i, j - 1) + apy_n * Pc(o, old, i, j + 1)) * dt + bp) / ap0;
}

/* ------------------------------------------------------------ one iteration */

static void iterate(orc *o, const level *prev, const level *old, level *nw, double *res)
{
    int nx = o->nx, ny = o->ny, i, j;
    double ru = 0, rv = 0, rp = 0, rT = 0;

    copy_level(o, nw, old);

    /* face densities and mass fluxes from the previous iterate */
    compute_fluxes(o, old, o->rho_u, o->rho_v, o->Fx, o->Fy);

    /* energy */
    ROWS
    for (j = 0; j < ny; j++)
        for (i = 0; i < nx; i++)
            if (fluid(o, i, j))
                nw->T[CI(o, i, j)] = temperature(o, prev, old, i, j);

    /* pseudo velocities; faces that are not unknowns keep their stored
     * velocity and d = 0 */
    ROWS
    for (j = 0; j < ny; j++)
        for (i = 0; i <= nx; i++) {
            int f = FU(o, i, j);
            if (u_active(o, i, j)) {
                pseudo_u(o, prev, old, i, j, &o->uhat[f], &o->du[f]);
            } else {
                o->uhat[f] = Uc(o, old, i, j);
                o->du[f] = 0.0;
            }
        }
    ROWS
    for (j = 0; j <= ny; j++)
        for (i = 0; i < nx; i++) {
            int f = FV(o, i, j);
            if (v_active(o, i, j)) {
                pseudo_v(o, prev, old, i, j, &o->vhat[f], &o->dv[f]);
            } else {
                o->vhat[f] = Vc(o, old, i, j);
                o->dv[f] = 0.0;
            }
        }

    /* pressure */
    ROWS
    for (j = 0; j < ny; j++)
        for (i = 0; i < nx; i++)
            if (fluid(o, i, j))
                nw->p[CI(o, i, j)] = pressure(o, prev, old, nw->T[CI(o, i, j)], i, j);

    /* velocity corrections, Eqs. pl18, pl19 */
    ROWS
    for (j = 0; j < ny; j++)
        for (i = 0; i <= nx; i++)
            if (u_active(o, i, j)) {
                int f = FU(o, i, j);
                nw->u[UI(o, i, j)] = o->uhat[f] - o->du[f] * (Pc(o, nw, i, j) - Pc(o, nw, i - 1, j));
            }
    ROWS
    for (j = 0; j <= ny; j++)
        for (i = 0; i < nx; i++)
            if (v_active(o, i, j)) {
                int f = FV(o, i, j);
                nw->v[VI(o, i, j)] = o->vhat[f] - o->dv[f] * (Pc(o, nw, i, j) - Pc(o, nw, i, j - 1));
            }

    /* equation of state and diffusion coefficient */
    ROWS
    for (j = 0; j < ny; j++)
        for (i = 0; i < nx; i++)
            if (fluid(o, i, j)) {
                int c = CI(o, i, j);
                nw->rho[c] = nw->p[c] / nw->T[c];
                nw->gam[c] = gamma_of_T(o, nw->T[c]);
            }

    ghost_fill(o, nw);

    /* maximum residuals over the unknowns */
    for (j = 0; j < ny; j++)
        for (i = 0; i <= nx; i++)
            if (u_active(o, i, j)) {
                double d = fabs(Uc(o, nw, i, j) - Uc(o, old, i, j));
                if (d > ru || d != d) ru = d != d ? d : maxd(ru, d);
            }
    for (j = 0; j <= ny; j++)
        for (i = 0; i < nx; i++)
            if (v_active(o, i, j)) {
                double d = fabs(Vc(o, nw, i, j) - Vc(o, old, i, j));
                if (d > rv || d != d) rv = d != d ? d : maxd(rv, d);
            }
    for (j = 0; j < ny; j++)
        for (i = 0; i < nx; i++)
            if (fluid(o, i, j)) {
                double dp = fabs(Pc(o, nw, i, j) - Pc(o, old, i, j));
                double dT = fabs(Tc(o, nw, i, j) - Tc(o, old, i, j));
                if (dp > rp || dp != dp) rp = dp != dp ? dp : maxd(rp, dp);
                if (dT > rT || dT != dT) rT = dT != dT ? dT : maxd(rT, dT);
            }
    res[0] = ru; res[1] = rv; res[2] = rp; res[3] = rT;
}

/* --------------------------------------------------------------- public API */

int orc_init(const orc_problem *P, double *u, double *v, double *p, double *T)
{
    orc o;
    int rc = orc_alloc(&o, P), nx, ny, i, j;
    if (rc) { orc_free(&o); return rc; }
    nx = P->nx; ny = P->ny;
    /* fluid starts at the inflow state of its row (at rest, T = p = 1 when the
     * west side is not an inflow), plus the seeded perturbation */
    for (j = 0; j < ny; j++)
        for (i = 0; i <= nx; i++) {
            double base = P->side_kind[ORC_W] == ORC_BC_INFLOW ? inflow_u(&o, j) : 0.0;
            double val = 0.0;
            if (u_active(&o, i, j))
                val = base * (1.0 + P->perturb * orc_splitmix_uniform(P->seed, 0, i, j));
            u[FU(&o, i, j)] = val;
        }
    for (j = 0; j <= ny; j++)
        for (i = 0; i < nx; i++) {
            double val = 0.0;
            if (v_active(&o, i, j))
                val = P->perturb * o.k.u_in * orc_splitmix_uniform(P->seed, 1, i, j);
            v[FV(&o, i, j)] = val;
        }
    for (j = 0; j < ny; j++)
        for (i = 0; i < nx; i++) {
            double pb = 1.0, Tb = 1.0;
            if (P->side_kind[ORC_W] == ORC_BC_INFLOW) { pb = inflow_p(&o, j); Tb = inflow_T(&o, j); }
            if (fluid(&o, i, j)) {
                pb = pb * (1.0 + P->perturb * orc_splitmix_uniform(P->seed, 2, i, j));
                Tb = Tb * (1.0 + P->perturb * orc_splitmix_uniform(P->seed, 3, i, j));
            }
            p[FC(&o, i, j)] = pb;
            T[FC(&o, i, j)] = Tb;
        }
    /* round trip through a level so boundary nodes carry their rule values */
    load_level(&o, &o.lv[0], u, v, p, T);
    store_level(&o, &o.lv[0], u, v, p, T);
    orc_free(&o);
    return 0;
}

int orc_run(const orc_problem *P, double *u, double *v, double *p, double *T,
            int nsteps, double *res, int *iters_last)
{
    orc o;
    int rc = orc_alloc(&o, P), step, it = 0, cur;
    double r[4] = {0, 0, 0, 0};
    if (rc) { orc_free(&o); return rc; }
    if (nsteps < 0) { orc_free(&o); return 1; }

    /* level 0 holds n-1 (the state at the start of the step) */
    load_level(&o, &o.lv[0], u, v, p, T);
    copy_level(&o, &o.lv[1], &o.lv[0]);
    copy_level(&o, &o.lv[2], &o.lv[0]);
    cur = 0;
    for (step = 0; step < nsteps; step++) {
        int prev = cur, old = cur, nw;
        if (!P->implicit)
            explicit_terms(&o, &o.lv[prev]);
        for (it = 1; it <= P->iters; it++) {
            double mx;
            nw = (old + 1) % 3;
            if (nw == prev) nw = (nw + 1) % 3;
            iterate(&o, &o.lv[prev], &o.lv[old], &o.lv[nw], r);
            old = nw;
            mx = maxd(maxd(r[0], r[1]), maxd(r[2], r[3]));
            if (r[0] != r[0] || r[1] != r[1] || r[2] != r[2] || r[3] != r[3] || isinf(mx)) {
                store_level(&o, &o.lv[old], u, v, p, T);
                if (res) memcpy(res, r, sizeof r);
                if (iters_last) *iters_last = it;
                orc_free(&o);
                return 3;
            }
            if (P->tol > 0.0 && mx <= P->tol)
                break;
        }
        if (it > P->iters) it = P->iters;
        cur = old;
    }
    store_level(&o, &o.lv[cur], u, v, p, T);
    if (res) memcpy(res, r, sizeof r);
    if (iters_last) *iters_last = it;
    orc_free(&o);
    return 0;
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
