/*
 * simplets.h -- C ABI of the GB300 implementation of the SIMPLE-TS time step
 * (K. S. Shterev, "GPU implementation of algorithm SIMPLE-TS for calculation
 * of unsteady, viscous, compressible and heat-conductive gas flows",
 * arXiv:1802.04243).
 *
 * The library advances the 2D Navier-Stokes-Fourier system of Section 2
 * (Eqs. pl4, pl2, pl3, pl6, pl5) on a staggered Cartesian finite-volume grid
 * (Section 3.2, "Cell volume") with the SIMPLE-TS Jacobi iteration of
 * Section 3.1 (Figs. 1 and 2, GPU column).  Every step of the sweep runs in
 * the library's CUDA kernels on the device; the host only enqueues work.
 *
 * Conventions
 *  - Every call returns a sim_status; nothing throws across the ABI.
 *  - A sim_t owns all the device memory it uses; the caller owns every host
 *    pointer it passes.  Input arrays are read during the call only.
 *  - Host field arrays are row-major with x fastest, in the logical shape
 *    (no ghost cells):  u: ny x (nx+1)   (u[j*(nx+1)+i], face i of row j)
 *                       v: (ny+1) x nx   (v[j*nx+i], face j of column i)
 *                       p, T, rho, Gamma: ny x nx.
 *  - Lengths are in units of the obstacle side, velocities in units of
 *    sqrt(2 R T0), p and T in units of the inflow pressure and the wall
 *    temperature (Section 4).
 *  - sim_step is asynchronous on the stream given to sim_create (NULL: the
 *    legacy default stream); sim_fields, sim_residuals, sim_set_fields and
 *    sim_destroy synchronise with it.
 *  - After SIM_EDIVERGED the handle is in an error state; every call except
 *    sim_set_fields, sim_fields, sim_last_error and sim_destroy then returns
 *    SIM_ESTATE.  sim_set_fields of all four fields clears the state.
 */
#ifndef SIMPLETS_H
#define SIMPLETS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sim_s *sim_t;

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = 1,      /* invalid argument or problem description */
    SIM_ENOMEM = 2,      /* device or pinned host allocation failed */
    SIM_ECUDA = 3,       /* a CUDA call failed (see sim_last_error) */
    SIM_EDIVERGED = 4,   /* a residual became NaN or infinite */
    SIM_ETIMEOUT = 5,    /* reserved */
    SIM_ESTATE = 6       /* handle is in the error state after a divergence */
} sim_status;

/* side indices and side kinds */
enum { SIM_W = 0, SIM_E = 1, SIM_S = 2, SIM_N = 3 };
enum { SIM_BC_WALL = 0, SIM_BC_SYMMETRY = 1, SIM_BC_INFLOW = 2, SIM_BC_OUTFLOW = 3 };
/* gas models */
enum { SIM_GAS_IDEAL_RE = 0, SIM_GAS_HARD_SPHERE_KN = 1 };
/* scheme flags for sim_step: time treatment of convection | spatial scheme */
enum { SIM_EXPLICIT = 0, SIM_IMPLICIT = 1, SIM_UPWIND = 0, SIM_TVD = 2 };
/* arithmetic of the sweep */
enum { SIM_FP64 = 0, SIM_MIXED = 1, SIM_DF64 = 2 };
/* field ids */
enum { SIM_FIELD_U = 0, SIM_FIELD_V = 1, SIM_FIELD_P = 2, SIM_FIELD_T = 3,
       SIM_FIELD_RHO = 4, SIM_FIELD_GAMMA = 5 };

/* Grid (Section 3.2): nx x ny cells.  dx/dy give the nx (ny) cell sizes; when
 * NULL the grid is uniform with sizes lx/nx and ly/ny.  nx, ny >= 4. */
typedef struct {
    int nx, ny;
    double lx, ly;
    const double *dx, *dy;
} sim_grid;

/* Gas and flow (Sections 2 and 4).
 * SIM_GAS_IDEAL_RE: gamma, prandtl, visc_exp (Gamma = Gamma^lambda = T^visc_exp),
 *   inflow Mach number and Reynolds number on the obstacle side give
 *   A = 1/2, U_in = M sqrt(gamma/2), B = U_in/Re, C^T1 = B/Pr,
 *   C^T2 = 2B(gamma-1)/gamma, C^T3 = (gamma-1)/gamma.
 * SIM_GAS_HARD_SPHERE_KN: Eq. pl37 with Knudsen number kn (gamma = 5/3,
 *   Pr = 2/3, Gamma = sqrt(T)); mach_in sets U_in.
 * gx, gy: body force per unit mass (the rho g terms of Eqs. pl2, pl3). */
typedef struct {
    int model;
    double gamma, prandtl, visc_exp;
    double mach_in, reynolds, kn;
    double gx, gy;
} sim_gas;

/* Boundaries, obstacles, start state and loop-2 control.
 * side_kind: per side (W, E, S, N).  INFLOW only on W, OUTFLOW only on E;
 *   S and N are WALL or SYMMETRY.  A wall is no-slip and isothermal (the
 *   zeta = tau = 0 limit of Eqs. pl38, pl39) with tangential velocity
 *   side_vel and temperature side_T.
 * Obstacles: n_rect cell rectangles [i0, j0, i1, j1) (4 ints each), at
 *   least 2 cells wide and at least 2 cells from every side; body_T is their
 *   wall temperature.
 * inflow_u/T/p: optional per-row inflow profile (ny entries); default
 *   U_in, 1, 1.
 * dt: time step; <= 0 selects cfl * min(dx, dy) / (U_ref + sqrt(gamma/2))
 *   with cfl (default 0.2 when <= 0).
 * iters: loop-2 iterations per step (>= 1); tol > 0 ends loop 2 early once
 *   every residual <= tol (this reads the residuals back every iteration).
 * seed, perturb: start state = inflow state of the row (rest when W is not an
 *   inflow) times (1 + perturb xi), xi in [-1, 1) from splitmix64 of
 *   (seed ^ (field<<40 + j<<20 + i)); v = perturb U_in xi.
 * precision: SIM_FP64; SIM_MIXED (FP32 assembly and relaxation, FP64
 *   pressure accumulation, equation of state and residuals; u, v, T and
 *   Gamma are FP32 values, widened into the FP64 state when read); SIM_DF64 (every
 *   kernel of the iteration in double-float arithmetic -- pairs of floats,
 *   about 48 significant bits -- on the FP32 pipe; the FP64 state is filled
 *   from it when read, and the residual maxima carry FP32 precision).
 * zeta_coef, tau_coef: velocity-slip and temperature-jump walls (Eqs. pl38,
 *   pl39), u_s - u_w = zeta du/dn and T_s - T_w = tau dT/dn with
 *   zeta = zeta_coef / rho_local and tau = tau_coef / rho_local (the paper's
 *   hard-sphere gas: 1.1466 Kn and 2.1904 Kn).  They apply at every wall side
 *   and obstacle; a tangential velocity slips, the normal one stays zero.
 *   0 gives no-slip isothermal walls; negative values are rejected. */
typedef struct {
    int side_kind[4];
    double side_vel[4];
    double side_T[4];
    double body_T;
    int n_rect;
    const int *rect;
    const double *inflow_u, *inflow_T, *inflow_p;
    double dt, cfl;
    int iters;
    double tol;
    uint64_t seed;
    double perturb;
    int precision;
    double zeta_coef, tau_coef;
} sim_bc;

/* Validate the problem, allocate every device buffer and set the start state.
 * stream: a cudaStream_t (may be NULL).  On success *out owns the handle.
 * Grids: 4 <= nx, ny < 2^20 and at most 2^31 - 1 elements in the padded grid
 * ((nx + 5) rounded up to a multiple of 8, times ny + 5).
 * Errors: SIM_EINVAL (bad description), SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_create(const sim_grid *grid, const sim_gas *gas, const sim_bc *bc,
                      void *stream, sim_t *out);

/* Advance n_steps time steps (Section 3.1, loop 1) with `scheme`
 * (SIM_EXPLICIT or SIM_IMPLICIT, or-ed with SIM_UPWIND or SIM_TVD).  Each step
 * runs the explicit convective terms (explicit scheme only; Eqs. pl15_11,
 * pl31_1) and then `iters` loop-2 iterations: face densities (Eqs. pl8-pl11),
 * temperature (Eqs. pl28-pl33), pseudo velocities (Eqs. pl14-pl16, pl20,
 * pl21), pressure (Eqs. pl23, pl24), velocity correction (Eqs. pl18, pl19),
 * rho = p/T (Eq. pl5) and the residual reduction.  Asynchronous unless
 * tol > 0.  Errors: SIM_EINVAL (n_steps < 0, bad scheme), SIM_ECUDA,
 * SIM_EDIVERGED (tol > 0 only), SIM_ESTATE. */
sim_status sim_step(sim_t sim, int n_steps, int scheme);

/* Copy one field of the current state into host_dst (n doubles, the logical
 * shape of that field, boundary values included).  Synchronous.
 * Errors: SIM_EINVAL (bad field or n), SIM_ECUDA. */
sim_status sim_fields(sim_t sim, int field, double *host_dst, size_t n);

/* Borrow the device array of one field of the current state.  *dev receives
 * the address of element (i, j) = (0, 0); element (i, j) is at
 * dev[j * (*pitch) + i] for -2 <= i, j (two ghost layers).  Valid until the
 * next sim_step, sim_set_fields or sim_destroy.  SIM_DF64 and SIM_MIXED: the
 * FP64 array is refreshed by work queued on the handle's stream (from the
 * double-float state; in SIM_MIXED u, v, T and Gamma from the FP32 values the
 * sweep keeps); synchronise with that stream before reading it elsewhere.
 * Errors: SIM_EINVAL. */
sim_status sim_field_ptr(sim_t sim, int field, void **dev, size_t *pitch);

/* Overwrite the unknowns of one field (u, v, p or T; logical shape) of the
 * current state from host_src; boundary values follow the boundary rules and
 * rho, Gamma are recomputed.  Used for restart.  Synchronous.
 * Errors: SIM_EINVAL, SIM_ECUDA. */
sim_status sim_set_fields(sim_t sim, int field, const double *host_src, size_t n);

/* Overwrite the unknowns of all four fields of the current state from host
 * arrays in the logical shapes (u: (nx+1) x ny, v: nx x (ny+1), p, T: nx x ny;
 * row-major, x fastest), as four sim_set_fields calls would, with one
 * synchronisation: the values are copied to the device and checked there
 * (finite; p, T > 0) before anything changes.  Arrays wholly in page-locked
 * host memory that the device addresses (cudaHostAlloc, cudaHostRegister)
 * are read by one kernel over the host link; other arrays are copied with
 * cudaMemcpyAsync.  On return the host arrays may be reused; the update
 * itself is queued on the handle's stream.  Clears the
 * error state of a diverged handle.  Errors: SIM_EINVAL (null array, or a
 * value not admissible: nothing is changed), SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_set_state(sim_t sim, const double *u, const double *v, const double *p, const double *T);

/* Copy all four fields of the current state into host arrays (logical shapes,
 * boundary values included) and, if res is not NULL, the residuals of the
 * last loop-2 iteration (as sim_residuals), with one synchronisation.
 * Page-locked destination arrays are written by the gather kernel directly;
 * others receive cudaMemcpyAsync copies of a device staging array.
 * Errors: SIM_EINVAL (null array), SIM_ECUDA; SIM_EDIVERGED if a residual is
 * not finite (the fields are copied all the same). */
sim_status sim_get_state(sim_t sim, double *u, double *v, double *p, double *T, double res[4]);

/* Maximum |new - old| of u, v, p, T over the unknowns in the last loop-2
 * iteration (Section 5: the only data read back per iteration), and the
 * number of loop-2 iterations of the last step.  Synchronous.
 * Returns SIM_EDIVERGED if a residual is NaN or infinite. */
sim_status sim_residuals(sim_t sim, double out[4], int *iters_last_step);

/* Non-dimensional coefficients in use: out[0..8] = A, B, C^T1_f, C^T2_f,
 * C^T3_f, omega, U_in, dt, cells.  Errors: SIM_EINVAL. */
sim_status sim_coefficients(sim_t sim, double out[9]);

/* Work distribution of the handle's equation kernels (not part of the method;
 * every distribution gives the same bits): tiles of tile_x x tile_y threads,
 * one grid position per thread, walked by `ctas` CTAs (0: one CTA per tile);
 * the assembly kernel by `asm_ctas` CTAs (0: as the others).
 * tile_x in {16, 32, 64, 128, 256}; tile_x * tile_y in {32, 64, 128, 256}.
 * Defaults (measured on the 4864x1216 channel): SIM_FP64 32 x 4 tiles, one
 * CTA per tile; SIM_MIXED 32 x 8 tiles, one CTA per tile, the assembly on 4
 * CTAs per SM; SIM_DF64 32 x 8, one CTA per tile.
 * Synchronous; the captured step graphs are rebuilt on the next sim_step.
 * Errors: SIM_EINVAL, SIM_ECUDA. */
sim_status sim_set_plan(sim_t sim, int tile_x, int tile_y, int ctas, int asm_ctas);

/* Kernel classes of the sweep, for sim_profile_read. */
enum { SIM_K_FACES = 0, SIM_K_ASSEMBLE = 1, SIM_K_PRESSURE = 2, SIM_K_VELOCITY = 3, SIM_K_GHOSTS = 4,
       SIM_K_EXPLICIT = 5, SIM_K_COUNT = 6 };

/* Measurement hooks (not part of the method).  sim_profile(sim, 1) clears the
 * counters and from then on brackets every kernel launch of sim_step with a
 * pair of CUDA events on the handle's stream (sim_step then launches kernels
 * one by one instead of replaying its captured step graphs);
 * sim_profile(sim, 2) only clears the counters; sim_profile(sim, 0) stops the
 * event timing.  Launches are counted whether or not timing is on.
 * Errors: SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_profile(sim_t sim, int enable);

/* Launches of kernel class `kernel_class` since the last sim_profile(sim, 1)
 * (or since sim_create), and their summed event-timed duration in ms (0 when
 * timing was off).  Synchronous.  Errors: SIM_EINVAL, SIM_ECUDA. */
sim_status sim_profile_read(sim_t sim, int kernel_class, double *ms, long long *launches);

/* Text of the last error on this handle (never NULL). */
const char *sim_last_error(sim_t sim);

/* ------------------------------------------------------------------------
 * Batches: many independent problems advanced together.  The paper solves one
 * channel at a time; a batch runs the same time step (Section 3.1) for n
 * problems of different sizes and parameters with one launch per kernel phase
 * over all of them (a tile list that spans every problem), and replays whole
 * steps as CUDA graphs.  The problems must share the precision and the number
 * of loop-2 iterations, and use tol = 0.
 * ------------------------------------------------------------------------ */
typedef struct sim_batch_s *sim_batch_t;

/* Create n problems (arrays of n descriptions, each as for sim_create) on one
 * stream.  Errors: SIM_EINVAL (n < 1, a bad description, mixed precisions or
 * loop-2 lengths, tol != 0), SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_batch_create(int n, const sim_grid *grids, const sim_gas *gases, const sim_bc *bcs,
                            void *stream, sim_batch_t *out);

/* Advance every problem n_steps time steps with `scheme` (as sim_step).
 * Asynchronous.  Errors: SIM_EINVAL, SIM_ECUDA. */
sim_status sim_batch_step(sim_batch_t batch, int n_steps, int scheme);

/* One field of problem `instance` (as sim_fields).  Synchronous. */
sim_status sim_batch_fields(sim_batch_t batch, int instance, int field, double *host_dst, size_t n);

/* Residuals of problem `instance` in its last loop-2 iteration (as sim_residuals). */
sim_status sim_batch_residuals(sim_batch_t batch, int instance, double out[4]);

/* Autotune the work distribution of the batched kernels for `scheme`: times a
 * few steps for each candidate tile shape (32x8, 64x4, 128x2, 16x16, 32x4,
 * 64x2 threads) and CTA count, keeps the fastest, and restores the state of every problem
 * afterwards.  out[0..2] = tile x, tile y, CTAs.  Synchronous; allocates a
 * temporary copy of the state.  Errors: SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_batch_tune(sim_batch_t batch, int scheme, int out[3]);

/* Set the work distribution of the batched kernels explicitly: tiles of
 * tile_x x tile_y threads (tile_x one of 16, 32, 64, 128, 256 and
 * tile_x * tile_y one of 32, 64, 128, 256) walked by `ctas` CTAs (0: one CTA
 * per tile).  Every distribution gives the same bits.  Synchronous.
 * Errors: SIM_EINVAL (null batch, another shape, ctas < 0), SIM_ECUDA. */
sim_status sim_batch_set_tiles(sim_batch_t batch, int tile_x, int tile_y, int ctas);

/* Run each time step of the batch as one persistent kernel (on != 0) instead
 * of one launch per phase: a cooperative launch of as many CTAs as stay
 * resident walks the tile list through every phase of the step (explicit
 * terms, face densities, assembly, pressure, velocity correction), with a
 * grid-wide barrier between the phases.  The phases run the same code as the
 * per-phase kernels.  The launch and the reset of its barrier are captured as
 * the step's CUDA graph (replayed every step), or launched directly when the
 * runtime refuses to capture the cooperative launch.  Each barrier wait is bounded (2 s): a wait that runs out
 * ends the step, and the next sim_batch_fields or sim_batch_residuals returns
 * SIM_ETIMEOUT.  Not available when a problem has a symmetry side (its ghost
 * refresh is a separate kernel).  sim_batch_tune also times this mode.
 * Synchronous.  Errors: SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_batch_set_persistent(sim_batch_t batch, int on);

/* The batch's work distribution: out[0..3] = tile x, tile y, CTAs of the
 * per-phase kernels, and 0 for one launch per phase, 1 for one persistent
 * kernel per step replayed from a CUDA graph, 2 for one persistent kernel per
 * step launched directly (graph capture refused). */
sim_status sim_batch_plan_info(sim_batch_t batch, int out[4]);

/* Text of the last error on this batch (never NULL). */
const char *sim_batch_last_error(sim_batch_t batch);

/* Release the batch and all its problems (NULL is a no-op). */
void sim_batch_destroy(sim_batch_t batch);

/* Release every resource of the handle (NULL is a no-op). */
void sim_destroy(sim_t sim);

/* ------------------------------------------------------------------------
 * x-strips: one problem decomposed into strips along x (the paper's
 * decomposition axis for several devices, Section 5), advanced on one device.
 * Each strip owns the cell columns [own0, own1) of a nearly equal split and
 * stores its own arrays for the columns it computes: its owned columns and a
 * halo of SIM_STRIP_HALO columns on each side that faces another strip.  Per
 * loop-2 iteration every strip runs the sweep's kernels over its owned
 * columns and its halo (recomputing the halo from the previous iterate), then
 * one kernel copies the new level's halo columns of every field from the
 * strip that owns them; the residual maxima count each strip's owned columns
 * only and are reduced over the strips.  Every owned value is computed by the
 * same arithmetic as in a whole-problem handle, so the fields and residuals
 * equal sim_create + sim_step bit for bit.  tol must be 0.
 * ------------------------------------------------------------------------ */
#define SIM_STRIP_HALO 4
typedef struct sim_strips_s *sim_strips_t;

/* Layout of strip `strip` of `n_strips` over nx cells (host only, no device
 * call): out[0..5] = own0, own1 (owned cell columns [own0, own1)), store0,
 * store1 (stored columns of the extended grid, [store0, store1)), comp0,
 * comp1 (computed grid positions, [comp0, comp1)).  1 <= n_strips <= 64 and
 * nx >= 2 * SIM_STRIP_HALO * n_strips.  Errors: SIM_EINVAL. */
sim_status sim_strips_layout(int nx, int n_strips, int strip, int out[6]);

/* Create the strips of one problem (as for sim_create) on one stream.
 * Errors: SIM_EINVAL (bad description, tol != 0, a layout outside the limits
 * above), SIM_ENOMEM, SIM_ECUDA. */
sim_status sim_strips_create(const sim_grid *grid, const sim_gas *gas, const sim_bc *bc, int n_strips,
                             void *stream, sim_strips_t *out);

/* Advance n_steps time steps with `scheme` (as sim_step); each step is one
 * captured CUDA graph.  Asynchronous.  Errors: SIM_EINVAL, SIM_ECUDA. */
sim_status sim_strips_step(sim_strips_t strips, int n_steps, int scheme);

/* One field of the whole problem, gathered from the strips' owned columns
 * (as sim_fields).  Synchronous.  Errors: SIM_EINVAL, SIM_ECUDA. */
sim_status sim_strips_fields(sim_strips_t strips, int field, double *host_dst, size_t n);

/* Residuals of the last loop-2 iteration over the whole problem (as
 * sim_residuals).  Synchronous.  SIM_EDIVERGED if one is not finite. */
sim_status sim_strips_residuals(sim_strips_t strips, double out[4]);

/* Text of the last error (never NULL). */
const char *sim_strips_last_error(sim_strips_t strips);

/* Release the strips (NULL is a no-op). */
void sim_strips_destroy(sim_strips_t strips);

#ifdef __cplusplus
}
#endif
#endif /* SIMPLETS_H */
