/*
 * simplets_noalloc.h -- the SIMPLE-TS time step for callers that cannot
 * allocate device memory.
 *
 * The paper has no counterpart to this entry point; it is a property of this
 * library.  sim_create allocates every buffer a problem needs with cudaMalloc.
 * Some callers cannot do that at the moment they want to run the solver:
 *   - applications that reserve their GPU memory once at start-up (their own
 *     pool or a fixed budget) and forbid allocations afterwards;
 *   - loops that cannot afford the device-wide synchronisation that
 *     cudaMalloc and cudaFree imply;
 *   - plug-ins called from a host framework that owns the device memory and
 *     hands them only the arrays to work on.
 * sim_step_noalloc serves them: it takes the problem description and the
 * caller's own device arrays, and carves everything else it needs out of one
 * static device array that is part of the library itself.
 */
#ifndef SIMPLETS_NOALLOC_H
#define SIMPLETS_NOALLOC_H

#include "simplets.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Size of the static scratch in MiB.  Every GPU that loads the library holds
 * this much device memory until the process exits. */
#define SIM_NOALLOC_SCRATCH_MB 96

/* Advance the state held in the caller's device arrays by n_steps time steps,
 * exactly as sim_create + sim_step (FP64) would, without allocating anything:
 * no cudaMalloc, no cudaFree, no allocating library routine.
 *
 * grid, gas, bc: the problem, as for sim_create (host structures and host
 *   arrays).  Restrictions: bc->precision must be SIM_FP64, bc->tol must be 0
 *   (every step runs bc->iters loop-2 iterations), at most 64 obstacles.
 * d_u, d_v, d_p, d_T: device arrays in the logical layout of sim_fields
 *   (u: ny x (nx+1), v: (ny+1) x nx, p and T: ny x nx).  On entry they hold
 *   the state; their unknowns (faces between fluid cells, fluid cells) are
 *   read and every other value follows the boundary rules.  On return they
 *   hold the state after n_steps, boundary values included.
 * stream: the cudaStream_t all work is queued on (NULL: legacy default).
 * res_out: NULL, or 4 host doubles receiving the residuals of the last
 *   loop-2 iteration (max |du|, |dv|, |dp|, |dT|); when given, the call waits
 *   for the stream.
 *
 * Scratch: one static 96 MiB device array holds three state levels, the
 * scratch of the sweep, the geometry tables and the residual words, about
 * 404 bytes per element of the padded grid (pitch x (ny + 5), pitch =
 * nx + 5 rounded up to a multiple of 8): up to about 249,000 elements,
 * e.g. 1000 x 240 or 490 x 490 cells.  A larger problem returns SIM_ENOMEM
 * before any work is queued.
 *
 * First call on a device: it looks up the device address of the static
 * array once (cudaGetSymbolAddress, with that device current), which can load
 * the library's GPU code.  Make the first call on each device before any
 * stream capture begins.  The address is kept per device and CUDA context:
 * a call from another context (for instance after cudaDeviceReset) looks it
 * up again.
 *
 * Host arrays of the description (grid->dx, grid->dy, bc->rect and the inflow
 * profiles) are copied to the scratch with cudaMemcpyAsync on `stream`; keep
 * them unchanged until the stream has reached the call's work.
 *
 * Sharing: all calls on a device use the same array, which keeps the last
 * call's contents; the call clears what must start at zero.  Two calls that
 * overlap on the GPU (other streams, other threads) race on the array and
 * corrupt each other's results: issue one call at a time per device.
 *
 * Returns SIM_OK, SIM_EINVAL (bad or unsupported description), SIM_ENOMEM
 * (problem too large for the static scratch), SIM_ECUDA (a CUDA call
 * failed), SIM_EDIVERGED (res_out given and a residual is not finite). */
sim_status sim_step_noalloc(const sim_grid *grid, const sim_gas *gas, const sim_bc *bc, int n_steps,
                            int scheme, double *d_u, double *d_v, double *d_p, double *d_T,
                            void *stream, double res_out[4]);

#ifdef __cplusplus
}
#endif
#endif
