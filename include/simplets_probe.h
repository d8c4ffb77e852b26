/*
 * simplets_probe.h -- arithmetic-throughput probe of the device, used as the
 * ALU roofline of the SIMPLE-TS sweep, and a check of the sweep's FP64
 * reciprocal against IEEE division.
 *
 * The paper measures operator cost with a "simplified test code": the energy
 * equation evaluated on private variables in a loop with no memory traffic
 * (Section 3.4).  This probe is the same idea reduced to the instruction the
 * sweep is bound by: independent fused multiply-add chains on registers,
 * in FP64 (the FP64 path) or FP32 (the mixed path), with no memory traffic.
 */
#ifndef SIMPLETS_PROBE_H
#define SIMPLETS_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Measure the device's sustained fused-multiply-add rate on `stream`.
 * kind: 0 = FP64 (DFMA), 1 = FP32 (FFMA).  The kernel fills every SM with
 * independent FMA chains for about `millis` milliseconds (>= 1) and times
 * itself with CUDA events.  *gflops receives 2 x FMAs / second / 1e9.
 * Returns 0 on success, 1 on a bad argument, 3 on a CUDA error.  Synchronous. */
int simplets_alu_peak(int kind, double millis, void *stream, double *gflops);

/* Check of the FP64 reciprocal the sweep uses in place of IEEE division
 * (from the FP32 reciprocal r of x, one step r <- r + r (e + e^2) with
 * e = 1 - x r, the geometric series of 1/x = r / (1 - e) to third order;
 * IEEE division for |x| outside [2^-100, 2^100]).
 * host_x: n doubles (host memory).  host_out: 2n doubles (host memory)
 * receiving, for each x[q], the sweep's reciprocal in host_out[2q] and the
 * IEEE quotient 1/x[q] in host_out[2q+1], both computed on the device.
 * Returns 0 on success, 1 on a bad argument, 3 on a CUDA error.  Synchronous;
 * allocates and frees its own device buffers. */
int simplets_recip_check(const double *host_x, int n, double *host_out);

/* Check of the FP64 square root the sweep uses for Gamma = T^(1/2) (two
 * Newton-Raphson steps s <- s + (x - s^2) y/2 from s = x y, y the FP32
 * reciprocal square root of x; the library's sqrt for |x| outside
 * [2^-100, 2^100]).  Same arguments and returns as simplets_recip_check, with
 * the sweep's root in host_out[2q] and the IEEE root in host_out[2q+1]. */
int simplets_sqrt_check(const double *host_x, int n, double *host_out);

/* Check of the grid barrier of the persistent batch step (sim_batch_set_persistent):
 * a cooperative launch of all resident CTAs of a 256-thread kernel crosses
 * `rounds` barriers, each expecting gridDim.x + extra_blocks CTAs.  With
 * extra_blocks = 0 every barrier completes; with extra_blocks > 0 no barrier
 * can complete, every wait runs out after its 2 s limit, the kernel ends and
 * *err_out is set.  *err_out receives the barrier's error word (0: every
 * barrier completed), *ctas_out the CTAs launched.  Returns 0 on success, 1 on
 * a bad argument, 3 on a CUDA error.  Synchronous; allocates and frees its own
 * device buffer. */
int simplets_barrier_check(int extra_blocks, int rounds, int *err_out, int *ctas_out);

#ifdef __cplusplus
}
#endif
#endif
