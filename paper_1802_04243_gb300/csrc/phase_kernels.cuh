// phase_kernels.cuh -- the equation kernels of one loop-2 iteration
// (K. S. Shterev, arXiv:1802.04243, Section 3.1, Figs. 1 and 2, GPU column)
// and their launchers for one arithmetic.  Each of phase_fp64.cu,
// phase_mixed.cu and phase_df64.cu includes this header and instantiates the
// launchers of its own arithmetic, and each of step_fp64.cu, step_mixed.cu
// and step_df64.cu the persistent step kernels of its own, so the six compile
// in parallel.
//   k_faces      rho^u, rho^v, mass fluxes and conductivities of every face (Eqs. pl8-pl11, pl33)
//   k_explicit   the explicit terms, once per step (Eqs. pl15_11, pl31_1 and the u mirror)
//   k_assemble   T, u^/d^u, v^/d^v of every node         (Eqs. pl14-pl16, pl20, pl21, pl28-pl33)
//   k_pressure   p, rho = p/T, Gamma = T^omega, |dp|, |dT| (Eqs. pl23, pl24, pl5)
//   k_velocity   u, v from the new p, |du|, |dv|          (Eqs. pl18, pl19)
// The bodies are in sweep_bodies.cuh.
#pragma once
#include "grid_barrier.cuh"
#include "sweep_bodies.cuh"

namespace stg {
namespace {

// ONE: the problem's descriptor is read from the launch parameters in place
// (a list of one problem; for_tiles says when the host takes it).
template <int PREC, bool TVD, bool ONE>
__global__ void __launch_bounds__(256) k_faces(const __grid_constant__ BatchPlan bp, int level, int limiters)
{
    faces_phase<PREC, TVD, ONE>(bp, level, limiters);
}

template <int PREC, bool TVD, bool ONE>
__global__ void __launch_bounds__(256) k_explicit(const __grid_constant__ BatchPlan bp, int prev)
{
    explicit_phase<PREC, TVD, ONE>(bp, prev);
}

// Resident CTAs per SM: two for the FP64 assembly (bound by the FP64 pipe),
// four for the FP32 and double-float ones, which are latency-bound
// (measured against three: FP32 at 64 registers with a few bytes of spills
// 5-6 % faster, double-float up to 2.5 % despite its spills; five CTAs were
// slower for FP32).
template <int PREC, bool IMPL, bool TVD, bool ONE>
__global__ void __launch_bounds__(256, PREC == PREC_FP64 ? 2 : 4) k_assemble(const __grid_constant__ BatchPlan bp,
                                                                              int prev, int old, int nw)
{
    assemble_phase<PREC, IMPL, TVD, ONE>(bp, prev, old, nw);
}

template <int PREC, bool ONE>
__global__ void __launch_bounds__(256) k_pressure(const __grid_constant__ BatchPlan bp, int prev, int old, int nw)
{
    pressure_phase<PREC, ONE>(bp, prev, old, nw);
}

// The double-float pressure kernel at six resident CTAs of 256 threads per SM
// (40 registers; 0.183 -> 0.166 ms on the 4864 x 1216 channel).
template <bool ONE>
__global__ void __launch_bounds__(256, 6)
    k_pressure_df64(const __grid_constant__ BatchPlan bp, int prev, int old, int nw)
{
    pressure_phase<PREC_DF64, ONE>(bp, prev, old, nw);
}

// The mixed path's pressure kernel, bound by its FP64 remainder, at eight
// resident CTAs of 256 threads per SM (32 registers): 0.148 -> 0.141 ms on
// the 4864 x 1216 channel.  (An explicit bound is not neutral for the other
// arithmetics: with a minimum of one CTA per SM the double-float pressure
// kernel took 72 registers instead of 48 and ran 25 % slower.)
template <bool ONE>
__global__ void __launch_bounds__(256, 8)
    k_pressure_mixed(const __grid_constant__ BatchPlan bp, int prev, int old, int nw)
{
    pressure_phase<PREC_MIXED, ONE>(bp, prev, old, nw);
}

template <int PREC, bool ONE>
__global__ void __launch_bounds__(256) k_velocity(const __grid_constant__ BatchPlan bp, int old, int nw)
{
    velocity_phase<PREC, ONE>(bp, old, nw);
}

// The mixed path's velocity kernel, latency-bound, held at eight resident
// CTAs of 256 threads per SM (32 registers; left to itself the compiler took
// 40 and the kernel ran 8 % slower).
template <bool ONE>
__global__ void __launch_bounds__(256, 8) k_velocity_mixed(const __grid_constant__ BatchPlan bp, int old, int nw)
{
    velocity_phase<PREC_MIXED, ONE>(bp, old, nw);
}

// One time step of a batch in one cooperative kernel (persistent.cu launches
// it): the phases of the list over the tile list, a grid barrier between each
// two; the descriptor is staged as in the per-phase kernels.
template <int PREC, bool IMPL, bool TVD>
__global__ void __launch_bounds__(256, PREC == PREC_FP64 ? 2 : 4)
    k_step(const __grid_constant__ BatchPlan bp, const __grid_constant__ PhaseList ph, GridBarrier *bar)
{
    for (int q = 0; q < ph.n; q++) {
        switch (ph.kind[q]) {
        case PH_FACES: faces_phase<PREC, TVD>(bp, ph.a[q], ph.b[q]); break;
        case PH_EXPLICIT: explicit_phase<PREC, TVD>(bp, ph.a[q]); break;
        case PH_ASSEMBLE: assemble_phase<PREC, IMPL, TVD>(bp, ph.a[q], ph.b[q], ph.c[q]); break;
        case PH_PRESSURE: pressure_phase<PREC>(bp, ph.a[q], ph.b[q], ph.c[q]); break;
        default: velocity_phase<PREC>(bp, ph.a[q], ph.b[q]); break;
        }
        if (q + 1 < ph.n && !grid_barrier(bar, gridDim.x)) return;
    }
}

// Whether a launch reads the descriptor in place: a list of one problem in
// FP32 or double-float arithmetic (the FP64 kernels are not compiled that way).
template <int PREC>
bool in_place(const BatchPlan &bp)
{
    return PREC != PREC_FP64 && bp.n_inst == 1;
}

template <int PREC, bool TVD>
void faces_variant(const BatchPlan &bp, int level, int lim, cudaStream_t s)
{
    const dim3 bl(bp.tx, bp.ty);
    if constexpr (PREC != PREC_FP64)
        if (in_place<PREC>(bp)) {
            k_faces<PREC, TVD, true><<<bp.grid, bl, 0, s>>>(bp, level, lim);
            return;
        }
    k_faces<PREC, TVD, false><<<bp.grid, bl, 0, s>>>(bp, level, lim);
}

template <int PREC, bool TVD>
void explicit_variant(const BatchPlan &bp, int prev, cudaStream_t s)
{
    const dim3 bl(bp.tx, bp.ty);
    if constexpr (PREC != PREC_FP64)
        if (in_place<PREC>(bp)) {
            k_explicit<PREC, TVD, true><<<bp.grid, bl, 0, s>>>(bp, prev);
            return;
        }
    k_explicit<PREC, TVD, false><<<bp.grid, bl, 0, s>>>(bp, prev);
}

// The assembly may run on its own CTA count (BatchPlan::grid_asm).
template <int PREC, bool IMPL, bool TVD>
void assemble_variant(const BatchPlan &bp, int prev, int old, int nw, cudaStream_t s)
{
    const dim3 bl(bp.tx, bp.ty);
    const int g = bp.grid_asm > 0 ? bp.grid_asm : bp.grid;
    if constexpr (PREC != PREC_FP64)
        if (in_place<PREC>(bp)) {
            k_assemble<PREC, IMPL, TVD, true><<<g, bl, 0, s>>>(bp, prev, old, nw);
            return;
        }
    k_assemble<PREC, IMPL, TVD, false><<<g, bl, 0, s>>>(bp, prev, old, nw);
}

}  // namespace

template <int PREC>
void launch_faces_of(const BatchPlan &bp, int level, bool tvd, int lim, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (tvd) faces_variant<PREC, true>(bp, level, lim, s);
    else faces_variant<PREC, false>(bp, level, 0, s);
}

template <int PREC>
void launch_explicit_of(const BatchPlan &bp, int prev, bool tvd, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (tvd) explicit_variant<PREC, true>(bp, prev, s);
    else explicit_variant<PREC, false>(bp, prev, s);
}

template <int PREC>
void launch_assemble_of(const BatchPlan &bp, int prev, int old, int nw, bool implicit, bool tvd, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (implicit && tvd) assemble_variant<PREC, true, true>(bp, prev, old, nw, s);
    else if (implicit) assemble_variant<PREC, true, false>(bp, prev, old, nw, s);
    else if (tvd) assemble_variant<PREC, false, true>(bp, prev, old, nw, s);
    else assemble_variant<PREC, false, false>(bp, prev, old, nw, s);
}

template <int PREC>
void launch_pressure_of(const BatchPlan &bp, int prev, int old, int nw, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 bl(bp.tx, bp.ty);
    if constexpr (PREC == PREC_MIXED) {
        if (in_place<PREC>(bp))
            k_pressure_mixed<true><<<bp.grid, bl, 0, s>>>(bp, prev, old, nw);
        else
            k_pressure_mixed<false><<<bp.grid, bl, 0, s>>>(bp, prev, old, nw);
    } else if constexpr (PREC == PREC_DF64) {
        if (in_place<PREC>(bp))
            k_pressure_df64<true><<<bp.grid, bl, 0, s>>>(bp, prev, old, nw);
        else
            k_pressure_df64<false><<<bp.grid, bl, 0, s>>>(bp, prev, old, nw);
    } else {
        k_pressure<PREC, false><<<bp.grid, bl, 0, s>>>(bp, prev, old, nw);
    }
}

template <int PREC>
void launch_velocity_of(const BatchPlan &bp, int old, int nw, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 bl(bp.tx, bp.ty);
    if constexpr (PREC == PREC_MIXED) {
        if (in_place<PREC>(bp))
            k_velocity_mixed<true><<<bp.grid, bl, 0, s>>>(bp, old, nw);
        else
            k_velocity_mixed<false><<<bp.grid, bl, 0, s>>>(bp, old, nw);
    } else if constexpr (PREC == PREC_DF64) {
        if (in_place<PREC>(bp))
            k_velocity<PREC, true><<<bp.grid, bl, 0, s>>>(bp, old, nw);
        else
            k_velocity<PREC, false><<<bp.grid, bl, 0, s>>>(bp, old, nw);
    } else {
        k_velocity<PREC, false><<<bp.grid, bl, 0, s>>>(bp, old, nw);
    }
}

template <int PREC>
void *step_kernel_for(bool implicit, bool tvd)
{
    if (implicit && tvd) return reinterpret_cast<void *>(&k_step<PREC, true, true>);
    if (implicit) return reinterpret_cast<void *>(&k_step<PREC, true, false>);
    if (tvd) return reinterpret_cast<void *>(&k_step<PREC, false, true>);
    return reinterpret_cast<void *>(&k_step<PREC, false, false>);
}

}  // namespace stg

// The launchers of one arithmetic, instantiated by its translation unit.
#define STG_PHASE_LAUNCHERS(PREC)                                                                              \
    namespace stg {                                                                                            \
    template void launch_faces_of<PREC>(const BatchPlan &, int, bool, int, void *);                            \
    template void launch_explicit_of<PREC>(const BatchPlan &, int, bool, void *);                              \
    template void launch_assemble_of<PREC>(const BatchPlan &, int, int, int, bool, bool, void *);              \
    template void launch_pressure_of<PREC>(const BatchPlan &, int, int, int, void *);                          \
    template void launch_velocity_of<PREC>(const BatchPlan &, int, int, void *);                               \
    }

// The persistent step kernels of one arithmetic, instantiated by a
// translation unit of their own (step_*.cu: each holds every phase).
#define STG_STEP_KERNELS(PREC)                                                                                 \
    namespace stg {                                                                                            \
    template void *step_kernel_for<PREC>(bool, bool);                                                          \
    }
