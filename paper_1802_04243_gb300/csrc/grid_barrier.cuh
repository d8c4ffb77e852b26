// grid_barrier.cuh -- the bounded grid-wide barrier of the persistent step
// kernel (every CTA of a cooperative launch).
#pragma once
#include "stg_common.cuh"

namespace stg {
namespace {

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Longest wait at one barrier before the kernel gives up: far above a phase's
// duration on any problem that fits the device.
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;

// Barrier of all `nblocks` CTAs of the grid (generation counting).  Thread 0
// of each CTA takes the CTA's arrival: it reads the generation, fences its
// CTA's writes, counts itself in; the last CTA to arrive resets the count and
// advances the generation, the others wait for that with acquire loads.
// Returns false (in every thread of the CTA) once any CTA has timed out.
__device__ bool grid_barrier(GridBarrier *b, unsigned nblocks)
{
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned gen = load_acquire(&b->gen);
        __threadfence();
        if (atomicAdd(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (load_acquire(&b->gen) == gen) {
                if (load_acquire(&b->err)) break;
                if (global_ns() - t0 > kBarrierLimitNs) {
                    atomicOr(&b->err, 1u);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = load_acquire(&b->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace
}  // namespace stg
