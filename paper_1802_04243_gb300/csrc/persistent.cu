// persistent.cu -- one kernel per time step of a batch: every phase of the
// SIMPLE-TS iteration (arXiv:1802.04243, Section 3.1: explicit terms, then
// per loop-2 iteration face densities, assembly, pressure, velocity
// correction) over the batch's tile list, with a grid-wide barrier between
// the phases instead of a kernel boundary.  The phases run the same bodies as
// the per-phase kernels (sweep_bodies.cuh).  The kernel is launched
// cooperatively with no more CTAs than stay resident, so every CTA reaches
// every barrier; each barrier wait is bounded in time and a wait that runs
// out sets an error word and ends the kernel (the host reads it as
// SIM_ETIMEOUT).
#include <cuda_runtime.h>

#include "sweep_bodies.cuh"

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

template <int PREC, bool IMPL, bool TVD>
void *step_kernel()
{
    return reinterpret_cast<void *>(&k_step<PREC, IMPL, TVD>);
}

void *step_kernel_of(int prec, bool implicit, bool tvd)
{
    switch (prec * 4 + (implicit ? 2 : 0) + (tvd ? 1 : 0)) {
    case 0: return step_kernel<PREC_FP64, false, false>();
    case 1: return step_kernel<PREC_FP64, false, true>();
    case 2: return step_kernel<PREC_FP64, true, false>();
    case 3: return step_kernel<PREC_FP64, true, true>();
    case 4: return step_kernel<PREC_MIXED, false, false>();
    case 5: return step_kernel<PREC_MIXED, false, true>();
    case 6: return step_kernel<PREC_MIXED, true, false>();
    case 7: return step_kernel<PREC_MIXED, true, true>();
    case 8: return step_kernel<PREC_DF64, false, false>();
    case 9: return step_kernel<PREC_DF64, false, true>();
    case 10: return step_kernel<PREC_DF64, true, false>();
    default: return step_kernel<PREC_DF64, true, true>();
    }
}

// Crosses `rounds` barriers expecting `nblocks` CTAs.
__global__ void __launch_bounds__(256) k_barrier_check(GridBarrier *bar, unsigned nblocks, int rounds)
{
    for (int r = 0; r < rounds; r++)
        if (!grid_barrier(bar, nblocks)) return;
}

}  // namespace

int persistent_ctas(int prec, bool implicit, bool tvd, int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel_of(prec, implicit, tvd), threads, 0) !=
            cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t launch_step_persistent(const BatchPlan &bp, const PhaseList &ph, GridBarrier *bar, int prec, bool implicit,
                                   bool tvd, int ctas, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    BatchPlan p = bp;
    PhaseList l = ph;
    GridBarrier *b = bar;
    void *args[3] = {&p, &l, &b};
    return cudaLaunchCooperativeKernel(step_kernel_of(prec, implicit, tvd), dim3((unsigned)ctas),
                                       dim3((unsigned)bp.tx, (unsigned)bp.ty), args, 0, s);
}

}  // namespace stg

extern "C" int simplets_barrier_check(int extra_blocks, int rounds, int *err_out, int *ctas_out)
{
    using namespace stg;
    if (extra_blocks < 0 || extra_blocks > 1024 || rounds < 1 || rounds > 1000 || !err_out || !ctas_out) return 1;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_check, 256, 0) != cudaSuccess || per_sm < 1)
        return 3;
    GridBarrier *bar = nullptr;
    if (cudaMalloc(&bar, sizeof(GridBarrier)) != cudaSuccess) return 3;
    int rc = 0;
    const int ctas = per_sm * sms;
    unsigned nblocks = (unsigned)(ctas + extra_blocks);
    void *args[3] = {&bar, &nblocks, &rounds};
    GridBarrier h{};
    if (cudaMemset(bar, 0, sizeof(GridBarrier)) != cudaSuccess ||
        cudaLaunchCooperativeKernel((void *)k_barrier_check, dim3((unsigned)ctas), dim3(256), args, 0, nullptr) !=
            cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&h, bar, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = 3;
    cudaFree(bar);
    *err_out = (int)h.err;
    *ctas_out = ctas;
    return rc;
}
