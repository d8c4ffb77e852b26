// persistent.cu -- launch of the persistent step kernel of a batch (k_step,
// phase_kernels.cuh, compiled with the per-phase kernels of its arithmetic):
// every phase of the SIMPLE-TS iteration (arXiv:1802.04243, Section 3.1:
// explicit terms, then per loop-2 iteration face densities, assembly,
// pressure, velocity correction) over the batch's tile list, with a
// grid-wide barrier between the phases instead of a kernel boundary.  The
// kernel is launched cooperatively with no more CTAs than stay resident, so
// every CTA reaches every barrier; each barrier wait is bounded in time and a
// wait that runs out sets an error word and ends the kernel (the host reads
// it as SIM_ETIMEOUT).  Also the barrier's own check kernel.
#include <cuda_runtime.h>

#include "grid_barrier.cuh"

namespace stg {
namespace {

void *step_kernel_of(int prec, bool implicit, bool tvd)
{
    if (prec == PREC_DF64) return step_kernel_for<PREC_DF64>(implicit, tvd);
    if (prec == PREC_MIXED) return step_kernel_for<PREC_MIXED>(implicit, tvd);
    return step_kernel_for<PREC_FP64>(implicit, tvd);
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
