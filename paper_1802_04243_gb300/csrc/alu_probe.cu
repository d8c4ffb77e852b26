// alu_probe.cu -- FMA throughput probe (include/simplets_probe.h).
// Register-only FMA chains: eight independent accumulators per thread hide
// the pipeline latency; the result is stored only so the compiler keeps the
// work.  The loop count is calibrated so one launch lasts about `millis` ms.
#include <cuda_runtime.h>

#include "simplets_probe.h"
#include "stg_common.cuh"

namespace {

template <typename T>
__global__ void k_fma_chains(int iters, T a, T b, T *sink)
{
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int k = 0; k < iters; k++) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == (T)-1.2345) sink[blockIdx.x] = s;     // practically never true
}

template <typename T>
int run(double millis, cudaStream_t st, double *gflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 3;
    const int threads = 256, blocks = sms * 8;
    T *sink = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&sink, blocks * sizeof(T)) != cudaSuccess) return 3;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int iters = 64;
    float ms = 0.f;
    int rc = 0;
    for (int pass = 0; pass < 12; pass++) {
        cudaEventRecord(e0, st);
        k_fma_chains<T><<<blocks, threads, 0, st>>>(iters, (T)0.999999, (T)1e-7, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = 3; break; }
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms >= 0.8 * millis) break;
        const double grow = ms > 0.05 ? millis / ms : 16.0;
        iters = (int)(iters * (grow > 16.0 ? 16.0 : grow) + 1);
    }
    if (!rc && cudaGetLastError() != cudaSuccess) rc = 3;
    if (!rc) {
        const double fmas = (double)blocks * threads * (double)iters * 64.0;
        *gflops = 2.0 * fmas / (ms * 1e-3) / 1e9;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

}  // namespace

extern "C" int simplets_alu_peak(int kind, double millis, void *stream, double *gflops)
{
    if (!gflops || !(millis >= 1.0) || (kind != 0 && kind != 1)) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    return kind == 0 ? run<double>(millis, st, gflops) : run<float>(millis, st, gflops);
}

// Both checks: copy x in, run one of the check kernels, copy the pairs out.
static int run_check(const double *host_x, int n, double *host_out, bool root)
{
    if (n < 0 || (n > 0 && (!host_x || !host_out))) return 1;
    if (n == 0) return 0;
    double *d = nullptr;
    if (cudaMalloc(&d, 3 * (size_t)n * sizeof(double)) != cudaSuccess) return 3;
    int rc = 0;
    if (cudaMemcpy(d, host_x, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) rc = 3;
    if (!rc) {
        if (root)
            stg::launch_sqrt_check(d, d + n, n, nullptr);
        else
            stg::launch_recip_check(d, d + n, n, nullptr);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(host_out, d + n, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = 3;
    }
    cudaFree(d);
    return rc;
}

extern "C" int simplets_recip_check(const double *host_x, int n, double *host_out)
{
    return run_check(host_x, n, host_out, false);
}

extern "C" int simplets_sqrt_check(const double *host_x, int n, double *host_out)
{
    return run_check(host_x, n, host_out, true);
}
