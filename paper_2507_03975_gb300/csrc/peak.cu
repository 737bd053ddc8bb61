// FP64 FMA rate of the device (gsis_measure_fp64_fma): the denominator of
// the ALU-bound kernels' rooflines.  Every thread runs kChains independent
// dependent-FMA chains, so each sub-partition always has FP64 instructions
// to issue; the grid fills every SM with kBlocksPerSm blocks.
#include <cuda_runtime.h>

#include "gsis.h"
#include "host.h"

using namespace gsis;

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ double g_fma_sink;

__global__ void __launch_bounds__(kThreads) fma_rate_kernel(double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-6 + c;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) g_fma_sink = s;   // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int gsis_measure_fp64_fma(double* gflops, void* stream)
{
    if (!gflops) return fail(GSIS_ERR_ARG, "gflops is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * kBlocksPerSm;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 0.f;
    for (int rep = 0; rep < 4; ++rep) {   // the first is the warm-up
        CK(cudaEventRecord(e0, st));
        fma_rate_kernel<<<grid, kThreads, 0, st>>>(0.999999999, 1e-9);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    const double flops = 2.0 * kChains * (double)kIters * kThreads * grid;
    *gflops = flops / (best * 1e-3) / 1e9;
    return GSIS_OK;
}
