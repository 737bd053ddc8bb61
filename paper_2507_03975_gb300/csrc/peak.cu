// FP64 and FP32 FMA rates of the device (gsis_measure_fp64_fma,
// gsis_measure_fp32_fma): the denominators of the ALU-bound kernels'
// rooflines.  Every thread runs kChains independent dependent-FMA chains, so
// each sub-partition always has FMA instructions to issue; the grid fills
// every SM with kBlocksPerSm blocks.
#include <cuda_runtime.h>

#include "gsis.h"
#include "host.h"

using namespace gsis;

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ double g_sink_d;
__device__ float g_sink_f;
__device__ __forceinline__ void sink(double v) { g_sink_d = v; }
__device__ __forceinline__ void sink(float v) { g_sink_f = v; }

template <typename T, int ITERS>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x * 1e-6 + c);
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)12345.678) sink(s);   // keeps the chains live; never true for these inputs
}

// Best of three timed launches after one warm-up, in GFLOP/s.
template <typename T, int ITERS>
int measure(double* gflops, void* stream)
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
    for (int rep = 0; rep < 4; ++rep) {
        CK(cudaEventRecord(e0, st));
        fma_rate_kernel<T, ITERS><<<grid, kThreads, 0, st>>>((T)0.999999999, (T)1e-9);
        CK(cudaGetLastError());
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    const double flops = 2.0 * kChains * (double)ITERS * kThreads * grid;
    *gflops = flops / (best * 1e-3) / 1e9;
    return GSIS_OK;
}

}  // namespace

extern "C" int gsis_measure_fp64_fma(double* gflops, void* stream) { return measure<double, 2048>(gflops, stream); }

extern "C" int gsis_measure_fp32_fma(double* gflops, void* stream) { return measure<float, 65536>(gflops, stream); }
