// FP32 FMA throughput of the current device, measured (the denominator of the near-field
// roofline: the ULI sum is bound by the FP32 pipe).  Every thread runs eight independent
// dependency chains of fused multiply-adds, as scalar FP32 or as the two-wide float2 form the
// near-field kernel uses, on a grid that fills every SM; no memory traffic inside the loop.
#include <cuda_runtime.h>

#include "../../include/fmm.h"
#include "devutil.cuh"
#include "fmm_internal.h"

namespace fmm {
namespace {

constexpr int kPeakThreads = 256, kPeakBlocksPerSM = 8, kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) ffma_kernel(float *sink, int iters, float a, float b) {
    float x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = (float)threadIdx.x * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i];
    if (s == -1.f) sink[0] = s;   // never true for these inputs; keeps the chains alive
}

__global__ void __launch_bounds__(kPeakThreads) ffma2_kernel(float *sink, int iters, float a, float b) {
    float2 x[kPeakChains];
    const float2 va = make_float2(a, a), vb = make_float2(b, b);
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = make_float2((float)threadIdx.x * 1e-3f + (float)i, (float)i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kPeakChains; ++i) x[i] = __ffma2_rn(x[i], va, vb);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i].x + x[i].y;
    if (s == -1.f) sink[0] = s;
}

}  // namespace
}  // namespace fmm

extern "C" fmm_status fmm_measure_fp32_peak(int iters, double *tflops_scalar, double *tflops_pair) {
    using namespace fmm;
    if (iters <= 0 || !tflops_scalar || !tflops_pair) return FMM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return FMM_ECUDA;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *sink = nullptr;
    fmm_status st = FMM_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc((void **)&sink, sizeof(float)) != cudaSuccess) {
        st = FMM_ECUDA;
    } else {
        const dim3 grid(sms * kPeakBlocksPerSM);
        const double lanes = (double)grid.x * kPeakThreads * kPeakChains * iters;
        for (int pass = 0; pass < 2 && st == FMM_OK; ++pass) {
            float ms = 0;
            for (int rep = 0; rep < 2 && st == FMM_OK; ++rep) {   // the first launch warms up
                cudaEventRecord(e0, s);
                if (pass == 0) ffma_kernel<<<grid, kPeakThreads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
                else ffma2_kernel<<<grid, kPeakThreads, 0, s>>>(sink, iters, 0.999f, 1e-3f);
                count_launch();
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    st = FMM_ECUDA;
            }
            const double flops = 2.0 * lanes * (pass == 0 ? 1.0 : 2.0);
            (pass == 0 ? *tflops_scalar : *tflops_pair) = flops / (ms * 1e-3) / 1e12;
        }
    }
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return st;
}
