// Arithmetic-pipe throughput probe behind les_measure_peak: the denominators
// of the compute-bound roofline fractions (FP64 FMA for the FP64 stage
// kernels; FP32 FMA, scalar and paired, for the FP32 stage), measured on the
// running GPU instead of derived from unit counts and the maximum clock.
//
// Every thread runs NCHAIN independent multiply-add chains for `iters`
// rounds; the chains are independent, so the pipe, not the dependency
// latency, bounds the rate once a few warps per scheduler are resident.  The
// operands come from arguments and the result is stored under a condition
// that is never true, so the compiler can neither fold nor drop the loop.
#include <cuda_runtime.h>

#include "les.h"

namespace {

constexpr int NCHAIN = 8;
constexpr int UNROLL = 16;

template <int KIND>
__global__ void __launch_bounds__(256) k_fma_probe(double *sink, int iters, double a0, double b0)
{
    if constexpr (KIND == 0) {
        double acc[NCHAIN];
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) acc[c] = a0 + c + threadIdx.x;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
#pragma unroll
                for (int c = 0; c < NCHAIN; ++c) acc[c] = fma(acc[c], b0, a0);
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) s += acc[c];
        if (s == -1.2345e300) sink[threadIdx.x] = s;
    } else if constexpr (KIND == 1) {
        const float a = (float)a0, b = (float)b0;
        float acc[NCHAIN];
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) acc[c] = a + c + threadIdx.x;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
#pragma unroll
                for (int c = 0; c < NCHAIN; ++c) acc[c] = fmaf(acc[c], b, a);
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) s += acc[c];
        if (s == -1.2345e30f) sink[threadIdx.x] = s;
    } else {
        // paired FP32: one fma.rn.f32x2 per chain and round, two lanes each
        const float2 a = make_float2((float)a0, (float)a0), b = make_float2((float)b0, (float)b0);
        float2 acc[NCHAIN];
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) acc[c] = make_float2(a.x + c + threadIdx.x, a.x - c - threadIdx.x);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
#pragma unroll
                for (int c = 0; c < NCHAIN; ++c) acc[c] = __ffma2_rn(acc[c], b, a);
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) s += acc[c].x + acc[c].y;
        if (s == -1.2345e30f) sink[threadIdx.x] = s;
    }
}

} // namespace

extern "C" int les_measure_peak(int kind, double *tflops)
{
    if (!tflops || kind < 0 || kind > 2) return LES_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LES_ERR_CUDA;
    // FP64 runs at a small fraction of the FP32 rate: fewer rounds
    const int iters = kind == 0 ? 512 : 2048;
    const int blocks = nsm * 8, threads = 256;
    double *sink = nullptr; // never written (the store's condition is false)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return LES_ERR_CUDA;
    }
    float best = 1e30f;
    int rc = LES_OK;
    for (int rep = 0; rep < 6 && rc == LES_OK; ++rep) {
        cudaEventRecord(e0, nullptr);
        if (kind == 0) k_fma_probe<0><<<blocks, threads>>>(sink, iters, 1.0000001, 0.9999999);
        else if (kind == 1) k_fma_probe<1><<<blocks, threads>>>(sink, iters, 1.0000001, 0.9999999);
        else k_fma_probe<2><<<blocks, threads>>>(sink, iters, 1.0000001, 0.9999999);
        cudaEventRecord(e1, nullptr);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = LES_ERR_CUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms; // the first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LES_OK) return rc;
    const double lanes = kind == 2 ? 2.0 : 1.0;
    const double flop = 2.0 * lanes * NCHAIN * UNROLL * (double)iters * blocks * threads;
    *tflops = flop / (best * 1e-3) / 1e12;
    return LES_OK;
}
