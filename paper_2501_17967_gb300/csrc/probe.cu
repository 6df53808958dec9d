// Throughput probe for the FP64 FMA pipe: the roofline denominator of the
// FP64 passes (the paper's arithmetic is FP64 throughout).
#include <cuda_runtime.h>

#include "bc_internal.h"

namespace bc {
namespace {

constexpr int kChains = 8;

__global__ void k_dfma_probe(int iters, double seed, double *out)
{
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = seed + threadIdx.x * 1e-9 + c;
    const double m = 0.9999999, b = 1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fma(a[c], m, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == 12345.678) out[0] = s;   // never true; keeps the chains live
}

}  // namespace
}  // namespace bc

extern "C" bc_status bc_debug_fp64_peak(int device, double *tflops)
{
    using namespace bc;
    if (!tflops) { set_error("bc_debug_fp64_peak: NULL argument"); return BC_ERR_ARG; }
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    double *out = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int threads = 256, blocks = sms * 8, iters = 4096;
    float best = 1e30f;
    for (int rep = 0; e == cudaSuccess && rep < 4; rep++) {
        cudaEventRecord(t0);
        k_dfma_probe<<<blocks, threads>>>(iters, 1.0 + rep, out);
        cudaEventRecord(t1);
        e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best) best = ms;
    }
    if (out) cudaFree(out);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) {
        set_error("bc_debug_fp64_peak: %s", cudaGetErrorString(e));
        return BC_ERR_CUDA;
    }
    double flops = 2.0 * kChains * double(iters) * threads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    return BC_OK;
}
