// Roofline probes: sustained FP64 / FP32 FMA and exp throughput of the
// current device, measured with CUDA events around register-resident kernels
// that run on every SM (8 independent dependency chains per thread so the
// pipes, not latency, are the limit).
#include "../../include/bgk.h"
#include "bgk_internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T *sink, int iters, T b, T c) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == (T)-12345.0) sink[threadIdx.x] = s;   // never true; keeps the chains live
}

__global__ void __launch_bounds__(256) k_exp64(double *sink, int iters) {
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = -(double)(threadIdx.x + i) * 1e-4;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = exp(-a[i]) - 1.5;   // stays in (-1.5, -0.5)
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == -12345.0) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_exp32(float *sink, int iters) {
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = -(float)(threadIdx.x + i) * 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = exp2f(-a[i]) - 1.5f;
    }
    float s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == -12345.0f) sink[threadIdx.x] = s;
}

cudaError_t run_probe(int kind, int iters, dim3 grid, void *sink, float *ms) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    switch (kind) {
        case 0: k_fma<double><<<grid, 256>>>((double *)sink, iters, 0.999999, 1e-7); break;
        case 1: k_fma<float><<<grid, 256>>>((float *)sink, iters, 0.999999f, 1e-7f); break;
        case 2: k_exp64<<<grid, 256>>>((double *)sink, iters); break;
        default: k_exp32<<<grid, 256>>>((float *)sink, iters); break;
    }
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

}  // namespace

extern "C" BGK_API bgk_status bgk_probe_peak(int kind, double *value) {
    if (!value || kind < 0 || kind > 3) return BGK_EINVAL;
    int dev, sms;
    if (cudaGetDevice(&dev) != cudaSuccess) return BGK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BGK_ECUDA;
    const dim3 grid(sms * 8);
    void *sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return BGK_ENOMEM;
    // calibrate to ~50 ms, then measure
    int iters = 256;
    float ms = 0.f;
    bgk_status st = BGK_OK;
    for (int pass = 0; pass < 8; ++pass) {
        if (run_probe(kind, iters, grid, sink, &ms) != cudaSuccess) { st = BGK_ECUDA; break; }
        if (ms >= 40.f) break;
        const double scale = ms > 0.05f ? 50.0 / ms : 16.0;
        const double next = iters * (scale > 16.0 ? 16.0 : scale);
        iters = next > 2.0e9 ? 2000000000 : (int)next;
    }
    if (st == BGK_OK && run_probe(kind, iters, grid, sink, &ms) != cudaSuccess) st = BGK_ECUDA;
    cudaFree(sink);
    if (st != BGK_OK) return st;
    const double ops = (double)grid.x * 256.0 * 8.0 * (double)iters;
    *value = (kind <= 1 ? 2.0 * ops : ops) / (ms * 1e-3);
    return BGK_OK;
}
