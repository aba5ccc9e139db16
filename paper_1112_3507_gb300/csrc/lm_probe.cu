// Arithmetic-rate probes: the measured float64 roof that the float64 kernels
// of the solver are measured against.
//
// GB300 issues float64 at a small fraction of its float32 rate, so a float64
// stencil can be bound by its arithmetic rather than by HBM.  These kernels
// time long chains of independent fused multiply-adds (and of float64 <->
// float32 conversions) on every SM, so the roof comes from this GPU at its
// current clocks rather than from a datasheet.  No clocks or other device
// settings are touched.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/lowmach.h"
#include "lm_kernels.h"

namespace {

constexpr int PROBE_CHAINS = 8;     // independent chains per thread (covers the pipe latency)
constexpr int PROBE_THREADS = 256;

// Each chain iterates v <- v * m + a, a contraction towards a / (1 - m) = 1,
// so the values stay finite for any number of steps.
template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(int steps, T m, T a, T* __restrict__ sink) {
    T v[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = fma(v[c], m, a);
    }
    T t = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) t += v[c];
    if (t == (T)-1) sink[0] = t;      // never true; keeps the chains live
}

// Chains of a float64 -> float32 -> float64 round trip around a float32 FMA:
// two conversions per step.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_cvt(int steps, float* __restrict__ sink) {
    double v[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = (double)fmaf(__double2float_rn(v[c]), 0.999f, 1e-3f);
    }
    double t = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) t += v[c];
    if (t == -1.0) sink[0] = (float)t;
}

}  // namespace

extern "C" int lm_probe_rate(int which, int steps, double* ops_per_s, void* stream) {
    if (!ops_per_s || which < 0 || which > 2 || steps < 1) return LM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return LM_ERR_CUDA;
    const int blocks = 8 * sms;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return LM_ERR_OUT_OF_MEMORY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int n) {
        lm::count_launches(1);
        if (which == 0) k_probe_fma<double><<<blocks, PROBE_THREADS, 0, s>>>(n, 0.999999, 1e-6, (double*)sink);
        else if (which == 1) k_probe_fma<float><<<blocks, PROBE_THREADS, 0, s>>>(n, 0.999f, 1e-3f, (float*)sink);
        else k_probe_cvt<<<blocks, PROBE_THREADS, 0, s>>>(n, (float*)sink);
    };
    launch(steps / 8 + 1);                       // warm-up
    cudaEventRecord(e0, s);
    launch(steps);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) {
        fprintf(stderr, "lowmach: probe failed: %s\n", cudaGetErrorString(err));
        return LM_ERR_CUDA;
    }
    const double ops = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)steps * (which == 2 ? 2.0 : 1.0);
    *ops_per_s = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
    return LM_OK;
}
