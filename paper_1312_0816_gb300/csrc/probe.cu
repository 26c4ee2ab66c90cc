// probe.cu -- measurement support, not part of the navigator: issue-rate
// probes of the arithmetic pipes the navigator uses (FP32 FMA, FP64 FMA, FP64
// divide and square root, FP32 divide and square root), timed with CUDA
// events.  The roofline of the ALU-bound kernels divides by these rates.
#include <cuda_runtime.h>
#include <cstdint>
#include "../../include/geo.h"

namespace {

constexpr int kChains = 8;

template <typename T, int WHAT>
__global__ void __launch_bounds__(256) k_probe(int64_t iters, T seed, T* out) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + T(threadIdx.x + c) * T(1e-3);
    const T m = T(0.999999), k = T(1e-7), one = T(1.0);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (WHAT == 0) a[c] = a[c] * m + k;                 // fused multiply-add
            else if (WHAT == 1) a[c] = one / a[c] + k;          // divide (+ an add)
            else a[c] = sqrt(a[c]) + k;                         // square root (+ an add)
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == T(-12345.0)) out[threadIdx.x] = s;   // keeps the chains alive
}

template <typename T, int WHAT>
double run(int64_t iters, int blocks, cudaStream_t st, T* scratch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe<T, WHAT><<<blocks, 256, 0, st>>>(iters / 8, T(1.5), scratch);   // warm-up
    cudaEventRecord(e0, st);
    k_probe<T, WHAT><<<blocks, 256, 0, st>>>(iters, T(1.5), scratch);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double ops = double(blocks) * 256.0 * double(iters) * kChains;
    return ms > 0.f ? ops / (double(ms) * 1e-3) : 0.0;
}

}  // namespace

extern "C" {

// Measures the issue rate (operations per second over the whole GPU) of one
// arithmetic operation: what = 0 FP32 FMA, 1 FP64 FMA, 2 FP64 divide,
// 3 FP64 square root, 4 FP32 divide, 5 FP32 square root.  `scratch` is a
// device buffer of at least 256 doubles.  Synchronises `stream`.
geo_status geo_probe_pipe(int32_t what, int64_t iters, int32_t blocks, void* scratch, void* stream,
                          double* ops_per_s) {
    if (!ops_per_s || !scratch || iters <= 0 || blocks <= 0) return GEO_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double r = 0.0;
    switch (what) {
        case 0: r = run<float, 0>(iters, blocks, st, static_cast<float*>(scratch)); break;
        case 1: r = run<double, 0>(iters, blocks, st, static_cast<double*>(scratch)); break;
        case 2: r = run<double, 1>(iters, blocks, st, static_cast<double*>(scratch)); break;
        case 3: r = run<double, 2>(iters, blocks, st, static_cast<double*>(scratch)); break;
        case 4: r = run<float, 1>(iters, blocks, st, static_cast<float*>(scratch)); break;
        case 5: r = run<float, 2>(iters, blocks, st, static_cast<float*>(scratch)); break;
        default: return GEO_ERR_INVALID_ARG;
    }
    if (cudaGetLastError() != cudaSuccess) return GEO_ERR_CUDA;
    *ops_per_s = r;
    return GEO_OK;
}

}  // extern "C"
