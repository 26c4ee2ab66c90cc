// queries.cu -- kernels of the FP32-filtered Contains and Safety (the
// per-point routines and the argument for their exactness are in
// queries.cuh).  One thread per point, grid-stride; the FP32 daughter table
// is staged in shared memory with the bulk-copy engine when it fits.
#include <cuda_runtime.h>

#include "launch.cuh"
#include "queries.cuh"
#include "stage.cuh"

namespace geonav {

constexpr int kQueryTable32Max = 96 * 1024;   // bytes of FP32 records staged per block

template <bool SMEM>
__global__ void __launch_bounds__(256) k_contains32(VolView v, Basket b, int32_t* __restrict__ where) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const ShapeRec32* t32 = v.d32;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d32, uint32_t(v.nd) * sizeof(ShapeRec32), &bar, v.status)) return;
        t32 = reinterpret_cast<const ShapeRec32*>(smem_raw);
    }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        double p[3];
        float p32[3];
        point32(b, i, p, p32);
        where[i] = contains_filter(v, t32, p, p32);
    }
}

template <bool SMEM>
__global__ void __launch_bounds__(256) k_safety32(VolView v, Basket b, double* __restrict__ saf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const ShapeRec32* t32 = v.d32;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d32, uint32_t(v.nd) * sizeof(ShapeRec32), &bar, v.status)) return;
        t32 = reinterpret_cast<const ShapeRec32*>(smem_raw);
    }
    const float tau = safety_tau(v);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        double p[3];
        float p32[3];
        point32(b, i, p, p32);
        int nev;
        saf[i] = safety_filter(v, t32, p, p32, tau, &nev);
    }
}

#define GEO_LAUNCH32(KER, ...)                                                                  \
    do {                                                                                        \
        const int bytes = v.nd * int(sizeof(ShapeRec32));                                       \
        if (bytes <= kQueryTable32Max) {                                                        \
            cudaError_t e = prep(KER<true>, bytes);                                             \
            if (e != cudaSuccess) return e;                                                     \
            KER<true><<<blocks_for(KER<true>, b.n, bytes, num_sms), 256, bytes, s>>>(__VA_ARGS__); \
        } else {                                                                                \
            KER<false><<<blocks_for(KER<false>, b.n, 0, num_sms), 256, 0, s>>>(__VA_ARGS__);      \
        }                                                                                       \
        return cudaGetLastError();                                                              \
    } while (0)

cudaError_t launch_contains_filter(const VolView& v, const Basket& b, int32_t* where, cudaStream_t s,
                                   int num_sms) {
    GEO_LAUNCH32(k_contains32, v, b, where);
}

cudaError_t launch_safety_filter(const VolView& v, const Basket& b, double* saf, cudaStream_t s, int num_sms) {
    GEO_LAUNCH32(k_safety32, v, b, saf);
}

}  // namespace geonav
