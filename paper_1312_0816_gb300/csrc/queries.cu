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

// Safety: per tile of 256 points, the FP32 pass runs per thread; the first
// FP64 evaluation of every point (its smallest-bound candidate) is then
// binned by solid kind (mother, box, tube, cone) and evaluated by whole warps
// over the binned list, so a warp mostly runs one kind's code (a warp pays
// for every code path its lanes take, and the FP64 pipe charges a warp
// instruction whatever the number of active lanes).  Each point then
// finishes on its own thread (rarely with more FP64 work).  Which warp
// evaluates a task does not change its value, so results are deterministic.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_safety32(VolView v, Basket b, double* __restrict__ saf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ double s_p[3][256];
    __shared__ double s_res[256];
    __shared__ int s_task[256];
    __shared__ int s_list[256];
    __shared__ int s_cnt[4];
    const ShapeRec32* t32 = v.d32;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d32, uint32_t(v.nd) * sizeof(ShapeRec32), &bar, v.status)) return;
        t32 = reinterpret_cast<const ShapeRec32*>(smem_raw);
    }
    const float tau = safety_tau(v);
    const int t = threadIdx.x;
    const int64_t ntiles = (b.n + 255) / 256;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * 256 + t;
        const bool live = i < b.n;
        double p[3] = {0.0, 0.0, 0.0};
        float p32[3] = {0.f, 0.f, 0.f};
        if (live) point32(b, i, p, p32);
        SafetyState st;
        st.Lm = st.L2 = 0.f;
        st.j1 = -1;
        const bool in = live && safety_pass1(v, t32, p, p32, st);
        const int bin = in ? (st.j1 < 0 ? 0 : 1 + t32[st.j1].kind) : -1;
        s_p[0][t] = p[0];
        s_p[1][t] = p[1];
        s_p[2][t] = p[2];
        s_task[t] = st.j1;
        if (t < 4) s_cnt[t] = 0;
        __syncthreads();
        const int slot = bin >= 0 ? atomicAdd(&s_cnt[bin], 1) : 0;
        __syncthreads();
        int start = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < bin) start += s_cnt[q];
        if (bin >= 0) s_list[start + slot] = t;
        const int total = s_cnt[0] + s_cnt[1] + s_cnt[2] + s_cnt[3];
        __syncthreads();
        for (int q = t; q < total; q += 256) {
            const int o = s_list[q];
            const double po[3] = {s_p[0][o], s_p[1][o], s_p[2][o]};
            s_res[o] = safety_of(v, s_task[o], po);
        }
        __syncthreads();
        if (live) {
            double s = 0.0;
            if (in) {
                int nev;
                s = safety_finish(v, t32, p, p32, st, s_res[t], tau, &nev);
            }
            saf[i] = s;
        }
        __syncthreads();   // the tile's shared arrays are rewritten next
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
