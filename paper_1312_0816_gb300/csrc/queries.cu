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

// Contains: per tile of 256 points, the FP32 tests run per thread and give
// each point its first candidate (the first daughter whose inflated copy
// holds it); the FP64 decisions for those candidates are binned by solid
// kind and taken by whole warps over the binned list, as in the Safety
// kernel below (the FP64 pipe charges a warp instruction whatever its active
// lanes, and a thread-per-point loop runs the FP64 test once for every
// daughter that any lane of the warp stops at).  A point whose candidate
// fails goes on with the remaining candidates on its own thread (rare).
template <bool SMEM, bool SEGS>
__global__ void __launch_bounds__(256) k_contains32(VolView v, Basket b, int32_t* __restrict__ where) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ double s_p[3][256];
    __shared__ int s_task[256];
    __shared__ int s_list[256];
    __shared__ unsigned char s_in[256];
    __shared__ int s_cnt[5];
    const ShapeRec32* t32 = v.d32;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d32, uint32_t(v.nd) * sizeof(ShapeRec32), &bar, v.status)) return;
        t32 = reinterpret_cast<const ShapeRec32*>(smem_raw);
    }
    const int t = threadIdx.x;
    const int64_t ntiles = (b.n + 255) / 256;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * 256 + t;
        const bool live = i < b.n;
        double p[3] = {0.0, 0.0, 0.0};
        float p32[3] = {0.f, 0.f, 0.f};
        if (live) point32(b, i, p, p32);
        int w = -2, j1 = -1;
        if (live && mother_contains<SEGS>(v, p, p32)) {
            w = -1;
            j1 = contains_next(v, t32, p32, 0);
        }
        const int kd = j1 >= 0 ? v.d64[j1].kind : -1;
        const int bin = (kd >= 0 && kd < 5) ? kd : -1;
        s_p[0][t] = p[0];
        s_p[1][t] = p[1];
        s_p[2][t] = p[2];
        s_task[t] = j1;
        if (t < 5) s_cnt[t] = 0;
        __syncthreads();
        const int slot = bin >= 0 ? atomicAdd(&s_cnt[bin], 1) : 0;
        __syncthreads();
        int start = 0;
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (q < bin) start += s_cnt[q];
        if (bin >= 0) s_list[start + slot] = t;
        const int total = s_cnt[0] + s_cnt[1] + s_cnt[2] + s_cnt[3] + s_cnt[4];
        __syncthreads();
        for (int q = t; q < total; q += 256) {
            const int o = s_list[q];
            const double po[3] = {s_p[0][o], s_p[1][o], s_p[2][o]};
            s_in[o] = contains_daughter64<SEGS>(v, s_task[o], po) ? 1 : 0;
        }
        __syncthreads();
        if (live) {
            if (bin >= 0) w = s_in[t] ? j1 : contains_rest<SEGS>(v, t32, p, p32, j1);
            else if (j1 >= 0) w = contains_filter<SEGS>(v, t32, p, p32);   // a kind outside the bins
            where[i] = w;
        }
        __syncthreads();   // the tile's shared arrays are rewritten next
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
//
// Six resident blocks per SM for the lean instantiation (40 registers, a few
// spills): on the toy detector 0.985 ms instead of 1.03 ms at 64 registers
// and four blocks; the instantiation with the segment and polycone code keeps
// two blocks without spills.
template <bool SMEM, bool SEGS>
__global__ void __launch_bounds__(256, SEGS ? 2 : 6) k_safety32(VolView v, Basket b, double* __restrict__ saf) {
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
        const bool in = live && safety_pass1<SEGS>(v, t32, p, p32, st);
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
            s_res[o] = safety_of<SEGS>(v, s_task[o], po);
        }
        __syncthreads();
        if (live) {
            double s = 0.0;
            if (in) {
                int nev;
                s = safety_finish<SEGS>(v, t32, p, p32, st, s_res[t], tau, &nev);
            }
            saf[i] = s;
        }
        __syncthreads();   // the tile's shared arrays are rewritten next
    }
}

// The under-estimating safety (GEO_SAFETY_ESTIMATE): the FP32 pass alone.
// Every solid's bound is its inflated (mother: deflated) FP32 copy's
// distance lowered by a relative 2^-18: box and tube the exact distance to
// the copy, cone the largest supporting half-plane distance, tube segment
// and polycone their enclosing tube, segment and polycone mothers 0; a
// daughter's bound is raised to the distance to its copy's bounding sphere
// where that is larger, so the sphere cull cannot change the minimum.  The
// minimum is a lower bound of the exact safety; no FP64 work but the
// mother's containment test where its FP32 copies cannot decide.
template <bool SMEM, bool SEGS>
__global__ void __launch_bounds__(256) k_safety_est(VolView v, Basket b, double* __restrict__ saf) {
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
        float L = 0.f;
        if (mother_contains<SEGS>(v, p, p32)) {
            L = safety_in_lb32(v.m32, p32);
            for (int j = 0; j < v.nd && L > 0.f; ++j) {
                const ShapeRec32& r = t32[j];
                float o[3], x[3];
                const float c2 = offset32(r, p32, o);
                if (beyond(r, c2, L)) continue;   // the whole copy is farther than L
                local32(r, o, x);
                L = fminf(L, fmaxf(safety_out_lb32(r, x), sphere_lb32(r, c2)));
            }
        }
        saf[i] = double(L);
    }
}

// the FP32 table staged when it fits; the polycone's code only for volumes
// holding segments or polycones
template <bool SEGS, typename K1, typename K0, typename... A>
static cudaError_t launch32(K1 staged, K0 global, const VolView& v, const Basket& b, cudaStream_t s, int num_sms,
                            A... args) {
    const int bytes = v.nd * int(sizeof(ShapeRec32));
    if (bytes <= kQueryTable32Max) {
        cudaError_t e = prep(staged, bytes);
        if (e != cudaSuccess) return e;
        staged<<<blocks_for(staged, b.n, bytes, num_sms), 256, bytes, s>>>(v, b, args...);
    } else {
        global<<<blocks_for(global, b.n, 0, num_sms), 256, 0, s>>>(v, b, args...);
    }
    return cudaGetLastError();
}

cudaError_t launch_contains_filter(const VolView& v, const Basket& b, int32_t* where, cudaStream_t s,
                                   int num_sms) {
    if (v.segs) return launch32<true>(k_contains32<true, true>, k_contains32<false, true>, v, b, s, num_sms, where);
    return launch32<false>(k_contains32<true, false>, k_contains32<false, false>, v, b, s, num_sms, where);
}

cudaError_t launch_safety_estimate(const VolView& v, const Basket& b, double* saf, cudaStream_t s, int num_sms) {
    if (v.segs) return launch32<true>(k_safety_est<true, true>, k_safety_est<false, true>, v, b, s, num_sms, saf);
    return launch32<false>(k_safety_est<true, false>, k_safety_est<false, false>, v, b, s, num_sms, saf);
}

cudaError_t launch_safety_filter(const VolView& v, const Basket& b, double* saf, cudaStream_t s, int num_sms) {
    if (v.segs) return launch32<true>(k_safety32<true, true>, k_safety32<false, true>, v, b, s, num_sms, saf);
    return launch32<false>(k_safety32<true, false>, k_safety32<false, false>, v, b, s, num_sms, saf);
}

}  // namespace geonav
