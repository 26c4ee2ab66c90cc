// nav_refine.cu -- the navigator step of Fig. 1b with an FP32 filter and FP64
// refinement (GEO_FP32_REFINE).
//
// Pass 1 (FP32, every daughter): bounding-sphere cull against an upper bound
// U of the mother exit, master->local transform in a frame shifted to the
// track's closest approach to the daughter's origin, and a LOWER bound L_j of
// DistFromOutside from the daughter's inflated FP32 copy (shapes32.cuh).  The
// K smallest bounds are kept in registers, sorted.
// Pass 2 (FP64, few solids): candidates are refined in ascending order of
// their bounds, the mother (bound L_m of its exit) taking its place in that
// order, with the same FP64 routines as the plain kernel; refinement stops as
// soon as the next bound exceeds the best FP64 step.  Ties resolve as in the
// sequential algorithm of Fig. 1a (mother, then lowest index).  If a bound
// that had to be dropped from the list could still win, the track falls back
// to the full FP64 loop.  Every track therefore gets exactly the plain FP64
// kernel's answer.
#include <cuda_runtime.h>
#include "geo_internal.h"
#include "launch.cuh"
#include "nav_common.cuh"
#include "nav_refine.cuh"
#include "stage.cuh"

namespace geonav {

// Tracks are processed in tiles of one block (256).  After the FP32 pass each
// track names the first solid it must evaluate in FP64; these tasks are
// binned by solid kind (mother, box, tube, cone) in shared memory so that the
// FP64 evaluations run with whole warps on one code path: on this part the
// FP64 pipe issues one warp instruction per ~19 cycles per SM whether 1 or 32
// lanes are active, so divergent refinement would multiply its cost.  The
// remaining refinement (rare: a second candidate within the bounds) runs per
// thread.
constexpr int kTile = 256;

template <bool SMEM>
__global__ void __launch_bounds__(kTile, 2) k_dist_refine(VolView v, Basket b, double* __restrict__ step,
                                                       int32_t* __restrict__ hit, double* __restrict__ bpoint,
                                                       int32_t* __restrict__ nref) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ double s_pd[6][kTile];
    __shared__ double s_res[kTile];
    __shared__ int s_task[kTile];
    __shared__ int s_bins[4];
    const ShapeRec32* tab32 = v.d32;
    const ShapeRec64* tab64 = v.d64;
    if (SMEM) {
        const uint32_t b32 = uint32_t(v.nd) * sizeof(ShapeRec32);
        if (!stage_tables(smem_raw, v.d32, b32, smem_raw + b32, v.d64, uint32_t(v.nd) * sizeof(ShapeRec64), &bar,
                          v.status))
            return;
        tab32 = reinterpret_cast<const ShapeRec32*>(smem_raw);
        tab64 = reinterpret_cast<const ShapeRec64*>(smem_raw + b32);
    }
    const int t = threadIdx.x;
    for (int64_t base = int64_t(blockIdx.x) * kTile; base < b.n; base += int64_t(gridDim.x) * kTile) {
        const int64_t i = base + t;
        const bool live = i < b.n;
        double px = 0, py = 0, pz = 0, qx = 1, qy = 0, qz = 0;
        if (live) {
            px = b.x[i]; py = b.y[i]; pz = b.z[i];
            qx = b.dx[i]; qy = b.dy[i]; qz = b.dz[i];
        }
        s_pd[0][t] = px; s_pd[1][t] = py; s_pd[2][t] = pz;
        s_pd[3][t] = qx; s_pd[4][t] = qy; s_pd[5][t] = qz;
        RefineState st;
        double best = 0.0;
        int h = -2, nev = 0;
        st.status = 1;
        if (live) refine_pass1(v, tab32, tab64, px, py, pz, qx, qy, qz, st, best, h, nev);
        // ---- bin the first FP64 task of every track by solid kind ----
        int task = 0, bin = -1;
        if (st.status == 0) {
            task = first_task(st);
            bin = task < 0 ? 0 : 1 + tab64[task].kind;
        }
        if (t < 4) s_bins[t] = 0;
        __syncthreads();
        const int slot = bin >= 0 ? atomicAdd(&s_bins[bin], 1) : 0;
        __syncthreads();
        int start = 0, total = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = s_bins[k];
            if (k < bin) start += c;
            total += c;
        }
        if (bin >= 0) s_task[start + slot] = t | ((task + 1) << 8);
        __syncthreads();
        // ---- one kind-uniform FP64 evaluation per thread ----
        if (t < total) {
            const int e = s_task[t];
            const int owner = e & (kTile - 1), j = (e >> 8) - 1;
            s_res[owner] = eval64(v, tab64, j, s_pd[0][owner], s_pd[1][owner], s_pd[2][owner], s_pd[3][owner],
                                  s_pd[4][owner], s_pd[5][owner]);
        }
        __syncthreads();
        if (st.status == 0) refine_rest(v, tab64, st, s_res[t], px, py, pz, qx, qy, qz, best, h, nev);
        if (live) {
            store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
            if (nref) nref[i] = nev;
        }
        __syncthreads();   // s_pd / s_res are reused by the next tile
    }
}

cudaError_t launch_dist_refine_stats(const VolView& v, const Basket& b, double* step, int32_t* hit,
                                     double* bpoint, int32_t* nref, cudaStream_t s, int num_sms) {
    const int smem = v.smem_refine ? v.nd * int(sizeof(ShapeRec64) + sizeof(ShapeRec32)) : 0;
    if (v.smem_refine) {
        cudaError_t e = prep(k_dist_refine<true>, smem);
        if (e != cudaSuccess) return e;
        k_dist_refine<true><<<blocks_for(k_dist_refine<true>, b.n, smem, num_sms), kTile, smem, s>>>(
            v, b, step, hit, bpoint, nref);
    } else {
        k_dist_refine<false><<<blocks_for(k_dist_refine<false>, b.n, 0, num_sms), kTile, 0, s>>>(
            v, b, step, hit, bpoint, nref);
    }
    return cudaGetLastError();
}

cudaError_t launch_dist_refine(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                               cudaStream_t s, int num_sms) {
    return launch_dist_refine_stats(v, b, step, hit, bpoint, nullptr, s, num_sms);
}

}  // namespace geonav
