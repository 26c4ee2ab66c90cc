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

template <bool SMEM>
__global__ void __launch_bounds__(256) k_dist_refine(VolView v, Basket b, double* __restrict__ step,
                                                     int32_t* __restrict__ hit, double* __restrict__ bpoint,
                                                     int32_t* __restrict__ nref) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
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
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const double px = b.x[i], py = b.y[i], pz = b.z[i];
        const double qx = b.dx[i], qy = b.dy[i], qz = b.dz[i];
        double best;
        int h, nev;
        refine_track(v, tab32, tab64, px, py, pz, qx, qy, qz, best, h, nev);
        store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
        if (nref) nref[i] = nev;
    }
}

cudaError_t launch_dist_refine_stats(const VolView& v, const Basket& b, double* step, int32_t* hit,
                                     double* bpoint, int32_t* nref, cudaStream_t s, int num_sms) {
    const int smem = v.smem_refine ? v.nd * int(sizeof(ShapeRec64) + sizeof(ShapeRec32)) : 0;
    if (v.smem_refine) {
        cudaError_t e = prep(k_dist_refine<true>, smem);
        if (e != cudaSuccess) return e;
        k_dist_refine<true><<<blocks_for(k_dist_refine<true>, b.n, smem, num_sms), 256, smem, s>>>(
            v, b, step, hit, bpoint, nref);
    } else {
        k_dist_refine<false><<<blocks_for(k_dist_refine<false>, b.n, 0, num_sms), 256, 0, s>>>(v, b, step, hit,
                                                                                                 bpoint, nref);
    }
    return cudaGetLastError();
}

cudaError_t launch_dist_refine(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                               cudaStream_t s, int num_sms) {
    return launch_dist_refine_stats(v, b, step, hit, bpoint, nullptr, s, num_sms);
}

}  // namespace geonav
