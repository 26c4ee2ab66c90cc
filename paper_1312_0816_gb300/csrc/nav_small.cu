// nav_small.cu -- the FP32-filter step for small baskets in volumes of many
// daughters (the small-basket end of Fig. 3's basket-size axis): one warp per
// track.  The lanes share the track and split its daughters (lane l bounds
// daughters l, l + 32, ...) in FP32, as the filter kernel does per thread;
// the FP64 refinement then evaluates, round by round, every candidate whose
// bound does not exceed the best FP64 step so far (each lane its own next
// candidate, in parallel), and the mother when its bound does not; the warp
// takes the minimum over (step, index) with the ties of Fig. 1a (the mother,
// then the lowest index).  A candidate left out has a bound above the final
// step's FP32 upper bound, so it could neither win nor tie: the answer is the
// plain FP64 loop's, bit for bit.
//
// A one-track warp charges every FP64 instruction for 32 lanes, but a basket
// of a few tracks per SM is bound by the latency of one track's walk through
// its daughters, which the lanes cut by 32: on the toy detector (40
// daughters) one call on 16 or 1024 tracks.
#include <cuda_runtime.h>

#include "geo_internal.h"
#include "launch.cuh"
#include "nav_common.cuh"
#include "nav_refine.cuh"

namespace geonav {

// (value, index) minimum over the warp with the navigator's tie order: the
// smaller step (bit pattern of a value >= 0), then the smaller index (the
// mother is -1).  +inf with index INT_MAX marks an empty lane.
__device__ __forceinline__ void warp_min_pair(double& s, int& j) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, s, off);
        const int oj = __shfl_xor_sync(0xffffffffu, j, off);
        if (LT(os, s) || (BITS(os) == BITS(s) && oj < j)) {
            s = os;
            j = oj;
        }
    }
}

template <bool SEGS>
__global__ void __launch_bounds__(256) k_dist_warp_filter(VolView v, Basket b, double* __restrict__ step,
                                                         int32_t* __restrict__ hit, double* __restrict__ bpoint) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < b.n; i += nwarps) {
        const double px = b.x[i], py = b.y[i], pz = b.z[i];
        const double qx = b.dx[i], qy = b.dy[i], qz = b.dz[i];
        RefineState rs;
        double best;
        int h, nev;
        refine_pass1<0, SEGS>(v, v.d32, v.d64, px, py, pz, qx, qy, qz, rs, best, h, nev, lane, 32);
        if (rs.status == 0) {   // the same for every lane: it depends on the track only
            best = d_inf();
            h = INT_MAX;   // nothing yet
            bool mdone = false;
            int k = 0;     // this lane's next candidate
            for (;;) {
                const float up = LT(best, d_inf()) ? f64_to_f32_up(best) : f_inf();
                const bool mine = k < rs.c.n && rs.c.L[k] <= up;
                const bool moth = !mdone && rs.Lm <= up;
                if (!__any_sync(0xffffffffu, mine) && !moth) break;
                double s = d_inf();
                int j = INT_MAX;
                if (mine) {
                    j = rs.c.j[k];
                    s = eval64<SEGS>(v, v.d64, j, px, py, pz, qx, qy, qz);
                    ++k;
                }
                if (moth) {   // every lane the same value; it enters the minimum once, as index -1
                    const double sm = eval64<SEGS>(v, v.d64, -1, px, py, pz, qx, qy, qz);
                    mdone = true;
                    if (lane == 0 && (LT(sm, s) || (BITS(sm) == BITS(s)))) {
                        s = sm;
                        j = -1;
                    }
                }
                warp_min_pair(s, j);
                if (LT(s, best) || (BITS(s) == BITS(best) && j < h)) {
                    best = s;
                    h = j;
                }
            }
            // every lane's list holds all its daughters' bounds (at most two
            // daughters per lane for up to 64 daughters): none was dropped
        }
        if (lane == 0) store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
    }
}

bool small_basket_filter(const VolView& v, int64_t n, int num_sms) {
    return !v.voxelized && v.nd > 32 && v.nd <= 32 * kCand && n <= int64_t(kSmallFilterTracksPerSm) * num_sms;
}

cudaError_t launch_dist_warp_filter(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                                    cudaStream_t s, int num_sms) {
    const int64_t blocks = (b.n * 32 + 255) / 256;
    const int grid = int(blocks < int64_t(num_sms) * 8 ? blocks : int64_t(num_sms) * 8);
    if (v.segs) k_dist_warp_filter<true><<<grid, 256, 0, s>>>(v, b, step, hit, bpoint);
    else k_dist_warp_filter<false><<<grid, 256, 0, s>>>(v, b, step, hit, bpoint);
    return cudaGetLastError();
}

}  // namespace geonav
