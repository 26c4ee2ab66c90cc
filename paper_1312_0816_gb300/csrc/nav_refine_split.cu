// nav_refine_split.cu -- the filter step (GEO_FP32_REFINE) for small baskets
// in volumes of many daughters: one track's FP32 pass split over the warps of
// a block, daughter by daughter.
//
// A basket of a few thousand tracks leaves most of the GPU idle, and its time
// is the latency of one tile: in the pipelined kernel a warp walks every
// daughter of the volume for its 32 tracks, one after the other.  Here a block
// takes 32 tracks (one per lane) and kSplitWarps warps; warp w bounds the
// mother and daughters w, w + kSplitWarps, ... for all 32 tracks.  The warps'
// candidate lists are merged per track, and each track's first FP64 task is
// taken by the warp of its solid kind (mother, box, tube, cone: warps 0-3), so
// the lanes of a warp run one FP64 routine.  The merged list holds the
// smallest bounds over all daughters and the least of the bounds left out, so
// the refinement returns the plain FP64 bits, as every filter kernel does.
#include <cuda_runtime.h>
#include "geo_internal.h"
#include "launch.cuh"
#include "nav_common.cuh"
#include "nav_refine.cuh"
#include "refine_kernel.cuh"

namespace geonav {

constexpr int kSplitWarps = 8;
constexpr int kSplitBlocksPerSm = 4;   // resident blocks per SM (64 registers)
static_assert(kSplitWarps >= 4, "one warp per FP64 task kind");

struct SplitShared {
    float L[kSplitWarps][kCand][32];   // each warp's candidates, per lane (track)
    int j[kSplitWarps][kCand][32];
    int n[kSplitWarps][32];
    float dropped[kSplitWarps][32];
    float Lm[32];                      // the mother's bound (warp 0's copy)
    int status[32];                    // -1 no track, 0 refine, 1 final in the FP32 pass
    double best[32];
    int h[32];
    int nev[32];
};

template <bool SEGS>
__global__ void __launch_bounds__(kSplitWarps * 32, kSplitBlocksPerSm)
    k_dist_split(VolView v, Basket b, double* __restrict__ step, int32_t* __restrict__ hit,
                 double* __restrict__ bpoint, int32_t* __restrict__ nref) {
    __shared__ SplitShared sh;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = int64_t(blockIdx.x) * 32 + lane;
    const bool live = i < b.n;
    double px = 0, py = 0, pz = 0, qx = 1, qy = 0, qz = 0;
    if (live) {
        px = b.x[i]; py = b.y[i]; pz = b.z[i];
        qx = b.dx[i]; qy = b.dy[i]; qz = b.dz[i];
    }
    {
        RefineState rs;
        rs.status = 1;
        rs.c.n = 0;
        rs.c.dropped = f_inf();
        rs.Lm = 0.f;
#pragma unroll
        for (int q = 0; q < kCand; ++q) {
            rs.c.L[q] = f_inf();
            rs.c.j[q] = 0;
        }
        double best = 0.0;
        int h = -2, nev = 0;
        if (live) refine_pass1<0, SEGS>(v, v.d32, v.d64, px, py, pz, qx, qy, qz, rs, best, h, nev, w, kSplitWarps);
#pragma unroll
        for (int q = 0; q < kCand; ++q) {
            sh.L[w][q][lane] = rs.c.L[q];
            sh.j[w][q][lane] = rs.c.j[q];
        }
        sh.n[w][lane] = rs.status == 0 ? rs.c.n : 0;
        sh.dropped[w][lane] = rs.c.dropped;
        if (w == 0) {   // every warp bounded the mother alike
            sh.Lm[lane] = rs.Lm;
            sh.status[lane] = live ? rs.status : -1;
            sh.best[lane] = best;
            sh.h[lane] = h;
            sh.nev[lane] = nev;
        }
    }
    __syncthreads();
    if (w >= 4) return;
    const int status = sh.status[lane];
    if (status < 0) return;
    if (status != 0) {   // answered by the FP32 pass (invalid track, outside, fallback loop)
        if (w == 0) {
            store_result(i, b.n, sh.best[lane], sh.h[lane], px, py, pz, qx, qy, qz, step, hit, bpoint);
            if (nref) nref[i] = sh.nev[lane];
        }
        return;
    }
    // the warps' lists merged: the kCand smallest bounds, the least of the rest
    RefineState rs;
    rs.status = 0;
    rs.c.n = 0;
    rs.c.dropped = f_inf();
#pragma unroll
    for (int q = 0; q < kCand; ++q) {
        rs.c.L[q] = f_inf();
        rs.c.j[q] = 0;
    }
    rs.Lm = sh.Lm[lane];
#pragma unroll
    for (int u = 0; u < kSplitWarps; ++u) {
        const int nu = sh.n[u][lane];
#pragma unroll
        for (int q = 0; q < kCand; ++q)
            if (q < nu) cand_insert(rs.c, sh.L[u][q][lane], sh.j[u][q][lane]);
        rs.c.dropped = fminf(rs.c.dropped, sh.dropped[u][lane]);
    }
    const int task = first_task(rs);
    if ((task < 0 ? 0 : kind_bin(v.d64[task].kind)) != w) return;
    const double s_first = eval64<SEGS>(v, v.d64, task, px, py, pz, qx, qy, qz);
    double best;
    int h, nev = 1;
    if (!refine_fast(rs, s_first, best, h))
        refine_rest<SEGS>(v, v.d64, rs, s_first, px, py, pz, qx, qy, qz, best, h, nev);
    store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
    if (nref) nref[i] = nev;
}

// Volumes of more than 32 daughters (smaller volumes keep the warp-per-track
// kernel or the pipelined one), baskets that fill at most one wave of blocks
// (four 256-thread blocks per SM at 64 registers), two waves from 128
// daughters on in a volume without a uniform grid.  A volume with a grid is
// walked here daughter by daughter all the same: for a small basket the
// shared walk beats each lane's own walk through the cells.  Measured per
// call (CUDA graph of one call), pipelined kernel -> this one: toy detector
// (40 daughters) 16 tracks 21.8 -> 16.3 us, 1024 28.7 -> 18.3, 16384 30.7 ->
// 26.5, 32768 32.7 -> 40.9; 512 daughters without the grid 16 tracks 126.9
// -> 30.0 us, 16384 118.8 -> 34.8, 32768 118.8 -> 59.3, 65536 124.9 ->
// 100.3; the same with the grid (the pipelined kernel walking it) 16 tracks
// 45.0 -> 28.6 us, 16384 55.2 -> 34.8, 32768 55.3 -> 59.3.
bool split_basket(const VolView& v, int64_t n, int num_sms) {
    const int64_t wave = int64_t(kSplitBlocksPerSm) * num_sms * 32;
    return v.nd > 32 && n <= (v.nd >= 128 && !v.voxelized ? 2 : 1) * wave;
}

cudaError_t launch_dist_refine_split(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                                     int32_t* nref, cudaStream_t s) {
    if (b.n <= 0) return cudaSuccess;
    const unsigned blocks = unsigned((b.n + 31) / 32);
    if (v.segs)
        k_dist_split<true><<<blocks, kSplitWarps * 32, 0, s>>>(v, b, step, hit, bpoint, nref);
    else
        k_dist_split<false><<<blocks, kSplitWarps * 32, 0, s>>>(v, b, step, hit, bpoint, nref);
    return cudaGetLastError();
}

}  // namespace geonav
