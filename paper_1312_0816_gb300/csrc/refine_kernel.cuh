// refine_kernel.cuh -- the warp-specialised FP32-filter + FP64-refine kernel
// (one volume) and its launch templates, shared by the translation units that
// instantiate its two block configurations (nav_refine.cu: throughput;
// nav_refine_lat.cu: latency).  See nav_refine.cu for the scheme.
#pragma once
#include <cuda_runtime.h>
#include "geo_internal.h"
#include "launch.cuh"
#include "nav_common.cuh"
#include "nav_refine.cuh"
#include "stage.cuh"

namespace geonav {

// Warp-specialised persistent kernel.  A block holds 12 producer warps (one
// track per thread per tile of kTileTracks = 384) and 2 consumer warps; with
// two blocks per SM that is one consumer warp per SM sub-partition (the FP64
// units are per sub-partition, and the microbenchmark shows one warp with a
// dependent FP64 chain keeps one busy).  The FP32 pass sets the pace, and its
// latency is hidden by warps: on the toy detector 12 + 2 warps at a cap of 72
// registers take 0.31 ms where 8 + 4 warps at 80 registers took 0.35 ms (one
// consumer warp per block: 0.45 ms; at 64 registers: 0.33-0.37 ms).
//  producers: FP32 pass of tile k, then bin each track's first FP64 task by
//             solid kind (mother, box, tube, cone) into stage k%2, arrive on
//             full[k%2]; then wait done[(k-1)%2] and finish tile k-1 (rare
//             extra refinements, stores).
//  consumers: wait full[k%2], evaluate the binned tasks of tile k in FP64 (a
//             warp takes 32 consecutive tasks, so nearly always one kind),
//             arrive on done[k%2].
// The FP64 pipe therefore works on tile k while the FP32 pass of tile k+1 runs.
// Every wait is bounded; a wait that runs out records ST_SYNC_TIMEOUT.
// Two block configurations (P producer threads, one track each per tile, and
// C consumer threads):
//  * 12 + 2 warps, tiles of kTileTracks = 384: throughput (many tiles per
//    block; the batched launch);
//  * 8 + 4 warps, tiles of 256: baskets of at most two tiles per block,
//    where the latency of a tile's FP64 phase with 2 consumer warps would
//    set the time (1024 tracks: 32 us per call instead of 46 us).
constexpr int kProd = kTileTracks;   // the batched launch
constexpr int kCons = 64;
constexpr int kThreads = kProd + kCons;
constexpr int kLatProd = 256, kLatCons = 128;
constexpr int kOwnerBits = 9;   // binned task: owner | (solid + 1) << kOwnerBits
static_assert(kProd <= (1 << kOwnerBits) && kProd % 32 == 0 && kLatProd % 32 == 0, "task encoding");

template <int P>
struct Stage {
    double pd[6][P];        // the tile's positions and directions (FP64)
    double res[P];          // FP64 value of each track's first task
    float L[kCand][P];      // stashed FP32 state for the producers' second half
    int j[kCand][P];
    float Lm[P];
    float dropped[P];
    int n[P];               // candidate count, -1: answer already final
    int task[P];            // binned tasks: owner | (solid + 1) << kOwnerBits
    int cnt[4];
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait; after one timeout the caller stops waiting altogether (its
// results are then unreliable and the status word says so).
constexpr uint32_t kSyncPolls = 1u << 20;
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned int* status,
                                                  bool& healthy) {
    if (!healthy) return;
    for (uint32_t it = 0; it < kSyncPolls; ++it)
        if (mbar_try_wait(bar, parity)) return;
    atomicOr(status, ST_SYNC_TIMEOUT);
    healthy = false;
}

// FP64 task bins: 0 the mother, then box, tube (and tube segment), cone (and
// polycone)
__device__ __forceinline__ int kind_bin(int kind) { return kind == KTUBS ? 2 : (kind == KPCON ? 3 : 1 + kind); }

template <int P>
__device__ __forceinline__ void producer_barrier() { asm volatile("bar.sync 1, %0;" ::"r"(P) : "memory"); }

template <int P, int C, bool SMEM, int TRAV, bool SEGS>
__global__ void __launch_bounds__(P + C, 2) k_dist_refine(VolView v, Basket b, double* __restrict__ step,
                                                             int32_t* __restrict__ hit,
                                                             double* __restrict__ bpoint,
                                                             int32_t* __restrict__ nref) {
    // dynamic shared memory: the two stages, then (SMEM) the solid tables
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint64_t full[2], done[2];
    Stage<P>* S = reinterpret_cast<Stage<P>*>(smem_raw);
    unsigned char* tables = smem_raw + 2 * sizeof(Stage<P>);
    const ShapeRec32* tab32 = v.d32;
    const ShapeRec64* tab64 = v.d64;
    if (SMEM) {
        const uint32_t b32 = uint32_t(v.nd) * sizeof(ShapeRec32);
        if (!stage_tables(tables, v.d32, b32, tables + b32, v.d64, uint32_t(v.nd) * sizeof(ShapeRec64), &bar,
                          v.status))
            return;
        tab32 = reinterpret_cast<const ShapeRec32*>(tables);
        tab64 = reinterpret_cast<const ShapeRec64*>(tables + b32);
    }
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&full[0], P / 32);
        mbar_init(&full[1], P / 32);
        mbar_init(&done[0], C / 32);
        mbar_init(&done[1], C / 32);
    }
    __syncthreads();
    const int64_t ntiles = (b.n + P - 1) / P;
    const int K = int((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);   // tiles of this block
    const int lane = t & 31;
    bool healthy = true;

    if (t < P) {
        // ------------------------------------------------------ producers --
        for (int k = 0; k <= K; ++k) {
            if (k < K) {
                Stage<P>& st_ = S[k & 1];
                const int64_t i = (int64_t(blockIdx.x) + int64_t(k) * gridDim.x) * P + t;
                const bool live = i < b.n;
                double px = 0, py = 0, pz = 0, qx = 1, qy = 0, qz = 0;
                if (live) {
                    px = b.x[i]; py = b.y[i]; pz = b.z[i];
                    qx = b.dx[i]; qy = b.dy[i]; qz = b.dz[i];
                }
                st_.pd[0][t] = px; st_.pd[1][t] = py; st_.pd[2][t] = pz;
                st_.pd[3][t] = qx; st_.pd[4][t] = qy; st_.pd[5][t] = qz;
                RefineState rs;
                double best = 0.0;
                int h = -2, nev = 0;
                rs.status = 1;
                if (live) refine_pass1<TRAV, SEGS>(v, tab32, tab64, px, py, pz, qx, qy, qz, rs, best, h, nev);
                int task = 0, bin = -1;
                if (rs.status == 0) {
                    task = first_task(rs);
                    bin = task < 0 ? 0 : kind_bin(tab64[task].kind);
                }
                if (t < 4) st_.cnt[t] = 0;
                producer_barrier<P>();
                const int slot = bin >= 0 ? atomicAdd(&st_.cnt[bin], 1) : 0;
                producer_barrier<P>();
                int start = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < bin) start += st_.cnt[q];
                if (bin >= 0) st_.task[start + slot] = t | ((task + 1) << kOwnerBits);
                // stash the FP32 state; final answers are stored right away
                if (rs.status == 0) {
#pragma unroll
                    for (int q = 0; q < kCand; ++q) {
                        st_.L[q][t] = rs.c.L[q];
                        st_.j[q][t] = rs.c.j[q];
                    }
                    st_.Lm[t] = rs.Lm;
                    st_.dropped[t] = rs.c.dropped;
                    st_.n[t] = rs.c.n;
                } else {
                    st_.n[t] = -1;
                    if (live) {
                        // the track is read back from the stage: keeping it in
                        // registers through the FP32 pass would spill
                        store_result(i, b.n, best, h, st_.pd[0][t], st_.pd[1][t], st_.pd[2][t], st_.pd[3][t],
                                     st_.pd[4][t], st_.pd[5][t], step, hit, bpoint);
                        if (nref) nref[i] = nev;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[k & 1]);
            }
            if (k >= 1) {
                const int kp = k - 1;
                Stage<P>& sp = S[kp & 1];
                mbar_wait_bounded(&done[kp & 1], uint32_t((kp >> 1) & 1), v.status, healthy);
                const int64_t i = (int64_t(blockIdx.x) + int64_t(kp) * gridDim.x) * P + t;
                if (i < b.n && sp.n[t] >= 0) {
                    RefineState rs;
                    rs.status = 0;
                    rs.c.n = sp.n[t];
#pragma unroll
                    for (int q = 0; q < kCand; ++q) {
                        rs.c.L[q] = sp.L[q][t];
                        rs.c.j[q] = sp.j[q][t];
                    }
                    rs.c.dropped = sp.dropped[t];
                    rs.Lm = sp.Lm[t];
                    double best;
                    int h, nev = 1;
                    if (!refine_fast(rs, sp.res[t], best, h))
                        refine_rest<SEGS>(v, tab64, rs, sp.res[t], sp.pd[0][t], sp.pd[1][t], sp.pd[2][t], sp.pd[3][t],
                                          sp.pd[4][t], sp.pd[5][t], best, h, nev);
                    store_result(i, b.n, best, h, sp.pd[0][t], sp.pd[1][t], sp.pd[2][t], sp.pd[3][t], sp.pd[4][t],
                                 sp.pd[5][t], step, hit, bpoint);
                    if (nref) nref[i] = nev;
                }
            }
        }
    } else {
        // ------------------------------------------------------ consumers --
        const int c = t - P;
        for (int k = 0; k < K; ++k) {
            Stage<P>& st_ = S[k & 1];
            mbar_wait_bounded(&full[k & 1], uint32_t((k >> 1) & 1), v.status, healthy);
            const int total = st_.cnt[0] + st_.cnt[1] + st_.cnt[2] + st_.cnt[3];
            for (int q = c; q < total; q += C) {
                const int e = st_.task[q];
                const int o = e & ((1 << kOwnerBits) - 1), jj = (e >> kOwnerBits) - 1;
                st_.res[o] = eval64<SEGS>(v, tab64, jj, st_.pd[0][o], st_.pd[1][o], st_.pd[2][o], st_.pd[3][o],
                                    st_.pd[4][o], st_.pd[5][o]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[k & 1]);
        }
    }
}

template <int P, int C, typename K>
static int grid_refine(K kernel, int64_t n, int smem, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, P + C, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t need = (n + P - 1) / P;
    const int64_t cap = int64_t(per_sm) * num_sms;
    return int(need < cap ? need : cap);
}

template <int P, int C, typename K>
static cudaError_t launch_refine(K kernel, int smem, const VolView& v, const Basket& b, double* step, int32_t* hit,
                                 double* bpoint, int32_t* nref, cudaStream_t s, int num_sms) {
    cudaError_t e = prep(kernel, smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid_refine<P, C>(kernel, b.n, smem, num_sms), P + C, smem, s>>>(v, b, step, hit, bpoint, nref);
    return cudaGetLastError();
}

// SEGS: the instantiation with the tube segment's and the polycone's code
// only for volumes that hold one, so the others keep the leaner kernel
template <int P, int C>
static cudaError_t launch_refine_cfg(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                                     int32_t* nref, cudaStream_t s, int num_sms) {
    static_assert(sizeof(Stage<P>) % 16 == 0, "stage size keeps the tables 16-byte aligned");
    const int smem = 2 * int(sizeof(Stage<P>)) +
                     (v.smem_refine ? v.nd * int(sizeof(ShapeRec64) + sizeof(ShapeRec32)) : 0);
    if (v.voxelized) {
        if (v.segs)
            return launch_refine<P, C>(k_dist_refine<P, C, false, 1, true>, smem, v, b, step, hit, bpoint, nref, s,
                                       num_sms);
        return launch_refine<P, C>(k_dist_refine<P, C, false, 1, false>, smem, v, b, step, hit, bpoint, nref, s,
                                   num_sms);
    }
    if (v.smem_refine) {
        if (v.segs)
            return launch_refine<P, C>(k_dist_refine<P, C, true, 0, true>, smem, v, b, step, hit, bpoint, nref, s,
                                       num_sms);
        return launch_refine<P, C>(k_dist_refine<P, C, true, 0, false>, smem, v, b, step, hit, bpoint, nref, s,
                                   num_sms);
    }
    if (v.segs)
        return launch_refine<P, C>(k_dist_refine<P, C, false, 0, true>, smem, v, b, step, hit, bpoint, nref, s,
                                   num_sms);
    return launch_refine<P, C>(k_dist_refine<P, C, false, 0, false>, smem, v, b, step, hit, bpoint, nref, s,
                               num_sms);
}

}  // namespace geonav
