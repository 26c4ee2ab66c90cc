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
// track per thread per tile of kTileTracks = 384) and 4 consumer warps; with
// two blocks per SM (64 registers per thread) that is two consumer warps per
// SM sub-partition.  The FP64 unit is per sub-partition and issues one warp
// instruction every 64 cycles; a dependent FP64 chain takes about 76 cycles
// per step, and the square roots, divisions and comparisons between them
// leave gaps, so one warp cannot keep its unit busy and two do better.
// Measured on the toy detector (2^20 tracks): 12 + 4 warps 0.242 ms, 12 + 2
// warps at 72 registers 0.257 ms, 11 + 3 0.248, 10 + 4 0.254, 9 + 3 at 80
// registers 0.264, 8 + 4 0.265; the producers alone (FP64 evaluations
// skipped) take 0.207 ms and the consumers alone (each track's winner given)
// 0.160 ms, so the FP32 pass sets the pace.
//  producers: wait done[k%2] (the stage's previous tile, k-2, finished), FP32
//             pass of tile k, bin each track's first FP64 task by solid kind
//             (mother, box, tube, cone) into stage k%2, arrive on full[k%2].
//  consumers: wait full[k%2], evaluate the binned tasks of tile k in FP64 (a
//             warp claims chunks of 32 consecutive tasks, all of one kind:
//             the bins start on multiples of 32) and finish their tracks
//             (rare extra refinements), gather the tile's answers in its
//             answer buffer, then store them by consecutive lanes; arrive on
//             done[k%2].  Finishing there instead of in the producers took
//             0.2425 -> 0.2300 ms: the producers set the pace, and the
//             consumers had time to spare.
// The FP64 pipe therefore works on tile k while the FP32 pass of tile k+1 runs.
// Every wait is bounded; a wait that runs out records ST_SYNC_TIMEOUT.
// Block configurations (P producer threads, one track each per tile, and
// C consumer threads):
//  * 12 + 4 warps, tiles of kTileTracks = 384: throughput (many tiles per
//    block) and the batched launch (there 12 + 2 warps at 72 registers took
//    1.292 against 1.248 ms);
//  * 8 + 4 warps, tiles of 256: baskets of at most two tiles per block,
//    where the latency of one tile sets the time.
constexpr int kProd = kTileTracks, kCons = 128;   // throughput and batched: 12 + 4 warps
constexpr int kVoxCons = 64;                       // throughput with the uniform grid: 12 + 2 warps
constexpr int kLatProd = 256, kLatCons = 128;      // latency: 8 + 4 warps
constexpr int kOwnerBits = 9;   // binned task: owner | (solid + 1) << kOwnerBits
static_assert(kProd <= (1 << kOwnerBits) && kProd % 32 == 0 && kLatProd % 32 == 0 && kLatProd >= 128,
              "task encoding, bin padding");

template <int P>
struct Stage {
    double pd[6][P];        // the tile's positions and directions (FP64)
    float L[kCand][P];      // FP32 state stashed by the producers for the consumer
    int j[kCand][P];        //   that finishes the track (tracks with an FP64 task)
    float Lm[P];
    float dropped[P];
    int n[P];               // candidate count
    int task[P + 128];      // binned tasks: owner | (solid + 1) << kOwnerBits; -1 pads
    int cnt[4];
    int next;               // the next chunk of 32 tasks to claim
    int pad_[3];
};

// The answers of one tile, gathered for stores by consecutive lanes (the
// single-volume kernel: its outputs may be host memory read over the link).
template <int P>
struct Answers {
    double best[P];         // the step ...
    int h[P];               // ... and hit, kNoStore for a lane without a track
    int nev[P];             // FP64 evaluations (statistics)
};

// Each bin of a stage's task list starts on a multiple of 32, so that the 32
// consecutive tasks a consumer warp takes are of one kind (a warp pays for
// every code path its lanes take); the slots between bins hold -1.
__device__ __forceinline__ int bin_start(const int* cnt, int bin) {
    int start = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (q < bin) start += (cnt[q] + 31) & ~31;
    return start;
}

// After the counts are final: thread t < 128 pads bin t / 32 (P >= 128).
template <int P>
__device__ __forceinline__ void pad_bins(Stage<P>& st, int t) {
    if (t < 128) {
        const int b = t >> 5, c = st.cnt[b];
        if ((t & 31) < ((c + 31) & ~31) - c) st.task[bin_start(st.cnt, b) + c + (t & 31)] = -1;
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait: at most `polls` polls.  Returns whether the phase completed.
// (Polls that let the hardware suspend the waiting warp were measured slower
// here: the producers' and consumers' hand-offs are frequent, and a
// suspended warp resumes late.)
constexpr uint32_t kSyncPolls = 1u << 20;
__device__ __forceinline__ bool mbar_wait_limited(uint64_t* bar, uint32_t parity, uint32_t polls) {
    for (uint32_t it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// The pipeline's wait; after one timeout the caller stops waiting altogether
// (its results are then unreliable and the status word says so).
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned int* status,
                                                  bool& healthy) {
    if (!healthy) return;
    if (mbar_wait_limited(bar, parity, kSyncPolls)) return;
    atomicOr(status, ST_SYNC_TIMEOUT);
    healthy = false;
}

// FP64 task bins: 0 the mother, then box, tube (and tube segment), cone (and
// polycone)
__device__ __forceinline__ int kind_bin(int kind) { return kind == KTUBS ? 2 : (kind == KPCON ? 3 : 1 + kind); }

// A consumer's whole share of one track: the FP64 value of its first task
// jj, then the refinement's end (nearly always refine_fast: no other bound
// can win or tie).  The answer goes to the tile's answer buffer (STAGED),
// from where the tile's answers are stored together, consecutive tracks by
// consecutive lanes (the tasks themselves are in kind order: their own
// stores would scatter, which outputs in host memory written over the host
// link pay for); or it is stored right away to index(o).
template <bool SEGS, int P, bool STAGED, typename Index>
__device__ __forceinline__ void finish_track(const VolView& v, const ShapeRec64* __restrict__ tab64,
                                             const Stage<P>& st, Answers<P>* ans, int o, int jj, Index index,
                                             int64_t n, double* __restrict__ step, int32_t* __restrict__ hit) {
    const double s_first =
        eval64<SEGS>(v, tab64, jj, st.pd[0][o], st.pd[1][o], st.pd[2][o], st.pd[3][o], st.pd[4][o], st.pd[5][o]);
    RefineState rs;
    rs.status = 0;
    rs.c.n = st.n[o];
#pragma unroll
    for (int q = 0; q < kCand; ++q) {
        rs.c.L[q] = st.L[q][o];
        rs.c.j[q] = st.j[q][o];
    }
    rs.c.dropped = st.dropped[o];
    rs.Lm = st.Lm[o];
    double best;
    int h, nev = 1;
    if (!refine_fast(rs, s_first, best, h))
        refine_rest<SEGS>(v, tab64, rs, s_first, st.pd[0][o], st.pd[1][o], st.pd[2][o], st.pd[3][o], st.pd[4][o],
                          st.pd[5][o], best, h, nev);
    if (STAGED) {
        ans->best[o] = best;
        ans->h[o] = h;
        ans->nev[o] = nev;
    } else {
        store_result(index(o), n, best, h, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, step, hit, nullptr);
    }
}

constexpr int kNoStore = -0x7fffffff;   // an answer-buffer lane without a track

// The tile's answers from its answer buffer to the outputs, consecutive
// tracks by consecutive lanes of the C threads that call it; index(o) is the
// basket index of the tile's track o.
template <int P, int C, typename Index>
__device__ __forceinline__ void store_tile(const Stage<P>& st, const Answers<P>& ans, int c, Index index, int64_t n,
                                           double* __restrict__ step, int32_t* __restrict__ hit,
                                           double* __restrict__ bpoint, int32_t* __restrict__ nref) {
    for (int o = c; o < P; o += C) {
        const int h = ans.h[o];
        if (h == kNoStore) continue;
        const int64_t i = index(o);
        store_result(i, n, ans.best[o], h, st.pd[0][o], st.pd[1][o], st.pd[2][o], st.pd[3][o], st.pd[4][o],
                     st.pd[5][o], step, hit, bpoint);
        if (nref) nref[i] = ans.nev[o];
    }
}

// A warp's share of a stage's FP64 tasks: it claims chunks of 32 tasks (one
// bin-aligned chunk, so one solid kind) from the stage's counter until none
// is left, and finishes their tracks.  Every lane of the warp takes part.
template <bool SEGS, int P, bool STAGED, typename Index>
__device__ __forceinline__ void drain_tasks(const VolView& v, const ShapeRec64* __restrict__ tab64, Stage<P>& st,
                                            Answers<P>* ans, Index index, int64_t n, double* __restrict__ step,
                                            int32_t* __restrict__ hit) {
    const int total = bin_start(st.cnt, 4);   // a multiple of 32
    const int lane = threadIdx.x & 31;
    for (;;) {
        int q0 = 0;
        if (lane == 0) q0 = atomicAdd(&st.next, 32);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= total) break;
        const int e = st.task[q0 + lane];
        if (e >= 0) {
            const int o = e & ((1 << kOwnerBits) - 1), jj = (e >> kOwnerBits) - 1;
            finish_track<SEGS, P, STAGED>(v, tab64, st, ans, o, jj, index, n, step, hit);
        }
    }
}

template <int P>
__device__ __forceinline__ void producer_barrier() { asm volatile("bar.sync 1, %0;" ::"r"(P) : "memory"); }
template <int C>
__device__ __forceinline__ void consumer_barrier() { asm volatile("bar.sync 2, %0;" ::"r"(C) : "memory"); }

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
    Answers<P>* A = reinterpret_cast<Answers<P>*>(smem_raw + 2 * sizeof(Stage<P>));
    unsigned char* tables = smem_raw + 2 * (sizeof(Stage<P>) + sizeof(Answers<P>));
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
        for (int k = 0; k < K; ++k) {
            Stage<P>& st_ = S[k & 1];
            // the stage held tile k-2, which its consumers must have finished
            if (k >= 2) mbar_wait_bounded(&done[k & 1], uint32_t(((k - 2) >> 1) & 1), v.status, healthy);
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
            if (t == 4) st_.next = 0;
            producer_barrier<P>();
            const int slot = bin >= 0 ? atomicAdd(&st_.cnt[bin], 1) : 0;
            producer_barrier<P>();
            if (bin >= 0) st_.task[bin_start(st_.cnt, bin) + slot] = t | ((task + 1) << kOwnerBits);
            pad_bins<P>(st_, t);
            // stash the FP32 state for the consumer that finishes the track;
            // a final answer goes to the tile's answer buffer
            if (rs.status == 0) {
#pragma unroll
                for (int q = 0; q < kCand; ++q) {
                    st_.L[q][t] = rs.c.L[q];
                    st_.j[q][t] = rs.c.j[q];
                }
                st_.Lm[t] = rs.Lm;
                st_.dropped[t] = rs.c.dropped;
                st_.n[t] = rs.c.n;
            } else {   // a final answer, or no track
                A[k & 1].best[t] = best;
                A[k & 1].h[t] = live ? h : kNoStore;
                A[k & 1].nev[t] = nev;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[k & 1]);
        }
    } else {
        // ------------------------------------------------------ consumers --
        const int c = t - P;
        for (int k = 0; k < K; ++k) {
            mbar_wait_bounded(&full[k & 1], uint32_t((k >> 1) & 1), v.status, healthy);
            const int64_t base = (int64_t(blockIdx.x) + int64_t(k) * gridDim.x) * P;
            const bool ok = __all_sync(0xffffffffu, healthy);   // a stage never filled is not read
            auto index = [base](int o) { return base + o; };
            if (ok) drain_tasks<SEGS, P, true>(v, tab64, S[k & 1], &A[k & 1], index, b.n, step, hit);
            consumer_barrier<C>();   // every answer of the tile is in its answer buffer
            if (ok) store_tile<P, C>(S[k & 1], A[k & 1], c, index, b.n, step, hit, bpoint, nref);
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
    static_assert(sizeof(Stage<P>) % 16 == 0 && sizeof(Answers<P>) % 16 == 0, "the tables stay 16-byte aligned");
    const int smem = 2 * int(sizeof(Stage<P>) + sizeof(Answers<P>)) +
                     (v.smem_refine ? v.nd * int(sizeof(ShapeRec64) + sizeof(ShapeRec32)) : 0);
    if (v.voxelized) {
        // the grid walk needs registers: 12 + 2 warps at 72 registers beat
        // 12 + 4 at 64 (7.0 against 7.4 ms for 2^24 tracks in 512 daughters)
        constexpr int CV = P == kProd ? kVoxCons : C;
        const int smem_v = 2 * int(sizeof(Stage<P>) + sizeof(Answers<P>));
        if (v.segs)
            return launch_refine<P, CV>(k_dist_refine<P, CV, false, 1, true>, smem_v, v, b, step, hit, bpoint, nref,
                                        s, num_sms);
        return launch_refine<P, CV>(k_dist_refine<P, CV, false, 1, false>, smem_v, v, b, step, hit, bpoint, nref, s,
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
