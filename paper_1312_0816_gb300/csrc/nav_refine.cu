// nav_refine.cu -- the navigator step of Fig. 1b with an FP32 filter and FP64
// refinement (GEO_FP32_REFINE).
//
// Pass 1 (FP32, every daughter): bounding-sphere cull against an upper bound
// U of the mother exit, master->local transform in a frame shifted to the
// track's closest approach to the daughter's origin, and a LOWER bound L_j of
// DistFromOutside from the daughter's inflated FP32 copy (shapes32.cuh).  The
// kCand = 2 smallest bounds are kept in registers, sorted.
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
#include "refine_kernel.cuh"

namespace geonav {

size_t refine_stage_bytes() { return 2 * (sizeof(Stage<kProd>) + sizeof(Answers<kProd>)); }

// ---------------------------------------------------------------------------
// Batched persistent launch: tiles of many logical volumes, claimed in order
// from a device counter (largest estimated cost first when the host sorted
// them so), with the same producer / consumer pipeline.  The tile header of a
// stage carries a copy of the tile's volume view; the solid tables are read
// from global memory through L1 (a table change per tile would otherwise
// need a restage while the other stage still uses the previous one).  A
// packed tile (negative count) lists its tracks' indices in bv.idx from its
// base on (the ragged tails of a volume's baskets gathered into full tiles).
struct __align__(16) TileHdr {
    VolView vol;
    int64_t base;
    int count;
    int tile;   // -1: the queue is empty
    int vol_index;
    int pad[3];
};

// SEGS = false: no volume of the batch holds a tube segment or a polycone.
// VOX = false: no volume has a uniform grid, and the kernel carries only the
// all-daughter FP32 pass (10 % faster on the 64-volume batch than with the
// grid walk's code beside it).  P producer threads (one track each of a tile
// of P) and C consumer threads.
template <bool SEGS, bool VOX, int P, int C>
__global__ void __launch_bounds__(P + C, 2) k_dist_batched(BatchView bv, Basket b, double* __restrict__ step,
                                                              int32_t* __restrict__ hit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t full[2], done[2];
    Stage<P>* S = reinterpret_cast<Stage<P>*>(smem_raw);
    TileHdr* H = reinterpret_cast<TileHdr*>(smem_raw + 2 * sizeof(Stage<P>));
    const int t = threadIdx.x;
    const int lane = t & 31;
    bool healthy = true;
    if (t == 0) {
        mbar_init(&full[0], P / 32);
        mbar_init(&full[1], P / 32);
        mbar_init(&done[0], C / 32);
        mbar_init(&done[1], C / 32);
    }
    __syncthreads();
    constexpr int kWords = int(sizeof(VolView) / sizeof(int4));

    if (t < P) {
        // ------------------------------------------------------ producers --
        for (int k = 0;; ++k) {
            Stage<P>& st_ = S[k & 1];
            TileHdr& hd = H[k & 1];
            // the stage and its header held tile k-2, which its consumers must
            // have finished
            if (k >= 2) mbar_wait_bounded(&done[k & 1], uint32_t(((k - 2) >> 1) & 1), bv.status, healthy);
            if (t == 0) {
                const unsigned q = atomicAdd(bv.counter, 1u);
                if (int64_t(q) < bv.ntiles) {
                    const BatchTile tl = bv.tiles[q];
                    hd.tile = int(q);
                    hd.base = tl.base;
                    hd.count = tl.count;
                    hd.vol_index = tl.vol;
                } else {
                    hd.tile = -1;
                }
                st_.cnt[0] = st_.cnt[1] = st_.cnt[2] = st_.cnt[3] = 0;
                st_.next = 0;
            }
            producer_barrier<P>();
            const int tile = hd.tile;
            if (tile >= 0) {
                if (t < kWords)
                    reinterpret_cast<int4*>(&hd.vol)[t] = reinterpret_cast<const int4*>(bv.vols + hd.vol_index)[t];
                const int64_t base = hd.base;
                const bool packed = hd.count < 0;
                const int count = packed ? -hd.count : hd.count;
                producer_barrier<P>();
                const VolView& v = hd.vol;
                bool live = t < count;
                int64_t i = live ? (packed ? bv.idx[base + t] : base + t) : 0;
                if (live && (i < 0 || i >= b.n)) {   // a stale or corrupt tile list: skip, and say so
                    atomicOr(bv.status, ST_BAD_INDEX);
                    atomicOr(v.status, ST_BAD_INDEX);
                    live = false;
                    i = 0;
                }
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
                if (live) refine_pass1<VOX ? 2 : 0>(v, v.d32, v.d64, px, py, pz, qx, qy, qz, rs, best, h, nev);
                int task = 0, bin = -1;
                if (rs.status == 0) {
                    task = first_task(rs);
                    bin = task < 0 ? 0 : kind_bin(v.d64[task].kind);
                }
                const int slot = bin >= 0 ? atomicAdd(&st_.cnt[bin], 1) : 0;
                producer_barrier<P>();
                if (bin >= 0) st_.task[bin_start(st_.cnt, bin) + slot] = t | ((task + 1) << kOwnerBits);
                pad_bins<P>(st_, t);
                if (rs.status == 0) {
#pragma unroll
                    for (int q = 0; q < kCand; ++q) {
                        st_.L[q][t] = rs.c.L[q];
                        st_.j[q][t] = rs.c.j[q];
                    }
                    st_.Lm[t] = rs.Lm;
                    st_.dropped[t] = rs.c.dropped;
                    st_.n[t] = rs.c.n;
                } else if (live) {
                    store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, nullptr);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[k & 1]);
            if (tile < 0) break;
        }
    } else {
        // ------------------------------------------------------ consumers --
        for (int k = 0;; ++k) {
            Stage<P>& st_ = S[k & 1];
            TileHdr& hd = H[k & 1];
            mbar_wait_bounded(&full[k & 1], uint32_t((k >> 1) & 1), bv.status, healthy);
            // warp-uniform; all consumer warps see the same tile
            if (!__all_sync(0xffffffffu, healthy) || hd.tile < 0) break;
            const VolView& v = hd.vol;
            const int64_t base = hd.base;
            const bool packed = hd.count < 0;
            const int64_t* idx = bv.idx;
            // the outputs are in device memory: each track is stored as it is
            // finished (staging the tile's answers was 4 % slower here)
            drain_tasks<SEGS, P, false>(v, v.d64, st_, nullptr, [=](int o) { return packed ? idx[base + o] : base + o; },
                                        b.n, step, hit);
            __syncwarp();
            if (lane == 0) mbar_arrive(&done[k & 1]);
        }
    }
    // a wait that ran out is also reported in every volume's status word,
    // which geo_check_device_status reads
    if (!healthy)
        for (int q = 0; q < bv.nvols; ++q) atomicOr(bv.vols[q].status, ST_SYNC_TIMEOUT);
}

// A bounded wait that runs out: one warp waits, with `polls` polls of the
// pipeline's own wait (mbar_wait_limited), on an mbarrier that no thread
// arrives at, then records ST_SYNC_TIMEOUT in the status word and returns
// (the failure path of every wait of the pipeline, exercised on purpose by
// the tests).
__global__ void k_wait_selftest(unsigned int* status, uint32_t polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (mbar_wait_limited(&bar, 0, polls)) return;
    if (threadIdx.x == 0) atomicOr(status, ST_SYNC_TIMEOUT);
}

cudaError_t launch_wait_selftest(unsigned int* status, uint32_t polls, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, polls);
    return cudaGetLastError();
}

template <bool SEGS, bool VOX, int P, int C>
static int batched_blocks_per_sm() {
    static int cached = 0;
    if (cached == 0) {
        const int smem = 2 * int(sizeof(Stage<P>) + sizeof(TileHdr));
        int per_sm = 0;
        if (cudaFuncSetAttribute(k_dist_batched<SEGS, VOX, P, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dist_batched<SEGS, VOX, P, C>, P + C, smem) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        cached = per_sm;
    }
    return cached;
}

template <bool SEGS, bool VOX, int P, int C>
static cudaError_t launch_batched(const BatchView& bv, const Basket& b, double* step, int32_t* hit, int blocks_per_sm,
                                  cudaStream_t s, int num_sms) {
    const int smem = 2 * int(sizeof(Stage<P>) + sizeof(TileHdr));
    const int maxb = batched_blocks_per_sm<SEGS, VOX, P, C>();
    const int per_sm = (blocks_per_sm <= 0 || blocks_per_sm > maxb) ? maxb : blocks_per_sm;
    cudaError_t e =
        cudaFuncSetAttribute(k_dist_batched<SEGS, VOX, P, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_dist_batched<SEGS, VOX, P, C><<<per_sm * num_sms, P + C, smem, s>>>(bv, b, step, hit);
    return cudaGetLastError();
}

// Two tile shapes, the autotuner's choice per batch: tiles of kTileTracks =
// 384 tracks with 12 producer + 4 consumer warps, or tiles of 256 with 8 + 4.
cudaError_t launch_dist_batched(const BatchView& bv, const Basket& b, double* step, int32_t* hit, int blocks_per_sm,
                                int tile_tracks, cudaStream_t s, int num_sms) {
    static_assert(sizeof(TileHdr) % 16 == 0 && sizeof(VolView) % 16 == 0, "16-byte copies");
    const int code = (bv.segs ? 1 : 0) + (bv.vox ? 2 : 0);
    if (tile_tracks == kLatProd) {
        switch (code) {
            case 0: return launch_batched<false, false, kLatProd, kLatCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
            case 1: return launch_batched<true, false, kLatProd, kLatCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
            case 2: return launch_batched<false, true, kLatProd, kLatCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
            default: return launch_batched<true, true, kLatProd, kLatCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
        }
    }
    switch (code) {
        case 0: return launch_batched<false, false, kProd, kCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
        case 1: return launch_batched<true, false, kProd, kCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
        case 2: return launch_batched<false, true, kProd, kCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
        default: return launch_batched<true, true, kProd, kCons>(bv, b, step, hit, blocks_per_sm, s, num_sms);
    }
}

// A small basket in a volume of many daughters takes the split kernel
// (split_basket()); otherwise a basket of at most two tiles of 256 tracks per
// resident block (two blocks per SM) takes the latency configuration, larger
// ones the throughput configuration (toy detector, one call: 65536 tracks
// 43.8 us instead of 59.1 us, 131072 tracks 66.5 us instead of 78.5 us; from
// 196608 tracks on the two are equal, and at 2^20 the throughput
// configuration is 13 % faster).
cudaError_t launch_dist_refine_stats(const VolView& v, const Basket& b, double* step, int32_t* hit,
                                     double* bpoint, int32_t* nref, cudaStream_t s, int num_sms) {
    if (split_basket(v, b.n, num_sms)) return launch_dist_refine_split(v, b, step, hit, bpoint, nref, s);
    if (b.n <= int64_t(4) * num_sms * kLatProd)
        return launch_dist_refine_latency(v, b, step, hit, bpoint, nref, s, num_sms);
    return launch_refine_cfg<kProd, kCons>(v, b, step, hit, bpoint, nref, s, num_sms);
}

// Small baskets take the warp-per-track FP64 kernel (the same answers: both
// modes return the plain FP64 bits); the filter pays off only when its
// threads are many.
cudaError_t launch_dist_refine(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                               cudaStream_t s, int num_sms) {
    if (small_basket(v, b.n, num_sms)) return launch_dist_warp(v, b, step, hit, bpoint, s, num_sms);
    return launch_dist_refine_stats(v, b, step, hit, bpoint, nullptr, s, num_sms);
}

}  // namespace geonav
