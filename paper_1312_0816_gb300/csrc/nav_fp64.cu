// nav_fp64.cu -- the plain FP64 vector navigator of Fig. 1b on the GPU (and,
// for small baskets, its warp-per-track form with a shuffle (step, index)
// minimum), and the navigator-level Contains and Safety of Sec. 3.1.
//
// One thread per track (grid-stride over the basket).  The basket is read as
// coalesced FP64 structure-of-arrays.  The volume's FP64 daughter table is
// staged once per block into shared memory with the bulk-copy engine and read
// warp-uniformly (every lane of a warp visits daughter j together, so each
// record field is a broadcast).  Per daughter: a bounding-sphere test against
// the current best step, the master->local transform, DistFromOutside, and a
// running (step, index) minimum with strict '<' (mother first, then lowest
// index win ties).
#include <cuda_runtime.h>
#include "geo_internal.h"
#include "nav_common.cuh"
#include "shapes64.cuh"
#include "stage.cuh"
#include "launch.cuh"

namespace geonav {

template <bool SMEM>
__global__ void __launch_bounds__(256) k_dist_fp64(VolView v, Basket b, double* __restrict__ step,
                                                   int32_t* __restrict__ hit, double* __restrict__ bpoint) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const ShapeRec64* tab = v.d64;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d64, uint32_t(v.nd) * sizeof(ShapeRec64), &bar, v.status)) return;
        tab = reinterpret_cast<const ShapeRec64*>(smem_raw);
    }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const double px = b.x[i], py = b.y[i], pz = b.z[i];
        const double qx = b.dx[i], qy = b.dy[i], qz = b.dz[i];
        double best;
        int h;
        const double p[3] = {px, py, pz};
        if (!valid_track(px, py, pz, qx, qy, qz)) {
            best = d_nan();
            h = -2;
        } else if (!contains64(v.m64, p)) {
            best = 0.0;
            h = -2;
        } else if (v.voxelized) {
            nav_vox64(v, tab, px, py, pz, qx, qy, qz, best, h);
        } else {
            nav_all64(v.m64, tab, v.nd, px, py, pz, qx, qy, qz, best, h);
        }
        store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
    }
}

// Small baskets: one warp per track.  The lanes take the daughters j = lane,
// lane + 32, ... (bounding-sphere cull against the mother's step), each keeps
// its (step, index) minimum with strict '<', and the warp reduces the pairs
// with shuffles (smaller step, then smaller index); the mother (index -1)
// wins ties.  That is the thread-per-track loop's answer bit for bit: it
// takes the daughters in index order with strict '<' after the mother, and
// a daughter it culls against its running best could not have won (the cull
// is conservative), so the lanes' weaker culls only evaluate more.  Every
// lane computes the track's mother step and containment (warp-uniform: the
// FP64 pipe charges a warp instruction whatever the active lanes).  The
// table is read through L1: a few tracks would not repay its staging.
template <bool SEGS>
__global__ void __launch_bounds__(256) k_dist_warp(VolView v, Basket b, double* __restrict__ step,
                                                   int32_t* __restrict__ hit, double* __restrict__ bpoint) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < b.n; i += nwarps) {
        const double px = b.x[i], py = b.y[i], pz = b.z[i];
        const double qx = b.dx[i], qy = b.dy[i], qz = b.dz[i];
        const double p[3] = {px, py, pz}, q[3] = {qx, qy, qz};
        double best;
        int h;
        if (!valid_track(px, py, pz, qx, qy, qz)) {
            best = d_nan();
            h = -2;
        } else if (!contains64<SEGS>(v.m64, p)) {
            best = 0.0;
            h = -2;
        } else {
            const double sm = dist_in64<false, SEGS>(v.m64, p, q);
            const double dd = qx * qx + qy * qy + qz * qz;
            const double dn = sqrt(dd);
            double lb = d_inf();
            int lh = 0x7fffffff;
            for (int j = lane; j < v.nd; j += 32) {
                const ShapeRec64& r = v.d64[j];
                const double w0 = r.t[0] - px, w1 = r.t[1] - py, w2 = r.t[2] - pz;
                const double proj = w0 * qx + w1 * qy + w2 * qz;
                const double rb = r.brad * dn;
                if (proj + rb < 0.0) continue;
                if (proj - rb >= sm * dd) continue;
                const double ww = w0 * w0 + w1 * w1 + w2 * w2;
                if (ww * dd - proj * proj > rb * rb) continue;
                double x[3], u[3];
                to_local64(r, px, py, pz, qx, qy, qz, x, u);
                const double sj = dist_out64<false, SEGS>(r, x, u);
                if (LT(sj, lb)) {
                    lb = sj;
                    lh = j;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, lb, off);
                const int oh = __shfl_xor_sync(0xffffffffu, lh, off);
                if (LT(ob, lb) || (BITS(ob) == BITS(lb) && oh < lh)) {
                    lb = ob;
                    lh = oh;
                }
            }
            best = sm;
            h = -1;
            if (LT(lb, sm)) {
                best = lb;
                h = lh;
            }
        }
        if (lane == 0) store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
    }
}

template <bool SMEM>
__global__ void __launch_bounds__(256) k_contains(VolView v, Basket b, int32_t* __restrict__ where) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const ShapeRec64* tab = v.d64;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d64, uint32_t(v.nd) * sizeof(ShapeRec64), &bar, v.status)) return;
        tab = reinterpret_cast<const ShapeRec64*>(smem_raw);
    }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const double p[3] = {b.x[i], b.y[i], b.z[i]};
        int w = -2;
        if (contains64(v.m64, p)) {
            w = -1;
            for (int j = 0; j < v.nd; ++j) {
                const ShapeRec64& r = tab[j];
                const double w0 = p[0] - r.t[0], w1 = p[1] - r.t[1], w2 = p[2] - r.t[2];
                if (w0 * w0 + w1 * w1 + w2 * w2 > r.brad * r.brad) continue;
                double x[3], u[3];
                to_local64(r, p[0], p[1], p[2], 0.0, 0.0, 0.0, x, u);
                if (contains64(r, x)) {
                    w = j;
                    break;
                }
            }
        }
        where[i] = w;
    }
}

template <bool SMEM>
__global__ void __launch_bounds__(256) k_safety_fp64(VolView v, Basket b, double* __restrict__ saf) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const ShapeRec64* tab = v.d64;
    if (SMEM) {
        if (!stage_table(smem_raw, v.d64, uint32_t(v.nd) * sizeof(ShapeRec64), &bar, v.status)) return;
        tab = reinterpret_cast<const ShapeRec64*>(smem_raw);
    }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const double p[3] = {b.x[i], b.y[i], b.z[i]};
        double s = 0.0;
        if (contains64(v.m64, p)) {
            s = safety64(v.m64, p, true);
            for (int j = 0; j < v.nd && s > 0.0; ++j) {
                const ShapeRec64& r = tab[j];
                const double w0 = p[0] - r.t[0], w1 = p[1] - r.t[1], w2 = p[2] - r.t[2];
                const double c = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
                if (c - r.brad >= s) continue;   // the whole daughter is farther than s
                double x[3], u[3];
                to_local64(r, p[0], p[1], p[2], 0.0, 0.0, 0.0, x, u);
                s = fmin(s, safety64(r, x, false));
            }
        }
        saf[i] = s;
    }
}

// ------------------------------------------------------------ launchers ---

#define GEO_LAUNCH(KER, ...)                                                                 \
    do {                                                                                     \
        const int smem = v.smem64 ? v.nd * int(sizeof(ShapeRec64)) : 0;                      \
        if (v.smem64) {                                                                      \
            cudaError_t e = prep(KER<true>, smem);                                           \
            if (e != cudaSuccess) return e;                                                  \
            KER<true><<<blocks_for(KER<true>, b.n, smem, num_sms), 256, smem, s>>>(__VA_ARGS__); \
        } else {                                                                             \
            KER<false><<<blocks_for(KER<false>, b.n, 0, num_sms), 256, 0, s>>>(__VA_ARGS__);   \
        }                                                                                    \
        return cudaGetLastError();                                                           \
    } while (0)

// One warp per track when the basket is small (at most 8 tracks per SM: the
// latency of a track's serial daughter loop would set the time) and the
// daughters fit one pass of the lanes (at most 32).  With more daughters, or
// more tracks, the warp's FP64 instructions -- charged in full whatever the
// lanes that take part -- outweigh the latency it hides (the 40-daughter toy
// detector: 53 us per call instead of 36 us at 16..1024 tracks).
bool small_basket(const VolView& v, int64_t n, int num_sms) {
    return !v.voxelized && v.nd <= 32 && n <= int64_t(8) * num_sms;
}

cudaError_t launch_dist_warp(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                             cudaStream_t s, int num_sms) {
    if (v.segs) {
        k_dist_warp<true><<<blocks_for(k_dist_warp<true>, b.n * 32, 0, num_sms), 256, 0, s>>>(v, b, step, hit,
                                                                                             bpoint);
    } else {
        k_dist_warp<false><<<blocks_for(k_dist_warp<false>, b.n * 32, 0, num_sms), 256, 0, s>>>(v, b, step, hit,
                                                                                               bpoint);
    }
    return cudaGetLastError();
}

cudaError_t launch_dist_fp64(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                             cudaStream_t s, int num_sms) {
    if (small_basket(v, b.n, num_sms)) return launch_dist_warp(v, b, step, hit, bpoint, s, num_sms);
    GEO_LAUNCH(k_dist_fp64, v, b, step, hit, bpoint);
}

cudaError_t launch_contains(const VolView& v, const Basket& b, int32_t* where, int mode, cudaStream_t s,
                            int num_sms) {
    if (mode == GEO_FP32_REFINE) return launch_contains_filter(v, b, where, s, num_sms);
    GEO_LAUNCH(k_contains, v, b, where);
}

cudaError_t launch_safety(const VolView& v, const Basket& b, double* saf, int mode, cudaStream_t s,
                          int num_sms) {
    if (mode == GEO_FP32_REFINE) return launch_safety_filter(v, b, saf, s, num_sms);
    if (mode == GEO_SAFETY_ESTIMATE) return launch_safety_estimate(v, b, saf, s, num_sms);
    GEO_LAUNCH(k_safety_fp64, v, b, saf);
}

}  // namespace geonav
