// nav_fp64.cu -- the plain FP64 vector navigator of Fig. 1b on the GPU, and
// the navigator-level Contains and Safety of Sec. 3.1.
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

cudaError_t launch_dist_fp64(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                             cudaStream_t s, int num_sms) {
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
