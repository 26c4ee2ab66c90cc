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
#include "shapes32.cuh"
#include "shapes64.cuh"
#include "stage.cuh"

namespace geonav {

constexpr int kCand = 4;

struct Cands {
    float L[kCand];
    int j[kCand];
    int n;
    float dropped;   // smallest bound evicted from the list
};

__device__ __forceinline__ void cand_insert(Cands& c, float L, int j) {
    float Lc = L;
    int jc = j;
#pragma unroll
    for (int k = 0; k < kCand; ++k) {
        if (k < c.n) {
            if (Lc < c.L[k]) {
                const float tL = c.L[k];
                const int tj = c.j[k];
                c.L[k] = Lc;
                c.j[k] = jc;
                Lc = tL;
                jc = tj;
            }
        } else if (k == c.n) {
            c.L[k] = Lc;
            c.j[k] = jc;
            Lc = f_inf();
        }
    }
    if (c.n < kCand) ++c.n;
    else c.dropped = fminf(c.dropped, Lc);
}

// lower the FP32 parameter t by its rounding allowance
__device__ __forceinline__ float lower_bound(float t, float delta, float inv_dn) {
    return t - (16.f * kEps32f * fabsf(t) + delta * inv_dn);
}

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
        int h;
        int nev = 0;
        if (!valid_track(px, py, pz, qx, qy, qz)) {
            store_result(i, b.n, d_nan(), -2, px, py, pz, qx, qy, qz, step, hit, bpoint);
            if (nref) nref[i] = 0;
            continue;
        }
        const float p32[3] = {float(px), float(py), float(pz)};
        const float d32[3] = {float(qx), float(qy), float(qz)};
        const float dd = fmaf(d32[0], d32[0], fmaf(d32[1], d32[1], d32[2] * d32[2]));
        if (!(dd > 1e-30f && dd < 1e30f)) {
            // direction magnitude outside the range the FP32 bounds assume
            const double p[3] = {px, py, pz};
            if (contains64(v.m64, p)) nav_all64(v.m64, tab64, v.nd, px, py, pz, qx, qy, qz, best, h);
            else { best = 0.0; h = -2; }
            store_result(i, b.n, best, h, px, py, pz, qx, qy, qz, step, hit, bpoint);
            if (nref) nref[i] = 1000;
            continue;
        }
        const float inv_dd = __frcp_rn(dd);
        const float inv_dn = rsqrtf(dd) * (1.f + 4.f * kEps32f);
        // mother: the shrunk copy gives "surely inside" and a lower bound of
        // the exit, the grown copy an upper bound
        bool in_shrunk;
        const float e_lo = exit32(v.m32, p32, d32, in_shrunk);
        bool inside = in_shrunk;
        if (!in_shrunk) {
            const double p[3] = {px, py, pz};
            inside = contains64(v.m64, p);
        }
        if (!inside) {
            store_result(i, b.n, 0.0, -2, px, py, pz, qx, qy, qz, step, hit, bpoint);
            if (nref) nref[i] = 0;
            continue;
        }
        const float Lm = in_shrunk ? fmaxf(lower_bound(e_lo, v.m32.delta, inv_dn), 0.f) : 0.f;
        bool dummy;
        const float e_hi = exit32(v.m32u, p32, d32, dummy);
        const float Um = e_hi + 16.f * kEps32f * e_hi + v.m32u.delta * inv_dn;

        // ---------------- pass 1: FP32 lower bounds of every daughter -------
        Cands c;
        c.n = 0;
        c.dropped = f_inf();
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
            c.L[k] = f_inf();
            c.j[k] = 0;
        }
        for (int j = 0; j < v.nd; ++j) {
            const ShapeRec32& r = tab32[j];
            const float w0 = p32[0] - r.t[0], w1 = p32[1] - r.t[1], w2 = p32[2] - r.t[2];
            const float s0 = -fmaf(w0, d32[0], fmaf(w1, d32[1], w2 * d32[2])) * inv_dd;
            const float q0 = fmaf(s0, d32[0], w0), q1 = fmaf(s0, d32[1], w1), q2 = fmaf(s0, d32[2], w2);
            const float perp2 = fmaf(q0, q0, fmaf(q1, q1, q2 * q2));
            if (perp2 > r.brad * r.brad) continue;
            const float half = r.brad * inv_dn;
            if (s0 + half < 0.f || s0 - half > Um) continue;
            float x[3], u[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                x[k] = fmaf(r.R[6 + k], q2, fmaf(r.R[3 + k], q1, r.R[k] * q0));
                u[k] = fmaf(r.R[6 + k], d32[2], fmaf(r.R[3 + k], d32[1], r.R[k] * d32[0]));
            }
            const float tp = enter32(r, x, u, -s0);
            if (!(tp < f_inf())) continue;
            const float L = lower_bound(s0 + tp, r.delta, inv_dn);
            if (L > Um) continue;
            cand_insert(c, L, j);
        }

        // ---------------- pass 2: FP64 refinement in ascending bound order --
        const double p[3] = {px, py, pz}, q[3] = {qx, qy, qz};
        best = d_inf();
        h = -1;
        bool mdone = false;
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
            if (k < c.n) {
                const double L = double(c.L[k]);
                if (!mdone && double(Lm) <= L) {
                    const double sm = dist_in64(v.m64, p, q);
                    ++nev;
                    mdone = true;
                    if (sm <= best) {
                        best = sm;
                        h = -1;
                    }
                }
                if (L <= best) {
                    const int j = c.j[k];
                    const ShapeRec64& r = tab64[j];
                    double x[3], u[3];
                    to_local64(r, px, py, pz, qx, qy, qz, x, u);
                    const double s = dist_out64(r, x, u);
                    ++nev;
                    if (s < best || (s == best && h >= 0 && j < h)) {
                        best = s;
                        h = j;
                    }
                }
            }
        }
        if (!mdone && double(Lm) <= best) {
            const double sm = dist_in64(v.m64, p, q);
            ++nev;
            if (sm <= best) {
                best = sm;
                h = -1;
            }
        }
        if (double(c.dropped) <= best) {
            nav_all64(v.m64, tab64, v.nd, px, py, pz, qx, qy, qz, best, h);
            nev += 1000;   // marks a fallback in the statistics
        }
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
