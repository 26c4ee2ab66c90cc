// nav_refine.cuh -- per-track step of the FP32-filter + FP64-refine
// navigator (see nav_refine.cu for the scheme).  Shared by every kernel that
// navigates with the filter.
#pragma once
#include "geo_internal.h"
#include "nav_common.cuh"
#include "shapes32.cuh"
#include "shapes64.cuh"

namespace geonav {

// Candidates kept per track: the kCand smallest FP32 bounds, and the least
// bound evicted.  Two suffice: on every test scene, random and adversarial
// rays, no track falls back to the full FP64 loop, and the list's registers
// and insertion work are what the FP32 pass can least afford (toy detector:
// 0.283 ms with two, 0.298 with three, 0.312 with four, 0.408 with five).
constexpr int kCand = 2;

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

// FP32 lower bound of one daughter's DistFromOutside (bounding-sphere test,
// transform in the frame shifted to the closest approach, inflated solid),
// inserted into the candidate list when it can beat the mother's exit.
__device__ __forceinline__ void bound_daughter(const ShapeRec32& r, int j, const float* p32, const float* d32,
                                               float inv_dd, float inv_dn, float Um, Cands& c) {
    const float4 tb = *reinterpret_cast<const float4*>(r.t);   // t and brad^2
    const float w0 = p32[0] - tb.x, w1 = p32[1] - tb.y, w2 = p32[2] - tb.z;
    const float s0 = -fmaf(w0, d32[0], fmaf(w1, d32[1], w2 * d32[2])) * inv_dd;
    const float q0 = fmaf(s0, d32[0], w0), q1 = fmaf(s0, d32[1], w1), q2 = fmaf(s0, d32[2], w2);
    const float perp2 = fmaf(q0, q0, fmaf(q1, q1, q2 * q2));
    if (perp2 > tb.w) return;
    const float half = r.brad * inv_dn;
    if (s0 + half < 0.f || s0 - half > Um) return;
    float x[3], u[3];
    if (r.flags & kRec32Identity) {   // warp-uniform: every lane visits solid j together
        x[0] = q0; x[1] = q1; x[2] = q2;
        u[0] = d32[0]; u[1] = d32[1]; u[2] = d32[2];
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x[k] = fmaf(r.R[6 + k], q2, fmaf(r.R[3 + k], q1, r.R[k] * q0));
            u[k] = fmaf(r.R[6 + k], d32[2], fmaf(r.R[3 + k], d32[1], r.R[k] * d32[0]));
        }
    }
    const float tp = enter32(r, x, u, -s0);
    if (!(tp < f_inf())) return;
    const float L = lower_bound(s0 + tp, r.delta, inv_dn);
    if (L > Um) return;
    cand_insert(c, L, j);
}

// Walk of the uniform grid (3D-DDA) along the FP32 ray from its start to the
// parameter tend, calling visit(j) for every daughter listed in every cell
// entered.  At most gx + gy + gz + 3 cells.
template <class F>
__device__ __forceinline__ void vox_walk32(const VolView& v, const float* p, const float* d, float tend,
                                           F&& visit) {
    // per axis: cell index, step direction, next boundary parameter, increment
    int i0, i1, i2, s0, s1, s2;
    float m0, m1, m2, e0, e1, e2;
    auto setup = [&](int k, int& ii, int& st, float& tm, float& te) {
        const float lo = float(v.lo[k]), cell = float(v.cell[k]);
        const int g = v.grid[k];
        ii = int(floorf((p[k] - lo) * float(v.inv_cell[k])));
        ii = ii < 0 ? 0 : (ii >= g ? g - 1 : ii);
        if (d[k] > 0.f) {
            st = 1;
            tm = (fmaf(float(ii + 1), cell, lo) - p[k]) / d[k];
            te = cell / d[k];
        } else if (d[k] < 0.f) {
            st = -1;
            tm = (fmaf(float(ii), cell, lo) - p[k]) / d[k];
            te = -cell / d[k];
        } else {
            st = 0;
            tm = f_inf();
            te = f_inf();
        }
    };
    setup(0, i0, s0, m0, e0);
    setup(1, i1, s1, m1, e1);
    setup(2, i2, s2, m2, e2);
    const int g0 = v.grid[0], g1 = v.grid[1], g2 = v.grid[2];
    const int maxit = g0 + g1 + g2 + 3;
    for (int it = 0; it < maxit; ++it) {
        const int c = (i0 * g1 + i1) * g2 + i2;
        const int q1 = v.vox_off[c + 1];
        for (int q = v.vox_off[c]; q < q1; ++q) visit(v.vox_ids[q]);
        if (m0 <= m1 && m0 <= m2) {
            if (!(m0 <= tend)) break;
            i0 += s0;
            if (i0 < 0 || i0 >= g0) break;
            m0 += e0;
        } else if (m1 <= m2) {
            if (!(m1 <= tend)) break;
            i1 += s1;
            if (i1 < 0 || i1 >= g1) break;
            m1 += e1;
        } else {
            if (!(m2 <= tend)) break;
            i2 += s2;
            if (i2 < 0 || i2 >= g2) break;
            m2 += e2;
        }
    }
}

// The filter's cold FP64 paths (a direction magnitude outside the FP32
// range, a start between the mother's shrunk copy and the mother, a bound
// evicted from the list that could still win), out of line: inlined, their
// FP64 code raised the register pressure of the hot FP32 pass (spill stores
// 400 -> 148 bytes; toy detector 0.2268 -> 0.2237 ms, the batched launch
// 1.128 -> 1.106 ms).
template <bool SEGS>
static __device__ __noinline__ void nav_all64_cold(const ShapeRec64& m, const ShapeRec64* __restrict__ tab, int nd,
                                                   double px, double py, double pz, double qx, double qy, double qz,
                                                   double& best, int& h) {
    nav_all64<SEGS>(m, tab, nd, px, py, pz, qx, qy, qz, best, h);
}
template <bool SEGS>
static __device__ __noinline__ bool contains64_cold(const ShapeRec64& m, double px, double py, double pz) {
    const double p[3] = {px, py, pz};
    return contains64<SEGS>(m, p);
}

// State of one track between the FP32 pass and the FP64 refinement.
struct RefineState {
    Cands c;
    float Lm;       // lower bound of the mother's exit
    int status;     // 0: refine, 1: result already final (invalid / outside / fallback)
};

// FP32 pass: bounds of the mother and of every daughter.  When status == 1
// on return, best/h already hold the final answer.  TRAVERSAL: 0 = every
// daughter, 1 = the uniform grid, 2 = chosen per volume at run time.
// (TRAVERSAL 0 only) j_first, j_step: bound daughters j_first, j_first +
// j_step, ... alone (a share of the volume's daughters).
template <int TRAVERSAL, bool SEGS = true>
__device__ __forceinline__ void refine_pass1(const VolView& v, const ShapeRec32* __restrict__ tab32,
                                             const ShapeRec64* __restrict__ tab64, double px, double py,
                                             double pz, double qx, double qy, double qz, RefineState& st,
                                             double& best, int& h, int& nev, int j_first = 0, int j_step = 1) {
    nev = 0;
    st.status = 1;
    st.c.n = 0;
    st.c.dropped = f_inf();
#pragma unroll
    for (int k = 0; k < kCand; ++k) {
        st.c.L[k] = f_inf();
        st.c.j[k] = 0;
    }
    st.Lm = 0.f;
    if (!valid_track(px, py, pz, qx, qy, qz)) {
        best = d_nan();
        h = -2;
        return;
    }
    const float p32[3] = {f64_to_f32_trunc(px), f64_to_f32_trunc(py), f64_to_f32_trunc(pz)};
    const float d32[3] = {f64_to_f32_trunc(qx), f64_to_f32_trunc(qy), f64_to_f32_trunc(qz)};
    const float dd = fmaf(d32[0], d32[0], fmaf(d32[1], d32[1], d32[2] * d32[2]));
    if (!(dd > 1e-30f && dd < 1e30f)) {
        // direction magnitude outside the range the FP32 bounds assume
        const double p[3] = {px, py, pz};
        if (contains64<SEGS>(v.m64, p)) nav_all64_cold<SEGS>(v.m64, tab64, v.nd, px, py, pz, qx, qy, qz, best, h);
        else { best = 0.0; h = -2; }
        nev = 1000;
        return;
    }
    const float inv_dd = __frcp_rn(dd);
    const float inv_dn = rsqrtf(dd) * (1.f + 4.f * kEps32f);
    // mother: the shrunk copy gives "surely inside" and a lower bound of the
    // exit, the grown copy an upper bound
    bool in_shrunk;
    const float e_lo = exit32(v.m32, p32, d32, in_shrunk);
    bool inside = in_shrunk;
    if (!in_shrunk) {
        inside = contains64_cold<SEGS>(v.m64, px, py, pz);
    }
    if (!inside) {
        best = 0.0;
        h = -2;
        return;
    }
    st.Lm = in_shrunk ? fmaxf(lower_bound(e_lo, v.m32.delta, inv_dn), 0.f) : 0.f;
    bool dummy;
    const float e_hi = exit32(v.m32u, p32, d32, dummy);
    const float Um = e_hi + 16.f * kEps32f * e_hi + v.m32u.delta * inv_dn;
    const bool grid = TRAVERSAL == 1 || (TRAVERSAL == 2 && v.voxelized);
    if (!grid) {
        for (int j = j_first; j < v.nd; j += j_step) bound_daughter(tab32[j], j, p32, d32, inv_dd, inv_dn, Um, st.c);
    } else {
        // only daughters listed in the cells the track crosses before the
        // mother's exit (upper bound Um); a daughter met again is skipped
        // (4-entry mailbox, then the candidate list)
        int mb0 = -1, mb1 = -1, mb2 = -1, mb3 = -1;
        vox_walk32(v, p32, d32, Um, [&](int j) {
            if (j == mb0 || j == mb1 || j == mb2 || j == mb3) return;
            mb3 = mb2; mb2 = mb1; mb1 = mb0; mb0 = j;
#pragma unroll
            for (int k = 0; k < kCand; ++k)
                if (k < st.c.n && st.c.j[k] == j) return;
            bound_daughter(tab32[j], j, p32, d32, inv_dd, inv_dn, Um, st.c);
        });
    }
    st.status = 0;
}

// The first solid to refine: the mother (-1) when its bound comes first or
// there is no candidate, else candidate 0.
__device__ __forceinline__ int first_task(const RefineState& st) {
    return (st.c.n == 0 || st.Lm <= st.c.L[0]) ? -1 : st.c.j[0];
}

// FP64 evaluation of one solid for one track (the mother's DistFromInside or
// a daughter's transform + DistFromOutside).
template <bool SEGS = true>
__device__ __forceinline__ double eval64(const VolView& v, const ShapeRec64* __restrict__ tab64, int j, double px,
                                         double py, double pz, double qx, double qy, double qz) {
    if (j < 0) {
        const double p[3] = {px, py, pz}, q[3] = {qx, qy, qz};
        return dist_in64<false, SEGS>(v.m64, p, q);
    }
    const ShapeRec64& r = tab64[j];
    double x[3], u[3];
    to_local64(r, px, py, pz, qx, qy, qz, x, u);
    return dist_out64<false, SEGS>(r, x, u);
}

// The answer of refine_rest() when no further FP64 evaluation can change it
// (nearly every track): the first task's value s_first is finite and every
// other bound -- the remaining candidates, the mother's when it was not the
// first task, the least evicted one -- lies above its FP32 upper bound.  A
// solid's FP64 value is at least its bound, so none of them can win or tie.
// Returns false when refine_rest() has to run.
__device__ __forceinline__ bool refine_fast(const RefineState& st, double s_first, double& best, int& h) {
    const bool mother_first = first_task(st) < 0;
    if (!LT(s_first, d_inf())) return false;
    const float up = f64_to_f32_up(s_first);
    const int k0 = mother_first ? 0 : 1;
#pragma unroll
    for (int k = 0; k < kCand; ++k)
        if (k >= k0 && k < st.c.n && st.c.L[k] <= up) return false;
    if (!mother_first && st.Lm <= up) return false;
    if (st.c.dropped <= up) return false;
    best = s_first;
    h = mother_first ? -1 : st.c.j[0];
    return true;
}

// FP64 refinement in ascending bound order, given the value s_first of the
// first task (first_task()).  Ties resolve as in Fig. 1a: mother, then the
// lowest index.  The bounds are compared in FP32 against best_up >= best, so
// at least every solid that could tie or win is refined (a solid refined in
// excess cannot change the answer).
template <bool SEGS = true>
static __device__ __noinline__ void refine_rest(const VolView& v, const ShapeRec64* __restrict__ tab64,
                                         const RefineState& st, double s_first, double px, double py, double pz,
                                         double qx, double qy, double qz, double& best, int& h, int& nev) {
    best = d_inf();
    h = -1;
    nev = 1;
    bool mdone;
    int k0;
    if (first_task(st) < 0) {
        mdone = true;
        best = s_first;   // the mother always beats +inf
        k0 = 0;
    } else {
        mdone = false;
        if (LT(s_first, best)) {
            best = s_first;
            h = st.c.j[0];
        }
        k0 = 1;
    }
    float best_up = f64_to_f32_up(best);
#pragma unroll
    for (int k = 0; k < kCand; ++k) {
        if (k >= k0 && k < st.c.n) {
            const float L = st.c.L[k];
            if (!mdone && st.Lm <= L) {
                const double sm = eval64<SEGS>(v, tab64, -1, px, py, pz, qx, qy, qz);
                ++nev;
                mdone = true;
                if (LE(sm, best)) {
                    best = sm;
                    h = -1;
                    best_up = f64_to_f32_up(best);
                }
            }
            if (L <= best_up) {
                const int j = st.c.j[k];
                const double s = eval64<SEGS>(v, tab64, j, px, py, pz, qx, qy, qz);
                ++nev;
                // same order as the sequential loop: bit-pattern order of
                // non-negative steps, ties to the mother, then the lowest index
                if (LT(s, best) || (BITS(s) == BITS(best) && h >= 0 && j < h)) {
                    best = s;
                    h = j;
                    best_up = f64_to_f32_up(best);
                }
            }
        }
    }
    if (!mdone && st.Lm <= best_up) {
        const double sm = eval64<SEGS>(v, tab64, -1, px, py, pz, qx, qy, qz);
        ++nev;
        if (LE(sm, best)) {
            best = sm;
            h = -1;
            best_up = f64_to_f32_up(best);
        }
    }
    if (st.c.dropped <= best_up) {
        nav_all64_cold<SEGS>(v.m64, tab64, v.nd, px, py, pz, qx, qy, qz, best, h);
        nev += 1000;   // marks a fallback in the statistics
    }
}

// One track, all in this thread (used where no block-level compaction is
// available).  Same answers as nav_all64 with the mother prologue.
__device__ __forceinline__ void refine_track(const VolView& v, const ShapeRec32* __restrict__ tab32,
                                             const ShapeRec64* __restrict__ tab64, double px, double py,
                                             double pz, double qx, double qy, double qz, double& best, int& h,
                                             int& nev) {
    RefineState st;
    refine_pass1<2>(v, tab32, tab64, px, py, pz, qx, qy, qz, st, best, h, nev);
    if (st.status) return;
    const double s1 = eval64(v, tab64, first_task(st), px, py, pz, qx, qy, qz);
    refine_rest(v, tab64, st, s1, px, py, pz, qx, qy, qz, best, h, nev);
}

}  // namespace geonav
