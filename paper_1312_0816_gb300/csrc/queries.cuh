// queries.cuh -- navigator-level Contains and Safety of Sec. 3.1 with the FP32
// filter: one conservative FP32 pass over the daughters, FP64 only where the
// FP32 bounds cannot decide.  The answers are the same bits as those of the
// plain FP64 kernels (nav_fp64.cu):
//
//  * Contains.  A daughter is skipped only when the FP32 point lies outside
//    its bounding sphere or its inflated FP32 copy; the exact point is then
//    outside the true solid by more than the FP64 rounding, so the FP64 test
//    would be false as well.  The others are tested in FP64 in index order,
//    so the lowest containing index wins as in the plain kernel.  The mother
//    is decided in FP32 unless the point lies between its deflated and
//    inflated copies.
//  * Safety.  The FP32 pass gives a lower bound L_k of the FP64 safety of
//    every candidate (k = -1 the mother, inside-safety; k >= 0 a daughter,
//    outside-safety) and keeps the two smallest.  The smallest is evaluated in
//    FP64 (value S).  If the second bound exceeds S by more than the FP64
//    rounding, no other candidate can be below S, and S is the minimum.
//    Otherwise a second FP32 pass evaluates in FP64 every candidate whose
//    bound does not exceed the running minimum.  Either way the result is the
//    FP64 minimum over all candidates, which is what the plain kernel returns
//    (its bounding-sphere culls only skip daughters whose FP64 safety exceeds
//    its running minimum).
//
// Per-point routines; the kernels are in queries.cu.
#pragma once
#include "geo_internal.h"
#include "nav_common.cuh"
#include "shapes32.cuh"
#include "shapes64.cuh"

namespace geonav {

__device__ __forceinline__ void point32(const Basket& b, int64_t i, double* p, float* p32) {
    p[0] = b.x[i];
    p[1] = b.y[i];
    p[2] = b.z[i];
    p32[0] = f64_to_f32_trunc(p[0]);
    p32[1] = f64_to_f32_trunc(p[1]);
    p32[2] = f64_to_f32_trunc(p[2]);
}

// Mother containment: FP32 on the deflated copy (surely inside), on the
// inflated copy (surely outside), FP64 in between.  Non-finite points fail
// both FP32 tests and come out outside, as in FP64.
// SEGS = false: the volume holds no polycone (its code is left out).
template <bool SEGS = true>
__device__ __forceinline__ bool mother_contains(const VolView& v, const double* p, const float* p32) {
    if (contains32(v.m32, p32)) return true;
    if (!contains32(v.m32u, p32)) return false;
    return contains64<SEGS>(v.m64, p);
}

// Offset from the daughter's centre, its squared length and the local point.
__device__ __forceinline__ float offset32(const ShapeRec32& r, const float* p32, float* w) {
    w[0] = p32[0] - r.t[0];
    w[1] = p32[1] - r.t[1];
    w[2] = p32[2] - r.t[2];
    return fmaf(w[0], w[0], fmaf(w[1], w[1], w[2] * w[2]));
}

__device__ __forceinline__ void local32(const ShapeRec32& r, const float* w, float* x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = fmaf(r.R[6 + k], w[2], fmaf(r.R[3 + k], w[1], r.R[k] * w[0]));
}

// The first daughter from index `from` on whose inflated FP32 copy holds the
// point (-1: none).  A point inside a daughter is inside its copy, so no
// daughter skipped here can contain it.
__device__ __forceinline__ int contains_next(const VolView& v, const ShapeRec32* __restrict__ t32, const float* p32,
                                             int from) {
    for (int j = from; j < v.nd; ++j) {
        const ShapeRec32& r = t32[j];
        float o[3], x[3];
        const float c2 = offset32(r, p32, o);
        if (c2 > r.brad * r.brad * (1.f + kSafMargin)) continue;   // outside the bounding sphere
        local32(r, o, x);
        if (contains32(r, x)) return j;
    }
    return -1;
}

// The FP64 decision for daughter j, with the plain kernel's routines.
template <bool SEGS = true>
__device__ __forceinline__ bool contains_daughter64(const VolView& v, int j, const double* p) {
    const ShapeRec64& r64 = v.d64[j];
    double xl[3];
    point_to_local64(r64, p[0], p[1], p[2], xl);
    return contains64<SEGS>(r64, xl);
}

// After the FP64 test of candidate j failed: the remaining candidates in
// index order (rare: the inflated copies of daughters seldom overlap).
template <bool SEGS = true>
__device__ __forceinline__ int contains_rest(const VolView& v, const ShapeRec32* __restrict__ t32, const double* p,
                                             const float* p32, int j) {
    for (j = contains_next(v, t32, p32, j + 1); j >= 0; j = contains_next(v, t32, p32, j + 1))
        if (contains_daughter64<SEGS>(v, j, p)) return j;
    return -1;
}

// Contains of one point: -2, -1 or the lowest daughter index.
template <bool SEGS = true>
__device__ __forceinline__ int contains_filter(const VolView& v, const ShapeRec32* __restrict__ t32,
                                               const double* p, const float* p32) {
    if (!mother_contains<SEGS>(v, p, p32)) return -2;
    const int j = contains_next(v, t32, p32, 0);
    if (j < 0) return -1;
    if (contains_daughter64<SEGS>(v, j, p)) return j;
    return contains_rest<SEGS>(v, t32, p, p32, j);
}

// FP64 safety of candidate k (-1: mother inside-safety, else daughter k's
// outside-safety), with the plain kernel's routines.
template <bool SEGS = true>
__device__ __forceinline__ double safety_of(const VolView& v, int k, const double* p) {
    if (k < 0) return safety64<SEGS>(v.m64, p, true);
    const ShapeRec64& r = v.d64[k];
    double x[3];
    point_to_local64(r, p[0], p[1], p[2], x);
    return safety64<SEGS>(r, x, false);
}

// FP32 threshold above which a lower bound proves an FP64 safety larger than
// s: s rounded up to FP32, a relative 2^-20 (so the FP32 sum keeps the
// margin), and tau above the FP64 rounding of any safety in the mother.
__device__ __forceinline__ float above(double s, float tau) {
    return fmaf(f64_to_f32_up(s), 1.f + 9.536743e-07f, tau);
}

// Lower bound of the distance to daughter r from its bounding sphere (the
// inflated radius covers the FP32 position errors; the square root is
// lowered by the relative margin).
__device__ __forceinline__ float sphere_lb32(const ShapeRec32& r, float c2) {
    return fsqrt(c2) * (1.f - kSafMargin) - r.brad;
}

// Bounding-sphere cull of daughter r against a bound L: true when the whole
// sphere (inflated, so conservative) is farther than L.
__device__ __forceinline__ bool beyond(const ShapeRec32& r, float c2, float L) {
    const float lim = fmaf(L, 1.f + kSafMargin, r.brad);
    return c2 > lim * lim * (1.f + kSafMargin);
}

// FP32 pass of the safety of one point: the two smallest lower bounds (L1 of
// candidate j1, L2) and the mother's bound Lm.  Returns false when the point
// is outside the mother (safety 0, no FP64 work).
struct SafetyState {
    float Lm, L2;
    int j1;
};

template <bool SEGS = true>
__device__ __forceinline__ bool safety_pass1(const VolView& v, const ShapeRec32* __restrict__ t32, const double* p,
                                             const float* p32, SafetyState& st) {
    if (!mother_contains<SEGS>(v, p, p32)) return false;
    const float Lm = safety_in_lb32(v.m32, p32);
    float L1 = Lm, L2 = f_inf();
    int j1 = -1;
    for (int j = 0; j < v.nd; ++j) {
        const ShapeRec32& r = t32[j];
        float o[3], x[3];
        const float c2 = offset32(r, p32, o);
        if (beyond(r, c2, L2)) continue;   // cannot be among the two smallest
        local32(r, o, x);
        const float l = safety_out_lb32(r, x);
        if (l < L1) {
            L2 = L1;
            L1 = l;
            j1 = j;
        } else if (l < L2) {
            L2 = l;
        }
    }
    st.Lm = Lm;
    st.L2 = L2;
    st.j1 = j1;
    return true;
}

// Given s = the FP64 safety of candidate j1: done if the second bound
// exceeds s; otherwise every other candidate whose bound does not exceed the
// running minimum is evaluated in FP64.  *nev counts the evaluations.
template <bool SEGS = true>
__device__ __forceinline__ double safety_finish(const VolView& v, const ShapeRec32* __restrict__ t32,
                                                const double* p, const float* p32, const SafetyState& st,
                                                double s, float tau, int* nev) {
    int ne = 1;
    float th = above(s, tau);
    if (!(st.L2 > th)) {
        // another candidate may still be below s: visit them all
        if (st.j1 >= 0 && !(st.Lm > th)) {
            s = fmin(s, safety_of<SEGS>(v, -1, p));
            ++ne;
            th = above(s, tau);
        }
        for (int j = 0; j < v.nd; ++j) {
            if (j == st.j1) continue;
            const ShapeRec32& r = t32[j];
            float o[3], x[3];
            const float c2 = offset32(r, p32, o);
            if (beyond(r, c2, th)) continue;
            local32(r, o, x);
            if (safety_out_lb32(r, x) > th) continue;
            s = fmin(s, safety_of<SEGS>(v, j, p));
            ++ne;
            th = above(s, tau);
        }
    }
    *nev = ne;
    return s;
}

// Safety of one point (the two phases back to back).
template <bool SEGS = true>
__device__ __forceinline__ double safety_filter(const VolView& v, const ShapeRec32* __restrict__ t32,
                                                const double* p, const float* p32, float tau, int* nev) {
    SafetyState st;
    if (!safety_pass1<SEGS>(v, t32, p, p32, st)) {
        *nev = 0;
        return 0.0;
    }
    return safety_finish<SEGS>(v, t32, p, p32, st, safety_of<SEGS>(v, st.j1, p), tau, nev);
}

// 2^-36 of the mother's extent: far above the FP64 rounding of any safety
// (positions and daughters lie within that extent)
__device__ __forceinline__ float safety_tau(const VolView& v) { return v.m32u.brad * 1.4551915e-11f; }

}  // namespace geonav
