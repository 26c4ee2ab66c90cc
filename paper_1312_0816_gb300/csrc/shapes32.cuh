// shapes32.cuh -- FP32 bounding routines of the filter stage.
//
// The filter never decides an answer; it only produces, per (track, solid),
// a number that is provably not larger than the FP64 distance (a LOWER bound
// L), or for the mother an upper bound U of its exit distance.  The argument:
//
//  * The FP32 copy of every solid is inflated by delta (mm); see make_rec32()
//    and inflation() in geo_abi.cu.  delta exceeds the worst-case distance
//    between the FP32 ray (rounded inputs, rounded transform) and the exact
//    ray over the whole mother, so wherever the exact ray is inside the true
//    solid the FP32 ray is inside the inflated one.  Hence the entry of the
//    FP32 ray into the inflated solid is <= the true entry.
//  * delta also exceeds, in radius terms, the rounding of each quadric's
//    discriminant (8 eps32 brad^2 / r in the frame shifted to the closest
//    approach), so a ray that truly meets a quadric never sees a negative
//    discriminant for its inflated copy, and the computed entering root of the
//    inflated quadric is <= the true root.
//  * Acceptance tests of candidate crossings (is the z-plane crossing inside
//    the annulus, is the cylinder crossing inside the slab) are LENIENT by
//    delta: extra candidates can only lower the minimum, so leniency is safe.
//  * The result is finally lowered by 16 eps32 |t| + delta/|d|, which covers
//    the relative rounding of the crossing parameters.
// Upper bounds of the mother's exit use the inflated mother the same way;
// lower bounds of the exit use the mother shrunk by delta.
#pragma once
#include <cmath>
#include "geo_internal.h"

namespace geonav {

constexpr float kEps32f = 5.9604645e-08f;

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// Approximate division and square root (a few ulp): the filter's margins
// (16 eps32 |t| relative, plus the inflation delta) absorb them.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }

// FP64 -> FP32 by truncating the significand (integer operations only, so the
// FP64 pipe stays free).  Relative error below 2^-23, which the inflation
// covers.  Magnitudes outside the normal FP32 range take the ordinary
// conversion.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
    const unsigned hi = unsigned(__double2hiint(x)), lo = unsigned(__double2loint(x));
    const int e = int((hi >> 20) & 0x7ffu) - 1023;
    if (e < -126 || e > 127) return float(x);
    const unsigned bits = (hi & 0x80000000u) | (unsigned(e + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(bits);
}

// An FP32 value >= x for x >= 0 (x itself when exactly representable or one
// ulp above the truncation), integer operations only.
__device__ __forceinline__ float f64_to_f32_up(double x) {
    // x >= 0 here; compared on the bit pattern (3.0e38 as a double)
    if (!(__double_as_longlong(x) < 0x47EC363CBF21F28ALL)) return f_inf();
    const float t = f64_to_f32_trunc(x);
    return __uint_as_float(__float_as_uint(t) + 1u);
}

// ---------------------------------------------------------------- box ------
// inf{ t >= tmin : x + t u in box(h) }, lenient by tol at the start point.
__device__ __forceinline__ float box_enter32(const float* h, const float* x, const float* u, float tmin,
                                             float tol) {
    float tn = tmin, tf = f_inf();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (u[k] == 0.f) {
            if (fabsf(x[k]) > h[k] + tol) return f_inf();
        } else {
            const float inv = __fdividef(1.f, u[k]);
            const float a = (-h[k] - x[k]) * inv, b = (h[k] - x[k]) * inv;
            tn = fmaxf(tn, fminf(a, b));
            tf = fminf(tf, fmaxf(a, b));
        }
    }
    return tn <= tf ? tn : f_inf();
}

// exit of the box for a start point inside it (first t >= 0 leaving the slabs)
__device__ __forceinline__ float box_exit32(const float* h, const float* x, const float* u) {
    float tf = f_inf();
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (u[k] != 0.f) tf = fminf(tf, fdiv(copysignf(h[k], u[k]) - x[k], u[k]));
    return fmaxf(tf, 0.f);
}

// ------------------------------------------------------------- quadrics -----
// The routines below select operands instead of branching, so that the lanes
// of a warp bounding the same solid run one code path whatever their tracks.
//
// D with a tolerance: a discriminant within rounding of zero counts as a
// tangent (D = 0), which only adds candidates.
__device__ __forceinline__ bool disc32(float A, float B, float C, float& sq) {
    const float D = fmaf(B, B, -A * C);
    sq = fsqrt(fmaxf(D, 0.f));
    return D >= 0.f || D > -16.f * kEps32f * (B * B + fabsf(A * C));
}

// Roots are parameters relative to the (shifted) origin of the frame and may
// be negative: the caller compares them with its own tmin.
// falling root (F decreases through 0): (-B - sq)/A in stable form
__device__ __forceinline__ float root_falling32(float A, float B, float C) {
    float sq;
    const bool real = disc32(A, B, C, sq);
    const bool bneg = B < 0.f;
    const float q = fdiv(bneg ? C : -B - sq, bneg ? sq - B : A);
    return real && (bneg || A != 0.f) ? q : f_inf();
}

// rising root (F increases through 0): (-B + sq)/A in stable form
__device__ __forceinline__ float root_rising32(float A, float B, float C) {
    float sq;
    const bool real = disc32(A, B, C, sq);
    const bool bpos = B > 0.f;
    const float q = fdiv(bpos ? C : sq - B, bpos ? -B - sq : A);
    return real && (bpos || A != 0.f) ? q : f_inf();
}

// ---------------------------------------------------------------- tube -----
// e: [0] rmin'^2 (0 if no hole), [1] rmax'^2, [2] dz', [3] hole flag, and the
// acceptance limits, lenient by tol = delta (geo_abi.cu make_rec32):
// [4] (rmax' + delta)^2 rounded up, [5] (rmin' - delta)^2 rounded down (0
// without a hole), [6] dz' + delta rounded up.
__device__ __forceinline__ float tube_enter32(const float* e, const float* x, const float* u, float tmin) {
    const float dz = e[2], zl = e[6], ro2 = e[4], ri2 = e[5];
    // start point
    const float sx = fmaf(tmin, u[0], x[0]), sy = fmaf(tmin, u[1], x[1]), sz = fmaf(tmin, u[2], x[2]);
    const float sr2 = fmaf(sx, sx, sy * sy);
    if (fabsf(sz) <= zl && sr2 <= ro2 && sr2 >= ri2) return tmin;
    // the z-plane the start lies beyond, when the track approaches it
    const float tz = fdiv(copysignf(dz, sz) - x[2], u[2]);
    const float xh = fmaf(tz, u[0], x[0]), yh = fmaf(tz, u[1], x[1]);
    const float r2 = fmaf(xh, xh, yh * yh);
    float best = fabsf(sz) > dz && sz * u[2] < 0.f && r2 <= ro2 && r2 >= ri2 ? fmaxf(tz, tmin) : f_inf();
    const float A = fmaf(u[0], u[0], u[1] * u[1]);
    const float B = fmaf(x[0], u[0], x[1] * u[1]);
    const float rho2 = fmaf(x[0], x[0], x[1] * x[1]);
    {
        const float s = root_falling32(A, B, rho2 - e[1]);
        best = s >= tmin && s < best && fabsf(fmaf(s, u[2], x[2])) <= zl ? s : best;
    }
    if (e[3] != 0.f) {   // uniform across the warp: every lane bounds the same solid
        const float s = root_rising32(A, B, rho2 - e[0]);
        best = s >= tmin && s < best && fabsf(fmaf(s, u[2], x[2])) <= zl ? s : best;
    }
    return best;
}

// ---------------------------------------------------------------- cone -----
// e: [0] dz', [1] a_out', [2] b_out, [3] a_in', [4] b_in, [5] hole,
//    [6] rmin1'^2 [7] rmax1'^2 [8] rmin2'^2 [9] rmax2'^2 (at z = -dz', +dz'),
// and the end annuli's acceptance limits, lenient by tol = delta:
//    [10] (rmax1' + delta)^2 [11] (rmax2' + delta)^2 rounded up,
//    [12] (rmin1' - delta)^2 [13] (rmin2' - delta)^2 rounded down (0 where
//    there is no hole), [14] dz' + delta rounded up.
__device__ __forceinline__ float cone_enter32(const float* e, const float* x, const float* u, float tmin,
                                              float tol) {
    const float dz = e[0];
    const float zl = e[14];
    const bool hole = e[5] != 0.f;
    const float sx = fmaf(tmin, u[0], x[0]), sy = fmaf(tmin, u[1], x[1]), sz = fmaf(tmin, u[2], x[2]);
    const float sr2 = fmaf(sx, sx, sy * sy);
    {
        const float ro = fmaf(e[2], sz, e[1]) + tol, ri = fmaf(e[4], sz, e[3]) - tol;
        if (fabsf(sz) <= zl && sr2 <= ro * ro && (!hole || ri <= 0.f || sr2 >= ri * ri)) return tmin;
    }
    // the end plane the start lies beyond, when the track approaches it
    const float tz = fdiv(copysignf(dz, sz) - x[2], u[2]);
    const float xh = fmaf(tz, u[0], x[0]), yh = fmaf(tz, u[1], x[1]);
    const float r2 = fmaf(xh, xh, yh * yh);
    const bool up = sz > 0.f;
    const float hi2 = up ? e[11] : e[10], lo2 = up ? e[13] : e[12];
    float best = fabsf(sz) > dz && sz * u[2] < 0.f && r2 <= hi2 && r2 >= lo2 ? fmaxf(tz, tmin) : f_inf();
    const float A0 = fmaf(u[0], u[0], u[1] * u[1]);
    const float B0 = fmaf(x[0], u[0], x[1] * u[1]);
    const float rho2 = fmaf(x[0], x[0], x[1] * x[1]);
    {
        const float r0 = fmaf(e[2], x[2], e[1]), rs = e[2] * u[2];
        const float s = root_falling32(fmaf(-rs, rs, A0), fmaf(-r0, rs, B0), fmaf(-r0, r0, rho2));
        best = s >= tmin && s < best && fabsf(fmaf(s, u[2], x[2])) <= zl ? s : best;
    }
    if (hole) {   // uniform across the warp
        const float r0 = fmaf(e[4], x[2], e[3]), rs = e[4] * u[2];
        const float s = root_rising32(fmaf(-rs, rs, A0), fmaf(-r0, rs, B0), fmaf(-r0, r0, rho2));
        best = s >= tmin && s < best && fabsf(fmaf(s, u[2], x[2])) <= zl ? s : best;
    }
    return best;
}

// Lower bound on the entering distance in the shifted frame: x is the track's
// point of closest approach to the solid's origin, tmin = -s0 the parameter of
// the real start point.  Returns the entering parameter relative to x.
__device__ __forceinline__ float enter32(const ShapeRec32& r, const float* x, const float* u, float tmin) {
    const float tol = r.delta;
    if (r.kind == KBOX) return box_enter32(r.e, x, u, tmin, tol);
    if (r.kind == KTUBE) return tube_enter32(r.e, x, u, tmin);
    return cone_enter32(r.e, x, u, tmin, tol);
}

// ------------------------------------------------------- mother exit -------
// Exit distance of a start point x inside the (shrunk or grown) mother, in the
// mother's own frame (no shift).  Also reports whether x is inside it.
__device__ __forceinline__ float exit32(const ShapeRec32& r, const float* x, const float* u, bool& inside) {
    const float* e = r.e;
    if (r.kind == KBOX) {
        inside = fabsf(x[0]) <= e[0] && fabsf(x[1]) <= e[1] && fabsf(x[2]) <= e[2];
        return box_exit32(e, x, u);
    }
    const float rho2 = fmaf(x[0], x[0], x[1] * x[1]);
    const float A0 = fmaf(u[0], u[0], u[1] * u[1]);
    const float B0 = fmaf(x[0], u[0], x[1] * u[1]);
    float t, s;
    if (r.kind == KTUBE) {
        inside = fabsf(x[2]) <= e[2] && rho2 <= e[1] && (e[3] == 0.f || rho2 >= e[0]);
        t = u[2] != 0.f ? fdiv(copysignf(e[2], u[2]) - x[2], u[2]) : f_inf();
        s = root_rising32(A0, B0, rho2 - e[1]);
        if (s >= 0.f) t = fminf(t, s);
        if (e[3] != 0.f) {
            s = root_falling32(A0, B0, rho2 - e[0]);
            if (s >= 0.f) t = fminf(t, s);
        }
        return fmaxf(t, 0.f);
    }
    const float ro0 = fmaf(e[2], x[2], e[1]);
    const float ri0 = fmaf(e[4], x[2], e[3]);
    // inside test on the same rounded constants as the roots below, so that a
    // point counted inside never sees a root behind it
    const float co = fmaf(-ro0, ro0, rho2), ci = fmaf(-ri0, ri0, rho2);
    inside = fabsf(x[2]) <= e[0] && co <= 0.f && (e[5] == 0.f || ci >= 0.f);
    t = u[2] != 0.f ? fdiv(copysignf(e[0], u[2]) - x[2], u[2]) : f_inf();
    {
        const float rs = e[2] * u[2];
        s = root_rising32(fmaf(-rs, rs, A0), fmaf(-ro0, rs, B0), co);
        if (s >= 0.f) t = fminf(t, s);
    }
    if (e[5] != 0.f) {
        const float rs = e[4] * u[2];
        s = root_falling32(fmaf(-rs, rs, A0), fmaf(-ri0, rs, B0), ci);
        if (s >= 0.f) t = fminf(t, s);
    }
    return fmaxf(t, 0.f);
}

// ------------------------------------------------------- point queries ---
// Containment of a point on an FP32 copy.  On an inflated copy (daughters,
// the mother's m32u) a point that is exactly inside the true solid is inside
// the copy; on the deflated mother (m32) a point inside the copy is exactly
// inside the true mother, with a margin larger than the FP64 rounding.  The
// argument is the one above with the ray replaced by a point: delta exceeds
// the distance between the FP32 local point and the exact one plus the
// rounding of the radius arithmetic.
__device__ __forceinline__ bool contains32(const ShapeRec32& r, const float* x) {
    const float* e = r.e;
    if (r.kind == KBOX) return fabsf(x[0]) <= e[0] && fabsf(x[1]) <= e[1] && fabsf(x[2]) <= e[2];
    const float rho2 = fmaf(x[0], x[0], x[1] * x[1]);
    if (r.kind == KTUBE) return fabsf(x[2]) <= e[2] && rho2 <= e[1] && (e[3] == 0.f || rho2 >= e[0]);
    if (!(fabsf(x[2]) <= e[0])) return false;
    const float ro = fmaf(e[2], x[2], e[1]), ri = fmaf(e[4], x[2], e[3]);
    return fmaf(-ro, ro, rho2) <= 0.f && (e[5] == 0.f || fmaf(-ri, ri, rho2) >= 0.f);
}

// Relative margin of the safety bounds below: covers the rounding of the
// FP32 distance arithmetic relative to the distance itself (the absolute
// part, proportional to the solid's size, is inside delta).
constexpr float kSafMargin = 3.8146973e-06f;   // 2^-18

// Lower bound of the outside-safety of an INFLATED copy (distance from x to
// the solid).  Box and tube: the exact Euclidean distance to the copy (the
// tube in the meridian half-plane, to the rectangle [rmin, rmax] x [-dz, dz]).
// Cone: the largest distance to a supporting half-plane of its trapezoid
// (z-slab, outer and inner radius lines), which cannot exceed the distance to
// a convex section.  The copy contains the true solid grown by delta, so the
// distance to it is at most the true distance minus delta, and delta covers
// the FP32 position and radius errors; the result is lowered by kSafMargin.
__device__ __forceinline__ float safety_out_lb32(const ShapeRec32& r, const float* x) {
    const float* e = r.e;
    float s;
    if (r.kind == KBOX) {
        const float a = fmaxf(fabsf(x[0]) - e[0], 0.f), b = fmaxf(fabsf(x[1]) - e[1], 0.f),
                    c = fmaxf(fabsf(x[2]) - e[2], 0.f);
        s = fsqrt(fmaf(a, a, fmaf(b, b, c * c)));
    } else {
        const float rho = fsqrt(fmaf(x[0], x[0], x[1] * x[1]));
        const float az = fabsf(x[2]);
        if (r.kind == KTUBE) {
            float dr = rho - fsqrt(e[1]);
            if (e[3] != 0.f) dr = fmaxf(dr, fsqrt(e[0]) - rho);
            dr = fmaxf(dr, 0.f);
            const float dz = fmaxf(az - e[2], 0.f);
            s = fsqrt(fmaf(dr, dr, dz * dz));
        } else {
            s = az - e[0];
            s = fmaxf(s, (rho - fmaf(e[2], x[2], e[1])) * rsqrtf(fmaf(e[2], e[2], 1.f)));
            if (e[5] != 0.f) s = fmaxf(s, (fmaf(e[4], x[2], e[3]) - rho) * rsqrtf(fmaf(e[4], e[4], 1.f)));
            s = fmaxf(s, 0.f);
        }
    }
    return s * (1.f - kSafMargin);
}

// Lower bound of the inside-safety on the DEFLATED mother copy: for a point
// inside a solid whose meridian section is convex, the distance to the
// boundary is the smallest distance to a supporting line of the section
// (box: faces; tube: rmax, rmin, z planes; cone: z planes and radius lines).
// The copy lies delta inside the true solid, so its inside-distance is at most
// the true one minus delta; negative (the point is outside the copy) gives 0.
__device__ __forceinline__ float safety_in_lb32(const ShapeRec32& r, const float* x) {
    const float* e = r.e;
    float s;
    if (r.kind == KBOX) {
        s = fminf(e[0] - fabsf(x[0]), fminf(e[1] - fabsf(x[1]), e[2] - fabsf(x[2])));
    } else {
        const float rho = fsqrt(fmaf(x[0], x[0], x[1] * x[1]));
        const float az = fabsf(x[2]);
        if (r.kind == KTUBE) {
            s = fminf(fsqrt(e[1]) - rho, e[2] - az);
            if (e[3] != 0.f) s = fminf(s, rho - fsqrt(e[0]));
        } else {
            s = e[0] - az;
            s = fminf(s, (fmaf(e[2], x[2], e[1]) - rho) * rsqrtf(fmaf(e[2], e[2], 1.f)));
            if (e[5] != 0.f) s = fminf(s, (rho - fmaf(e[4], x[2], e[3])) * rsqrtf(fmaf(e[4], e[4], 1.f)));
        }
    }
    return fmaxf(s, 0.f) * (1.f - kSafMargin);
}

}  // namespace geonav
