// shapes64.cuh -- FP64 device routines for the shape queries of Sec. 3.1
// (distance to enter, distance to leave, inside check, safety) of Box, Tube,
// Cone, the tube segment and the polycone, plus the master->local transform
// of Sec. 3.1.
//
// Formulation: "candidate surfaces".  DistFromOutside of a closed solid is the
// smallest s >= 0 at which the ray crosses INTO the solid through one of its
// bounding surfaces (z-planes, outer and inner quadric), each crossing being
// accepted only if the crossing point satisfies the remaining constraints;
// DistFromInside is the first s >= 0 at which any constraint is violated.
// Quadric roots are taken in cancellation-free form (the product of the roots
// of A s^2 + 2 B s + C is C/A).
//
// Every FP64 operation is an explicitly rounded intrinsic, so the values do
// not depend on how the compiler contracts expressions in the kernel that
// inlines them: the plain FP64 kernel and the refine stage of the FP32-filter
// kernel produce bit-identical results.
#pragma once
#include <cmath>
#include "geo_internal.h"

namespace geonav {

__device__ __forceinline__ double d_inf() { return __longlong_as_double(0x7ff0000000000000LL); }
__device__ __forceinline__ double d_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

__device__ __forceinline__ double MUL(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ADD(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double SUB(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double FMA(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double DIV(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double SQRT(double a) { return __dsqrt_rn(a); }
// a*b + c*d with one rounding for c*d and a fused final step
__device__ __forceinline__ double DOT2(double a, double b, double c, double d) { return FMA(a, b, MUL(c, d)); }

// Comparisons on the bit patterns (integer ALU instead of the FP64 pipe).
// For non-negative doubles (and +inf) the IEEE order is the integer order of
// the bits; a NaN compares as larger than +inf, so "<=" and "<" against a
// finite or infinite bound are false for it, as in floating point.
__device__ __forceinline__ long long BITS(double a) { return __double_as_longlong(a); }
constexpr long long kAbsMask = 0x7fffffffffffffffLL;
__device__ __forceinline__ bool LE(double a, double b) { return BITS(a) <= BITS(b); }    // a, b >= 0
__device__ __forceinline__ bool LT(double a, double b) { return BITS(a) < BITS(b); }     // a, b >= 0
__device__ __forceinline__ bool ABS_LE(double x, double h) { return (BITS(x) & kAbsMask) <= BITS(h); }  // h >= 0
__device__ __forceinline__ bool ABS_GT(double x, double h) { return (BITS(x) & kAbsMask) > BITS(h); }   // h >= 0
__device__ __forceinline__ bool IS_ZERO(double a) { return (BITS(a) & kAbsMask) == 0; }
__device__ __forceinline__ bool IS_NEG(double a) { return BITS(a) < 0 && !IS_ZERO(a); }     // a < 0
__device__ __forceinline__ bool IS_POS(double a) { return BITS(a) > 0; }                    // a > 0
__device__ __forceinline__ bool NONNEG(double a) { return BITS(a) >= 0 || IS_ZERO(a); }     // a >= 0
// a * b < 0 without the product
__device__ __forceinline__ bool OPPOSITE(double a, double b) {
    return ((BITS(a) ^ BITS(b)) < 0) && !IS_ZERO(a) && !IS_ZERO(b);
}
// min / max of two values >= 0
__device__ __forceinline__ double MINP(double a, double b) { return LT(b, a) ? b : a; }
__device__ __forceinline__ double MAXP(double a, double b) { return LT(a, b) ? b : a; }

// x = R^T (p - t), u = R^T d (an identity rotation: x = p - t, u = d)
__device__ __forceinline__ void to_local64(const ShapeRec64& r, double px, double py, double pz,
                                           double qx, double qy, double qz, double* x, double* u) {
    const double w0 = SUB(px, r.t[0]), w1 = SUB(py, r.t[1]), w2 = SUB(pz, r.t[2]);
    if (r.flags & kRec64Identity) {
        x[0] = w0; x[1] = w1; x[2] = w2;
        u[0] = qx; u[1] = qy; u[2] = qz;
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        x[k] = FMA(r.R[6 + k], w2, FMA(r.R[3 + k], w1, MUL(r.R[k], w0)));
        u[k] = FMA(r.R[6 + k], qz, FMA(r.R[3 + k], qy, MUL(r.R[k], qx)));
    }
}

// x = R^T (p - t) alone (the same operations as to_local64, so the same bits)
__device__ __forceinline__ void point_to_local64(const ShapeRec64& r, double px, double py, double pz, double* x) {
    const double w0 = SUB(px, r.t[0]), w1 = SUB(py, r.t[1]), w2 = SUB(pz, r.t[2]);
    if (r.flags & kRec64Identity) {
        x[0] = w0; x[1] = w1; x[2] = w2;
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = FMA(r.R[6 + k], w2, FMA(r.R[3 + k], w1, MUL(r.R[k], w0)));
}

// F(s) = A s^2 + 2 B s + C.  Root where F falls through zero (F' = -2 sqrt(D)),
// s = (-B - sqrt(D)) / A; +inf when there is none.  May be negative.
// Both cancellation-free forms are selected operand-wise so that every lane
// of a warp runs the same single square root and division; a lane whose
// result is discarded takes the square root and quotient of 1, so that no
// lane of the warp diverges into the handling of a special operand (zero).
__device__ __forceinline__ double root_falling(double A, double B, double C) {
    const double D = FMA(B, B, -MUL(A, C));
    const bool real = NONNEG(D);
    const double sq = SQRT(real ? D : 1.0);
    const bool bneg = IS_NEG(B);
    const double num = bneg ? C : SUB(-B, sq);
    const double den = bneg ? SUB(sq, B) : A;
    const bool ok = real && (bneg || IS_NEG(A));
    const double s = DIV(ok ? num : 1.0, ok ? den : 1.0);
    return ok ? s : d_inf();
}

// Root where F rises through zero (F' = +2 sqrt(D)): s = (-B + sqrt(D)) / A.
__device__ __forceinline__ double root_rising(double A, double B, double C) {
    const double D = FMA(B, B, -MUL(A, C));
    const bool real = NONNEG(D);
    const double sq = SQRT(real ? D : 1.0);
    const bool bpos = IS_POS(B);
    const double num = bpos ? C : SUB(sq, B);
    const double den = bpos ? SUB(-B, sq) : A;
    const bool ok = real && (bpos || IS_POS(A));
    const double s = DIV(ok ? num : 1.0, ok ? den : 1.0);
    return ok ? s : d_inf();
}

// The same two roots whatever their sign (the parameter origin need not be
// the track's start): +inf only when there is none (D < 0, or a linear F that
// does not fall / rise through zero).
__device__ __forceinline__ double root_falling_any(double A, double B, double C) {
    const double D = FMA(B, B, -MUL(A, C));
    const bool real = NONNEG(D);
    const double sq = SQRT(real ? D : 1.0);
    const bool bneg = IS_NEG(B);
    const double num = bneg ? C : SUB(-B, sq);
    const double den = bneg ? SUB(sq, B) : A;
    const bool ok = real && (bneg || !IS_ZERO(A));
    const double s = DIV(ok ? num : 1.0, ok ? den : 1.0);
    return ok ? s : d_inf();
}

__device__ __forceinline__ double root_rising_any(double A, double B, double C) {
    const double D = FMA(B, B, -MUL(A, C));
    const bool real = NONNEG(D);
    const double sq = SQRT(real ? D : 1.0);
    const bool bpos = IS_POS(B);
    const double num = bpos ? C : SUB(sq, B);
    const double den = bpos ? SUB(-B, sq) : A;
    const bool ok = real && (bpos || !IS_ZERO(A));
    const double s = DIV(ok ? num : 1.0, ok ? den : 1.0);
    return ok ? s : d_inf();
}

__device__ __forceinline__ double rho2_of(const double* x) { return DOT2(x[0], x[0], x[1], x[1]); }

// ---------------------------------------------------- tube segment wedge ---
// (x, y) in the wedge of a tube segment (d as in geo_internal.h)
__device__ __forceinline__ bool wedge_has64(const double* d, double x, double y) {
    if (d[10] != 0.0) return true;
    const bool a = NONNEG(DOT2(d[5], x, d[6], y)), b = NONNEG(DOT2(d[7], x, d[8], y));
    return d[9] != 0.0 ? (a && b) : (a || b);
}

// Crossing of the cone rho = R(z) = Rc + b (z - zc) with the track, the
// quadric rho^2 - R(z)^2 formed about the track's point closest to (0, 0, zc)
// of the axis.  With zc at the cone's apex (Rc = 0) this resolves a track
// passing close to the apex: there the two roots nearly coincide, and the
// quadric about the start point, whose terms are as large as the start's
// distance squared, cannot separate them, while about the closest point its
// terms are as small as the miss distance.  RISING: the root where rho^2 -
// R^2 rises through zero, else the falling one.  Returns the parameter (+inf:
// none) and the crossing's x, y and height above zc.  inv_uu = 1 / |u|^2.
template <bool RISING>
__device__ __forceinline__ double cone_root_about(double zc, double Rc, double b, const double* x, const double* u,
                                                  double A0, double inv_uu, double& xh, double& yh, double& zh) {
    const double xz = SUB(x[2], zc);
    const double sc = MUL(-FMA(xz, u[2], DOT2(x[0], u[0], x[1], u[1])), inv_uu);
    const double c0 = FMA(sc, u[0], x[0]), c1 = FMA(sc, u[1], x[1]), c2 = FMA(sc, u[2], xz);
    const double Rq = FMA(b, c2, Rc), rs = MUL(b, u[2]);
    const double A = FMA(-rs, rs, A0), B = FMA(-Rq, rs, DOT2(c0, u[0], c1, u[1]));
    const double C = FMA(-Rq, Rq, DOT2(c0, c0, c1, c1));
    const double sg = RISING ? root_rising_any(A, B, C) : root_falling_any(A, B, C);
    xh = FMA(sg, u[0], c0);
    yh = FMA(sg, u[1], c1);
    zh = FMA(sg, u[2], c2);
    return ADD(sc, sg);
}

// Crossing of the cone of polycone section [zk, zk1], radius line through
// (r0 at zk) and (r1 at zk1) with slope b, formed about the apex when the
// radius vanishes at one of the section's planes, else about (0, 0, zk)
// (cone_root_about).  Sets the crossing's x, y and whether its height lies
// in [zk, zk1].
template <bool RISING>
__device__ __forceinline__ double pcon_sec_root(double r0, double r1, double b, double zk, double zk1, const double* x,
                                                const double* u, double A0, double inv_uu, double& xh, double& yh,
                                                bool& in_z) {
    const bool top = IS_ZERO(r1) && !IS_ZERO(r0);
    double zh;
    const double s = cone_root_about<RISING>(top ? zk1 : zk, top ? r1 : r0, b, x, u, A0, inv_uu, xh, yh, zh);
    in_z = top ? (zh >= SUB(zk, zk1) && zh <= 0.0) : (zh >= 0.0 && zh <= SUB(zk1, zk));
    return s;
}

// A crossing of a phi face's plane lies on the face when it is on the face's
// side of the axis.  Within rounding of the axis (r2 <= tau2, the squared
// rounding scale of the crossing point) that side is decided by rounding, and
// the track instead enters there, where the two faces meet, when the solid
// holds the axis (no inner radius there) and the track moves into the wedge.
__device__ __forceinline__ bool on_phi_face(const double* d, double ex, double ey, double xh, double yh, double r2,
                                            bool axis_in, double tau2, const double* u) {
    if (LE(r2, tau2)) return axis_in && wedge_has64(d, u[0], u[1]);
    return NONNEG(DOT2(ex, xh, ey, yh));
}

// ------------------------------------------------------------- polycone ---
// The plane table T (layout in geo_internal.h) is read with plain loads: it
// lives in global memory, or in a kernel's parameters for one-shape queries.
__device__ __forceinline__ const double* pcon_table(const double* d) {
    return reinterpret_cast<const double*>(__double_as_longlong(d[0]));
}

// the last section k (0 <= k <= n-2) with z[k] <= v
__device__ __forceinline__ int pcon_section(const double* z, int n, double v) {
    int lo = 0, hi = n - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (z[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// radius line of a section at height v: r0 + b (v - z0)
__device__ __forceinline__ double rline(double r0, double b, double z0, double v) { return FMA(b, SUB(v, z0), r0); }

// (rho^2 = r2, z = v) in the cross-section: in a section whose z-range holds
// v (on a plane: either of the two sharing it), between its radius lines
__device__ __forceinline__ bool pcon_in2(const double* T, int n, double r2, double v) {
    const double *z = T, *rn = T + n, *rx = T + 2 * n, *bi = T + 3 * n, *bo = bi + (n - 1);
    if (!(v >= z[0] && v <= z[n - 1])) return false;
    const int k0 = pcon_section(z, n, v);
    for (int k = k0; k >= 0 && k >= k0 - 1; --k) {
        if (!(v >= z[k] && v <= z[k + 1])) continue;
        const double ro = rline(rx[k], bo[k], z[k], v), ri = rline(rn[k], bi[k], z[k], v);
        if (LE(r2, MUL(ro, ro)) && (!(rn[k] > 0.0 || rn[k + 1] > 0.0) || LE(MUL(ri, ri), r2))) return true;
    }
    return false;
}

// out of line, so that the hot kernels do not carry the polycone's code
static __device__ __noinline__ bool pcon_contains64(const double* d, const double* T, double x0, double x1, double x2) {
    return pcon_in2(T, int(d[1]), DOT2(x0, x0, x1, x1), x2) && wedge_has64(d, x0, x1);
}

// ------------------------------------------------------------- contains ---
// SEGS = false (here and below): the caller's volumes hold no polycone, and
// its out-of-line code (whose registers a kernel that calls it must provide)
// is left out.
template <bool SEGS = true>
__device__ __forceinline__ bool contains64(const ShapeRec64& r, const double* x) {
    const double* d = r.d;
    if (r.kind == KBOX) return ABS_LE(x[0], d[0]) && ABS_LE(x[1], d[1]) && ABS_LE(x[2], d[2]);
    const double rho2 = rho2_of(x);
    if (SEGS && r.kind == KPCON) return pcon_contains64(d, pcon_table(d), x[0], x[1], x[2]);
    if (r.kind == KTUBE) return ABS_LE(x[2], d[2]) && LE(rho2, d[4]) && LE(d[3], rho2);
    if (r.kind == KTUBS)
        return ABS_LE(x[2], d[2]) && LE(rho2, d[4]) && LE(d[3], rho2) && wedge_has64(d, x[0], x[1]);
    if (!ABS_LE(x[2], d[0])) return false;
    const double ro = FMA(d[2], x[2], d[1]);
    const double ri = FMA(d[4], x[2], d[3]);
    return LE(rho2, MUL(ro, ro)) && (d[11] == 0.0 || LE(MUL(ri, ri), rho2));
}

// ------------------------------------------------------ DistFromOutside ---
// Slab method with one division: the entry parameter of axis k is
// N_k / a_k with a_k = |u_k| > 0 and N_k = -h_k - sign(u_k) x_k, its exit
// F_k / a_k with F_k = h_k - sign(u_k) x_k; the largest entry and smallest
// exit are chosen by comparing cross products, and only the entry is divided.
// Surface tags (FACE output of the routines below, used by the adjoint):
// box 0..5 = -x,+x,-y,+y,-z,+z; tube and cone 4/5 = -z/+z planes, 6 outer,
// 7 inner quadric; -1 = none (start point inside, or no crossing).
template <bool FACE = false>
__device__ __forceinline__ double box_out64(const double* h, const double* x, const double* u, int* face = nullptr) {
    if (FACE) *face = -1;
    if (ABS_LE(x[0], h[0]) && ABS_LE(x[1], h[1]) && ABS_LE(x[2], h[2])) return 0.0;
    double Nn = -1.0, An = 0.0;   // entry numerator / denominator so far (-inf)
    double Nf = 1.0, Af = 0.0;    // exit numerator / denominator so far (+inf)
    int fn = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (IS_ZERO(u[k])) {
            if (ABS_GT(x[k], h[k])) return d_inf();
            continue;
        }
        const double a = fabs(u[k]);
        const double xs = IS_POS(u[k]) ? x[k] : -x[k];   // sign(u_k) x_k
        const double N = SUB(-h[k], xs), F = SUB(h[k], xs);
        // N/a > Nn/An  <=>  N An > Nn a   (a, An >= 0; An == 0 encodes -inf)
        if (An == 0.0 || MUL(N, An) > MUL(Nn, a)) {
            Nn = N;
            An = a;
            if (FACE) fn = 2 * k + (IS_POS(u[k]) ? 0 : 1);   // entered through -h (u>0) or +h
        }
        if (Af == 0.0 || MUL(F, Af) < MUL(Nf, a)) { Nf = F; Af = a; }
    }
    // hit iff entry <= exit and exit >= 0
    if (!(Af == 0.0 || (MUL(Nn, Af) <= MUL(Nf, An) && NONNEG(Nf)))) return d_inf();
    if (FACE && IS_POS(Nn)) *face = fn;
    return IS_POS(Nn) ? DIV(Nn, An) : 0.0;
}


// REENTRY: the start point lies on the surface of a solid it has just left;
// the inside test is skipped and only entering crossings strictly after the
// start count (the crossing it left through is an exiting one).
template <bool FACE = false, bool REENTRY = false>
__device__ __forceinline__ double tube_out64(const double* d, const double* x, const double* u, int* face = nullptr) {
    if (FACE) *face = -1;
    const double rmin = d[0], dz = d[2], rmin2 = d[3], rmax2 = d[4];
    const double rho2 = rho2_of(x);
    if (!REENTRY && ABS_LE(x[2], dz) && LE(rho2, rmax2) && LE(rmin2, rho2)) return 0.0;
    double best = d_inf();
    {   // the z-plane the track approaches from outside the slab
        const bool zc = ABS_GT(x[2], dz) && OPPOSITE(x[2], u[2]);
        const double t = DIV(SUB(copysign(dz, x[2]), x[2]), zc ? u[2] : 1.0);
        const double xh = FMA(t, u[0], x[0]), yh = FMA(t, u[1], x[1]);
        const double r2 = DOT2(xh, xh, yh, yh);
        if (zc && LE(r2, rmax2) && LE(rmin2, r2)) {
            best = t;
            if (FACE) *face = IS_POS(x[2]) ? 5 : 4;
        }
    }
    const double A = DOT2(u[0], u[0], u[1], u[1]);
    const double B = DOT2(x[0], u[0], x[1], u[1]);
    {   // outer cylinder, crossed inwards
        const double s = root_falling(A, B, SUB(rho2, rmax2));
        if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && ABS_LE(FMA(s, u[2], x[2]), dz)) {
            best = s;
            if (FACE) *face = 6;
        }
    }
    if (rmin > 0.0) {   // inner cylinder, crossed outwards (out of the hole)
        const double s = root_rising(A, B, SUB(rho2, rmin2));
        if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && ABS_LE(FMA(s, u[2], x[2]), dz)) {
            best = s;
            if (FACE) *face = 7;
        }
    }
    return best;
}

// Tube segment: the tube's candidates restricted to the wedge, and the two
// phi faces (entered where the track crosses a face's plane into the wedge
// side, at a point of the face: rmin <= r <= rmax along the face's
// direction, |z| <= dz).
template <bool FACE = false, bool REENTRY = false>
__device__ __forceinline__ double tubs_out64(const double* d, const double* x, const double* u, int* face = nullptr) {
    if (FACE) *face = -1;
    const double rmin = d[0], dz = d[2], rmin2 = d[3], rmax2 = d[4];
    const double rho2 = rho2_of(x);
    if (!REENTRY && ABS_LE(x[2], dz) && LE(rho2, rmax2) && LE(rmin2, rho2) && wedge_has64(d, x[0], x[1]))
        return 0.0;
    double best = d_inf();
    {   // the z-plane the track approaches from outside the slab
        const bool zc = ABS_GT(x[2], dz) && OPPOSITE(x[2], u[2]);
        const double t = DIV(SUB(copysign(dz, x[2]), x[2]), zc ? u[2] : 1.0);
        const double xh = FMA(t, u[0], x[0]), yh = FMA(t, u[1], x[1]);
        const double r2 = DOT2(xh, xh, yh, yh);
        if (zc && LE(r2, rmax2) && LE(rmin2, r2) && wedge_has64(d, xh, yh)) {
            best = t;
            if (FACE) *face = IS_POS(x[2]) ? 5 : 4;
        }
    }
    const double A = DOT2(u[0], u[0], u[1], u[1]);
    const double B = DOT2(x[0], u[0], x[1], u[1]);
    {   // outer cylinder, crossed inwards
        const double s = root_falling(A, B, SUB(rho2, rmax2));
        if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && ABS_LE(FMA(s, u[2], x[2]), dz) &&
            wedge_has64(d, FMA(s, u[0], x[0]), FMA(s, u[1], x[1]))) {
            best = s;
            if (FACE) *face = 6;
        }
    }
    if (rmin > 0.0) {   // inner cylinder, crossed outwards (out of the hole)
        const double s = root_rising(A, B, SUB(rho2, rmin2));
        if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && ABS_LE(FMA(s, u[2], x[2]), dz) &&
            wedge_has64(d, FMA(s, u[0], x[0]), FMA(s, u[1], x[1]))) {
            best = s;
            if (FACE) *face = 7;
        }
    }
    if (d[10] == 0.0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double nx = d[5 + 2 * i], ny = d[6 + 2 * i];
            const double ex = i == 0 ? ny : -ny, ey = i == 0 ? -nx : nx;   // the face's direction
            const double wn = DOT2(nx, u[0], ny, u[1]);
            if (!IS_POS(wn)) continue;                                       // not moving to the wedge side
            const double s = DIV(-DOT2(nx, x[0], ny, x[1]), wn);
            if (!(REENTRY ? IS_POS(s) : NONNEG(s)) || !LT(s, best)) continue;
            const double xh = FMA(s, u[0], x[0]), yh = FMA(s, u[1], x[1]);
            const double r2 = DOT2(xh, xh, yh, yh);
            const double tau2 = MUL(0x1p-101, FMA(MUL(s, s), A, rho2));
            if (ABS_LE(FMA(s, u[2], x[2]), dz) && LE(r2, rmax2) && LE(rmin2, r2) &&
                on_phi_face(d, ex, ey, xh, yh, r2, IS_ZERO(rmin2), tau2, u)) {
                best = s;
                if (FACE) *face = 8 + i;
            }
        }
    }
    return best;
}

// Out-of-line entry of the tube segment, so that its code stays out of the
// kernels' hot paths (a segment is evaluated only where one is placed).
template <bool FACE, bool REENTRY>
__device__ __noinline__ double tubs_out64_call(const double* d, double x0, double x1, double x2, double u0, double u1,
                                               double u2, int* face) {
    const double x[3] = {x0, x1, x2}, u[3] = {u0, u1, u2};
    return tubs_out64<FACE, REENTRY>(d, x, u, face);
}
// Crossing of a cone's radius line R(z) = b (z - zc) through its apex at the
// end plane zc = -dz (low) or +dz, formed about the apex (cone_root_about);
// sets whether its height lies in [-dz, dz].  Out of line: apexes are rare,
// and the cone routine of the hot kernels keeps its registers.
static __device__ __noinline__ double cone_apex_root(bool rising, bool low, double dz, double b, double x0, double x1,
                                                     double x2, double u0, double u1, double u2, bool* in_z) {
    const double x[3] = {x0, x1, x2}, u[3] = {u0, u1, u2};
    const double A0 = DOT2(u0, u0, u1, u1);
    const double inv_uu = DIV(1.0, FMA(u2, u2, A0));
    double xh, yh, zh;
    const double zc = low ? -dz : dz;
    const double s = rising ? cone_root_about<true>(zc, 0.0, b, x, u, A0, inv_uu, xh, yh, zh)
                            : cone_root_about<false>(zc, 0.0, b, x, u, A0, inv_uu, xh, yh, zh);
    const double w = ADD(dz, dz);
    *in_z = low ? (zh >= 0.0 && zh <= w) : (zh <= 0.0 && zh >= -w);
    return s;
}

// APEX: the instantiation that forms the crossing of a cone through an apex on
// an end plane about that apex (volumes holding such a cone run it).
template <bool FACE = false, bool REENTRY = false, bool APEX = true>
__device__ __forceinline__ double cone_out64(const double* d, const double* x, const double* u, int* face = nullptr) {
    if (FACE) *face = -1;
    const double dz = d[0];
    const double rho2 = rho2_of(x);
    const double ro0 = FMA(d[2], x[2], d[1]);
    const double ri0 = FMA(d[4], x[2], d[3]);
    const bool hole = d[11] != 0.0;
    if (!REENTRY && ABS_LE(x[2], dz) && LE(rho2, MUL(ro0, ro0)) && (!hole || LE(MUL(ri0, ri0), rho2)))
        return 0.0;
    double best = d_inf();
    {   // the z-plane the track approaches from outside the slab
        const bool zc = ABS_GT(x[2], dz) && OPPOSITE(x[2], u[2]);
        const double t = DIV(SUB(copysign(dz, x[2]), x[2]), zc ? u[2] : 1.0);
        const double xh = FMA(t, u[0], x[0]), yh = FMA(t, u[1], x[1]);
        const double r2 = DOT2(xh, xh, yh, yh);
        const double lo2 = IS_POS(x[2]) ? d[7] : d[5];
        const double hi2 = IS_POS(x[2]) ? d[8] : d[6];
        if (zc && LE(r2, hi2) && LE(lo2, r2)) {
            best = t;
            if (FACE) *face = IS_POS(x[2]) ? 5 : 4;
        }
    }
    const double A0 = DOT2(u[0], u[0], u[1], u[1]);
    const double B0 = DOT2(x[0], u[0], x[1], u[1]);
    // a radius vanishing at an end plane (an apex there): that cone's
    // crossing is formed about the apex, out of line (cone_apex_root)
    const bool apex_o = IS_ZERO(d[6]) || IS_ZERO(d[8]), apex_i = hole && (IS_ZERO(d[5]) || IS_ZERO(d[7]));
    {   // outer cone rho^2 - (a + b z)^2, crossed inwards
        double s;
        bool in_z;
        if (APEX && apex_o) {
            s = cone_apex_root(false, IS_ZERO(d[6]), dz, d[2], x[0], x[1], x[2], u[0], u[1], u[2], &in_z);
        } else {
            const double rs = MUL(d[2], u[2]);
            s = root_falling(FMA(-rs, rs, A0), FMA(-ro0, rs, B0), FMA(-ro0, ro0, rho2));
            in_z = ABS_LE(FMA(s, u[2], x[2]), dz);
        }
        if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && in_z) {
            best = s;
            if (FACE) *face = 6;
        }
    }
    if (hole) {   // inner cone, crossed outwards
        double s;
        bool in_z;
        if (APEX && apex_i) {
            s = cone_apex_root(true, IS_ZERO(d[5]), dz, d[4], x[0], x[1], x[2], u[0], u[1], u[2], &in_z);
        } else {
            const double rs = MUL(d[4], u[2]);
            s = root_rising(FMA(-rs, rs, A0), FMA(-ri0, rs, B0), FMA(-ri0, ri0, rho2));
            in_z = ABS_LE(FMA(s, u[2], x[2]), dz);
        }
        if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && in_z) {
            best = s;
            if (FACE) *face = 7;
        }
    }
    return best;
}

// Polycone: the end planes (entered from outside the z-range at a point of
// the end annulus in the wedge), the phi faces (as for the tube segment, at a
// point of the cross-section), and every section's outer cone crossed inwards
// and inner cone crossed outwards at a height inside the section's z-range
// and an azimuth in the wedge.  Sections are visited in the order the track
// meets them, from the one holding its start, and the visit stops at the
// first section beyond the best candidate so far (the segment search).
template <bool FACE = false, bool REENTRY = false>
__device__ __forceinline__ double pcon_out64(const double* d, const double* T, const double* x, const double* u,
                                             int* face = nullptr) {
    if (FACE) *face = -1;
    const int n = int(d[1]);
    const double *z = T, *rn = T + n, *rx = T + 2 * n, *bi = T + 3 * n, *bo = bi + (n - 1);
    const double rho2 = rho2_of(x);
    if (!REENTRY && pcon_in2(T, n, rho2, x[2]) && wedge_has64(d, x[0], x[1])) return 0.0;
    double best = d_inf();
    {   // the end plane the track approaches from outside the z-range
        const bool lo = x[2] < z[0] && IS_POS(u[2]), hi = x[2] > z[n - 1] && IS_NEG(u[2]);
        const double t = DIV(SUB(lo ? z[0] : z[n - 1], x[2]), (lo || hi) ? u[2] : 1.0);
        const double xh = FMA(t, u[0], x[0]), yh = FMA(t, u[1], x[1]);
        const double r2 = DOT2(xh, xh, yh, yh);
        if ((lo || hi) && LE(r2, lo ? d[3] : d[12]) && LE(lo ? d[2] : d[4], r2) && wedge_has64(d, xh, yh)) {
            best = t;
            if (FACE) *face = lo ? 4 : 5;
        }
    }
    if (d[10] == 0.0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double nx = d[5 + 2 * i], ny = d[6 + 2 * i];
            const double ex = i == 0 ? ny : -ny, ey = i == 0 ? -nx : nx;   // the face's direction
            const double wn = DOT2(nx, u[0], ny, u[1]);
            if (!IS_POS(wn)) continue;                                       // not moving to the wedge side
            const double s = DIV(-DOT2(nx, x[0], ny, x[1]), wn);
            if (!(REENTRY ? IS_POS(s) : NONNEG(s)) || !LT(s, best)) continue;
            const double xh = FMA(s, u[0], x[0]), yh = FMA(s, u[1], x[1]);
            const double r2 = DOT2(xh, xh, yh, yh);
            const double tau2 = MUL(0x1p-101, FMA(MUL(s, s), DOT2(u[0], u[0], u[1], u[1]), rho2));
            if (pcon_in2(T, n, r2, FMA(s, u[2], x[2])) && on_phi_face(d, ex, ey, xh, yh, r2, true, tau2, u)) {
                best = s;
                if (FACE) *face = 8 + i;
            }
        }
    }
    const double A0 = DOT2(u[0], u[0], u[1], u[1]);
    const double inv_uu = DIV(1.0, FMA(u[2], u[2], A0));
    auto section = [&](int k) {
        const double zk = z[k], zk1 = z[k + 1];
        double xh, yh;
        bool in_z;
        {   // outer cone, crossed inwards
            const double s = pcon_sec_root<false>(rx[k], rx[k + 1], bo[k], zk, zk1, x, u, A0, inv_uu, xh, yh, in_z);
            if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && in_z && wedge_has64(d, xh, yh)) {
                best = s;
                if (FACE) *face = 16 + 2 * k;
            }
        }
        if (rn[k] > 0.0 || rn[k + 1] > 0.0) {   // inner cone, crossed outwards (out of the hole)
            const double s = pcon_sec_root<true>(rn[k], rn[k + 1], bi[k], zk, zk1, x, u, A0, inv_uu, xh, yh, in_z);
            if ((REENTRY ? IS_POS(s) : NONNEG(s)) && LT(s, best) && in_z && wedge_has64(d, xh, yh)) {
                best = s;
                if (FACE) *face = 17 + 2 * k;
            }
        }
    };
    // heights the track reaches before `best`, with a margin far above rounding
    auto reach = [&]() {
        const double zr = FMA(best, u[2], x[2]);
        return zr + copysign(1e-12 * (fabs(zr) + 1.0), u[2]);
    };
    if (IS_ZERO(u[2])) {
        if (x[2] >= z[0] && x[2] <= z[n - 1]) {
            const int k = pcon_section(z, n, x[2]);
            section(k);
            if (k > 0 && x[2] == z[k]) section(k - 1);
        }
    } else {
        // one loop for both directions (lanes moving up and down share its
        // iterations instead of running two loops one after the other)
        const bool up = IS_POS(u[2]);
        const int dk = up ? 1 : -1;
        for (int k = pcon_section(z, n, x[2]); k >= 0 && k < n - 1; k += dk) {
            const double r = reach();
            if (up ? z[k] > r : z[k + 1] < r) break;
            section(k);
        }
    }
    return best;
}

// Out-of-line entry of the polycone (see tubs_out64_call).
template <bool FACE, bool REENTRY>
__device__ __noinline__ double pcon_out64_call(const double* d, const double* T, double x0, double x1, double x2,
                                               double u0, double u1, double u2, int* face) {
    const double x[3] = {x0, x1, x2}, u[3] = {u0, u1, u2};
    return pcon_out64<FACE, REENTRY>(d, T, x, u, face);
}

// SEGS = false: the volume holds no tube segment or polycone, and their code
// is left out.
template <bool FACE = false, bool SEGS = true>
__device__ __forceinline__ double dist_out64(const ShapeRec64& r, const double* x, const double* u,
                                             int* face = nullptr) {
    if (r.kind == KBOX) return box_out64<FACE>(r.d, x, u, face);
    if (r.kind == KTUBE) return tube_out64<FACE>(r.d, x, u, face);
    if (SEGS && r.kind == KTUBS) return tubs_out64_call<FACE, false>(r.d, x[0], x[1], x[2], u[0], u[1], u[2], face);
    if (SEGS && r.kind == KPCON)
        return pcon_out64_call<FACE, false>(r.d, pcon_table(r.d), x[0], x[1], x[2], u[0], u[1], u[2], face);
    return cone_out64<FACE, false, SEGS>(r.d, x, u, face);
}

// Distance to enter again a solid the track has just left (its start point
// on the solid's surface): +inf for a convex solid, the crossing on the far
// side of the hole for a shell left into its hole.
template <bool FACE = false>
__device__ __forceinline__ double reentry64(const ShapeRec64& r, const double* x, const double* u,
                                           int* face = nullptr) {
    if (r.kind == KBOX) {
        if (contains64(r, x)) {
            if (FACE) *face = -1;
            return d_inf();
        }
        return box_out64<FACE>(r.d, x, u, face);
    }
    if (r.kind == KTUBE) return tube_out64<FACE, true>(r.d, x, u, face);
    if (r.kind == KTUBS) return tubs_out64_call<FACE, true>(r.d, x[0], x[1], x[2], u[0], u[1], u[2], face);
    if (r.kind == KPCON)
        return pcon_out64_call<FACE, true>(r.d, pcon_table(r.d), x[0], x[1], x[2], u[0], u[1], u[2], face);
    return cone_out64<FACE, true>(r.d, x, u, face);
}

// ------------------------------------------------------- DistFromInside ---
// First s >= 0 at which the track violates a constraint (x assumed inside).
__device__ __forceinline__ double slab_exit(double xk, double uk, double h) {
    const bool z = IS_ZERO(uk);
    const double t = DIV(SUB(copysign(h, uk), xk), z ? 1.0 : uk);
    return z ? d_inf() : t;
}

// Exit parameters of a point inside are >= 0 up to the sign of a zero; the
// minimum is taken on the bit patterns and the result clamped at +0.
__device__ __forceinline__ double clamp0(double t) { return NONNEG(t) && !IS_ZERO(t) ? t : 0.0; }

// Exit from the wedge of a segment (d as in geo_internal.h): each half-plane
// holds s where c + s w >= 0; take(exit, face) is called with the candidates.
template <typename Take>
__device__ __forceinline__ void wedge_exit64(const double* d, const double* x, const double* u, Take& take) {
    // the wedge: each half-plane holds s where c + s w >= 0
    const double c1 = DOT2(d[5], x[0], d[6], x[1]), w1 = DOT2(d[5], u[0], d[6], u[1]);
    const double c2 = DOT2(d[7], x[0], d[8], x[1]), w2 = DOT2(d[7], u[0], d[8], u[1]);
    const double e1 = IS_NEG(w1) ? DIV(-c1, w1) : d_inf();   // where the track leaves half-plane 1
    const double e2 = IS_NEG(w2) ? DIV(-c2, w2) : d_inf();
    if (d[9] != 0.0) {
        // intersection: leaves the wedge when it leaves either (when
        // dphi = pi the two planes coincide, and the face is the one
        // on whose side of the axis the track leaves)
        if (d[11] != 0.0) {
            const double ec = MINP(clamp0(e1), clamp0(e2));
            const double xh = FMA(ec, u[0], x[0]), yh = FMA(ec, u[1], x[1]);
            take(ec, NONNEG(DOT2(d[6], xh, -d[5], yh)) ? 8 : 9);
        } else {
            take(clamp0(e1), 8);
            take(clamp0(e2), 9);
        }
    } else {
        // union: of the half-lines holding the start (c >= 0), a
        // rising one (w >= 0) never ends; a falling one ends at e; a
        // rising one that starts later (at -c/w > 0) continues the
        // union if it starts before that end
        const bool in1 = NONNEG(c1), in2 = NONNEG(c2);
        const bool up1 = !IS_NEG(w1), up2 = !IS_NEG(w2);
        if (!((in1 && up1) || (in2 && up2))) {
            // every half-plane holding the start ends: the later end
            const double x1 = in1 ? clamp0(e1) : 0.0, x2 = in2 ? clamp0(e2) : 0.0;
            const bool second = in2 && (!in1 || LT(x1, x2));
            const double E = second ? x2 : x1;
            // a half-plane not holding the start but entered by then
            // continues the union
            const double a1 = (!in1 && IS_POS(w1)) ? DIV(-c1, w1) : d_inf();
            const double a2 = (!in2 && IS_POS(w2)) ? DIV(-c2, w2) : d_inf();
            if (!(LE(a1, E) || LE(a2, E))) take(E, second ? 9 : 8);
        }
    }
}

// Tube segment, DistFromInside: the tube's exits and the wedge's.
template <bool FACE = false>
__device__ __forceinline__ double tubs_in64(const double* d, const double* x, const double* u, int* face = nullptr) {
    double t = d_inf();
    int f = -1;
    auto take = [&](double c, int fc) {
        if (LT(c, t)) {
            t = c;
            if (FACE) f = fc;
        }
    };
    const double rho2 = rho2_of(x);
    const double A0 = DOT2(u[0], u[0], u[1], u[1]);
    const double B0 = DOT2(x[0], u[0], x[1], u[1]);
    double s;
    take(clamp0(slab_exit(x[2], u[2], d[2])), IS_POS(u[2]) ? 5 : 4);
    s = root_rising(A0, B0, SUB(rho2, d[4]));
    if (NONNEG(s)) take(clamp0(s), 6);
    if (d[0] > 0.0) {
        s = root_falling(A0, B0, SUB(rho2, d[3]));
        if (NONNEG(s)) take(clamp0(s), 7);
    }
    if (d[10] == 0.0) wedge_exit64(d, x, u, take);
    if (FACE) *face = f;
    return t;
}

// Out-of-line entry of the tube segment's DistFromInside (see tubs_out64_call).
template <bool FACE>
__device__ __noinline__ double tubs_in64_call(const double* d, double x0, double x1, double x2, double u0, double u1,
                                              double u2, int* face) {
    const double x[3] = {x0, x1, x2}, u[3] = {u0, u1, u2};
    return tubs_in64<FACE>(d, x, u, face);
}

// Polycone, DistFromInside.  The solid is the intersection of four
// constraints: the z-range, rho <= Rout(z) and rho >= Rin(z) (piecewise
// linear radii) and the wedge; the exit is the least of their exits.  The
// first violation of a radius constraint is the first crossing of a
// section's outer cone outwards (or inner cone inwards) at a height inside
// that section's z-range; sections are visited from the start's, in the
// track's direction, up to the least exit so far.
template <bool FACE = false>
__device__ __forceinline__ double pcon_in64(const double* d, const double* T, const double* x, const double* u,
                                            int* face = nullptr) {
    double t = d_inf();
    int f = -1;
    auto take = [&](double c, int fc) {
        if (LT(c, t)) {
            t = c;
            if (FACE) f = fc;
        }
    };
    const int n = int(d[1]);
    const double *z = T, *rn = T + n, *rx = T + 2 * n, *bi = T + 3 * n, *bo = bi + (n - 1);
    const double A0 = DOT2(u[0], u[0], u[1], u[1]);
    const double inv_uu = DIV(1.0, FMA(u[2], u[2], A0));
    if (!IS_ZERO(u[2])) {   // the end plane ahead
        const bool up = IS_POS(u[2]);
        take(clamp0(DIV(SUB(up ? z[n - 1] : z[0], x[2]), u[2])), up ? 5 : 4);
    }
    if (d[10] == 0.0) wedge_exit64(d, x, u, take);
    auto section = [&](int k) {
        const double zk = z[k], zk1 = z[k + 1];
        double xh, yh;
        bool in_z;
        {   // outer cone, crossed outwards
            const double s = pcon_sec_root<true>(rx[k], rx[k + 1], bo[k], zk, zk1, x, u, A0, inv_uu, xh, yh, in_z);
            if (NONNEG(s) && LT(clamp0(s), t) && in_z) take(clamp0(s), 16 + 2 * k);
        }
        if (rn[k] > 0.0 || rn[k + 1] > 0.0) {   // inner cone, crossed inwards (into the hole)
            const double s = pcon_sec_root<false>(rn[k], rn[k + 1], bi[k], zk, zk1, x, u, A0, inv_uu, xh, yh, in_z);
            if (NONNEG(s) && LT(clamp0(s), t) && in_z) take(clamp0(s), 17 + 2 * k);
        }
    };
    auto reach = [&]() {
        const double zr = FMA(t, u[2], x[2]);
        return zr + copysign(1e-12 * (fabs(zr) + 1.0), u[2]);
    };
    if (IS_ZERO(u[2])) {
        const int k = pcon_section(z, n, x[2]);
        section(k);
        if (k > 0 && x[2] == z[k]) section(k - 1);
    } else {
        const bool up = IS_POS(u[2]);
        const int dk = up ? 1 : -1;
        for (int k = pcon_section(z, n, x[2]); k >= 0 && k < n - 1; k += dk) {
            const double r = reach();
            if (up ? z[k] > r : z[k + 1] < r) break;
            section(k);
        }
    }
    if (FACE) *face = f;
    return t;
}

// Out-of-line entry of the polycone's DistFromInside (see tubs_out64_call).
template <bool FACE>
__device__ __noinline__ double pcon_in64_call(const double* d, const double* T, double x0, double x1, double x2,
                                              double u0, double u1, double u2, int* face) {
    const double x[3] = {x0, x1, x2}, u[3] = {u0, u1, u2};
    return pcon_in64<FACE>(d, T, x, u, face);
}

template <bool FACE = false, bool SEGS = true>
__device__ __forceinline__ double dist_in64(const ShapeRec64& r, const double* x, const double* u,
                                            int* face = nullptr) {
    // the exit is the least of the constraints' exit parameters (minimum on
    // the bit patterns of values >= 0; equal values are equal bit patterns)
    const double* d = r.d;
    if (SEGS && r.kind == KTUBS) return tubs_in64_call<FACE>(d, x[0], x[1], x[2], u[0], u[1], u[2], face);
    if (SEGS && r.kind == KPCON)
        return pcon_in64_call<FACE>(d, pcon_table(d), x[0], x[1], x[2], u[0], u[1], u[2], face);
    double t;
    int f = -1;
    auto take = [&](double c, int fc) {
        if (LT(c, t)) {
            t = c;
            if (FACE) f = fc;
        }
    };
    if (r.kind == KBOX) {
        t = d_inf();
#pragma unroll
        for (int k = 0; k < 3; ++k) take(clamp0(slab_exit(x[k], u[k], d[k])), 2 * k + (IS_POS(u[k]) ? 1 : 0));
        if (FACE) *face = f;
        return t;
    }
    const double rho2 = rho2_of(x);
    const double A0 = DOT2(u[0], u[0], u[1], u[1]);
    const double B0 = DOT2(x[0], u[0], x[1], u[1]);
    double s;
    if (r.kind == KTUBE) {
        t = d_inf();
        take(clamp0(slab_exit(x[2], u[2], d[2])), IS_POS(u[2]) ? 5 : 4);
        s = root_rising(A0, B0, SUB(rho2, d[4]));
        if (NONNEG(s)) take(clamp0(s), 6);
        if (d[0] > 0.0) {
            s = root_falling(A0, B0, SUB(rho2, d[3]));
            if (NONNEG(s)) take(clamp0(s), 7);
        }
        if (FACE) *face = f;
        return t;
    }
    t = d_inf();
    take(clamp0(slab_exit(x[2], u[2], d[0])), IS_POS(u[2]) ? 5 : 4);
    {
        const double ro0 = FMA(d[2], x[2], d[1]), rs = MUL(d[2], u[2]);
        s = root_rising(FMA(-rs, rs, A0), FMA(-ro0, rs, B0), FMA(-ro0, ro0, rho2));
        if (NONNEG(s)) take(clamp0(s), 6);
    }
    if (d[11] != 0.0) {
        const double ri0 = FMA(d[4], x[2], d[3]), rs = MUL(d[4], u[2]);
        s = root_falling(FMA(-rs, rs, A0), FMA(-ri0, rs, B0), FMA(-ri0, ri0, rho2));
        if (NONNEG(s)) take(clamp0(s), 7);
    }
    if (FACE) *face = f;
    return t;
}

// --------------------------------------------------------------- safety ---
// 2-D distance from (px, pz) to the segment a-b in the meridian half-plane.
__device__ __forceinline__ double seg2(double px, double pz, double ax, double az, double bx, double bz) {
    const double ex = SUB(bx, ax), ez = SUB(bz, az);
    const double l2 = DOT2(ex, ex, ez, ez);
    double f = l2 > 0.0 ? DIV(DOT2(SUB(px, ax), ex, SUB(pz, az), ez), l2) : 0.0;
    f = fmin(fmax(f, 0.0), 1.0);
    const double cx = SUB(FMA(f, ex, ax), px), cz = SUB(FMA(f, ez, az), pz);
    return SQRT(DOT2(cx, cx, cz, cz));
}

// 2-D distance from (r, v) to the boundary edges of a polycone's cross-section:
// the end caps, the outer edges and the inner edges (those on the axis only
// when `axis`).
__device__ __forceinline__ double pcon_edges(const double* T, int n, double r, double v, bool axis) {
    const double *z = T, *rn = T + n, *rx = T + 2 * n;
    double s = fmin(seg2(r, v, rn[0], z[0], rx[0], z[0]), seg2(r, v, rn[n - 1], z[n - 1], rx[n - 1], z[n - 1]));
    for (int k = 0; k < n - 1; ++k) {
        s = fmin(s, seg2(r, v, rx[k], z[k], rx[k + 1], z[k + 1]));
        if (axis || rn[k] > 0.0 || rn[k + 1] > 0.0) s = fmin(s, seg2(r, v, rn[k], z[k], rn[k + 1], z[k + 1]));
    }
    return s;
}

// Polycone safety: 2-D distances in the meridian half-plane to the edges of
// the cross-section (inside: the edges that are surfaces; outside, azimuth in
// the wedge: all of them), and for a wedge the distance to each phi face
// (its plane's normal distance and the 2-D distance of the projection to the
// cross-section; outside the wedge the nearest azimuth is an end).
static __device__ __noinline__ double pcon_safety64(const double* d, const double* T, double x0, double x1, double x2,
                                             bool in) {
    const int n = int(d[1]);
    const double rho = SQRT(DOT2(x0, x0, x1, x1));
    double fd[2] = {d_inf(), d_inf()};
    if (d[10] == 0.0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const double nx = d[5 + 2 * i], ny = d[6 + 2 * i];
            const double ex = i == 0 ? ny : -ny, ey = i == 0 ? -nx : nx;
            const double h = DOT2(nx, x0, ny, x1);
            const double rr = DOT2(ex, x0, ey, x1);
            const double d2 = (NONNEG(rr) && pcon_in2(T, n, MUL(rr, rr), x2)) ? 0.0 : pcon_edges(T, n, rr, x2, true);
            fd[i] = SQRT(FMA(h, h, MUL(d2, d2)));
        }
    }
    if (in) return fmin(pcon_edges(T, n, rho, x2, false), fmin(fd[0], fd[1]));
    if (d[10] != 0.0 || wedge_has64(d, x0, x1)) return pcon_edges(T, n, rho, x2, true);
    return fmin(fd[0], fd[1]);
}

// Distance to the boundary from a point inside (inside == true) or outside.
// Returns 0 if the point is on the other side.
template <bool SEGS = true>
__device__ __forceinline__ double safety64(const ShapeRec64& r, const double* x, bool inside) {
    const bool in = contains64<SEGS>(r, x);
    if (in != inside) return 0.0;
    const double* d = r.d;
    if (SEGS && r.kind == KPCON) return pcon_safety64(d, pcon_table(d), x[0], x[1], x[2], in);
    if (r.kind == KBOX) {
        const double a = SUB(fabs(x[0]), d[0]), b = SUB(fabs(x[1]), d[1]), c = SUB(fabs(x[2]), d[2]);
        if (in) return -fmax(a, fmax(b, c));
        const double a0 = fmax(a, 0.0), b0 = fmax(b, 0.0), c0 = fmax(c, 0.0);
        return SQRT(FMA(a0, a0, DOT2(b0, b0, c0, c0)));
    }
    const double rho = SQRT(rho2_of(x));
    const double az = fabs(x[2]);
    if (r.kind == KTUBS) {
        // phi faces: the rectangles rmin <= r <= rmax, |z| <= dz of the two
        // half-planes (distance with the foot clamped into the rectangle)
        double fd[2] = {d_inf(), d_inf()};
        if (d[10] == 0.0) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const double nx = d[5 + 2 * i], ny = d[6 + 2 * i];
                const double ex = i == 0 ? ny : -ny, ey = i == 0 ? -nx : nx;
                const double h = DOT2(nx, x[0], ny, x[1]);
                const double rr = DOT2(ex, x[0], ey, x[1]);
                const double rc = fmin(fmax(rr, d[0]), d[1]);
                const double dr = SUB(rr, rc), dzf = fmax(SUB(az, d[2]), 0.0);
                fd[i] = SQRT(FMA(h, h, DOT2(dr, dr, dzf, dzf)));
            }
        }
        if (in) {
            double s = fmin(SUB(d[1], rho), SUB(d[2], az));
            if (d[0] > 0.0) s = fmin(s, SUB(rho, d[0]));
            return fmin(s, fmin(fd[0], fd[1]));
        }
        if (wedge_has64(d, x[0], x[1])) {
            // azimuth in the wedge: the tube's distance in the meridian plane
            const double dzo = fmax(SUB(az, d[2]), 0.0);
            const double dro = fmax(fmax(SUB(d[0], rho), SUB(rho, d[1])), 0.0);
            return SQRT(DOT2(dzo, dzo, dro, dro));
        }
        // azimuth outside: the nearest azimuth of the wedge is one of its ends
        return fmin(fd[0], fd[1]);
    }
    if (r.kind == KTUBE) {
        if (in) {
            double s = fmin(SUB(d[1], rho), SUB(d[2], az));
            if (d[0] > 0.0) s = fmin(s, SUB(rho, d[0]));
            return s;
        }
        const double dzo = fmax(SUB(az, d[2]), 0.0);
        const double dro = fmax(fmax(SUB(d[0], rho), SUB(rho, d[1])), 0.0);
        return SQRT(DOT2(dzo, dzo, dro, dro));
    }
    // cone: trapezoid (rmin1,-dz) (rmax1,-dz) (rmax2,dz) (rmin2,dz)
    const double dz = d[0], z = x[2];
    if (in) {
        // inside a convex polygon the nearest boundary point lies on the
        // nearest supporting line of an edge
        double s = SUB(dz, az);
        s = fmin(s, MUL(SUB(FMA(d[2], z, d[1]), rho), d[9]));
        if (d[11] != 0.0) s = fmin(s, MUL(SUB(rho, FMA(d[4], z, d[3])), d[10]));
        return s;
    }
    const double r1i = r.p[1], r1o = r.p[2], r2i = r.p[3], r2o = r.p[4];
    double s = seg2(rho, z, r1i, -dz, r1o, -dz);
    s = fmin(s, seg2(rho, z, r1o, -dz, r2o, dz));
    s = fmin(s, seg2(rho, z, r2o, dz, r2i, dz));
    s = fmin(s, seg2(rho, z, r2i, dz, r1i, -dz));
    return s;
}

}  // namespace geonav
