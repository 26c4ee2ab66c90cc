// nav_common.cuh -- the FP64 navigator step of Fig. 1 for one track, shared by
// the plain FP64 kernel and by the fallback of the FP32-filter kernel, so
// both produce bit-identical answers.
#pragma once
#include "geo_internal.h"
#include "shapes64.cuh"

namespace geonav {

// Invalid input (non-finite or zero direction): NaN, -2.  Returns false.
// (exponent bits checked with integer operations)
__device__ __forceinline__ bool finite64(double a) { return (BITS(a) & kAbsMask) < 0x7ff0000000000000LL; }
__device__ __forceinline__ bool valid_track(double px, double py, double pz, double qx, double qy, double qz) {
    const bool finite = finite64(px) && finite64(py) && finite64(pz) && finite64(qx) && finite64(qy) &&
                        finite64(qz);
    return finite && !(IS_ZERO(qx) && IS_ZERO(qy) && IS_ZERO(qz));
}

// Mother DistFromInside, then for every daughter: bounding-sphere test against
// the current best, master->local transform, DistFromOutside, strict '<'
// (mother first, then the lowest index win ties).  Track assumed valid and
// inside the mother.
__device__ __forceinline__ void nav_all64(const ShapeRec64& m, const ShapeRec64* __restrict__ tab, int nd,
                                          double px, double py, double pz, double qx, double qy, double qz,
                                          double& best, int& h) {
    const double p[3] = {px, py, pz}, q[3] = {qx, qy, qz};
    best = dist_in64(m, p, q);
    h = -1;
    const double dd = qx * qx + qy * qy + qz * qz;
    const double dn = sqrt(dd);
    for (int j = 0; j < nd; ++j) {
        const ShapeRec64& r = tab[j];
        // bounding sphere about t: centre parameter proj/dd, radius brad/|d|
        // (brad is enlarged on the host, so these culls are conservative)
        const double w0 = r.t[0] - px, w1 = r.t[1] - py, w2 = r.t[2] - pz;
        const double proj = w0 * qx + w1 * qy + w2 * qz;
        const double rb = r.brad * dn;
        if (proj + rb < 0.0) continue;                  // sphere entirely behind
        if (proj - rb >= best * dd) continue;           // sphere starts beyond best
        const double ww = w0 * w0 + w1 * w1 + w2 * w2;
        if (ww * dd - proj * proj > rb * rb) continue;  // line misses the sphere
        double x[3], u[3];
        to_local64(r, px, py, pz, qx, qy, qz, x, u);
        const double s = dist_out64(r, x, u);
        if (LT(s, best)) {
            best = s;
            h = j;
        }
    }
}

__device__ __forceinline__ void store_result(int64_t i, int64_t n, double best, int h, double px, double py,
                                             double pz, double qx, double qy, double qz, double* step,
                                             int32_t* hit, double* bpoint) {
    step[i] = best;
    hit[i] = h;
    if (bpoint) {
        bpoint[i] = FMA(best, qx, px);
        bpoint[n + i] = FMA(best, qy, py);
        bpoint[2 * n + i] = FMA(best, qz, pz);
    }
}

}  // namespace geonav
