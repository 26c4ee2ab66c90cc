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
template <bool SEGS = true>
__device__ __forceinline__ void nav_all64(const ShapeRec64& m, const ShapeRec64* __restrict__ tab, int nd,
                                          double px, double py, double pz, double qx, double qy, double qz,
                                          double& best, int& h) {
    const double p[3] = {px, py, pz}, q[3] = {qx, qy, qz};
    best = dist_in64<false, SEGS>(m, p, q);
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
        const double s = dist_out64<false, SEGS>(r, x, u);
        if (LT(s, best)) {
            best = s;
            h = j;
        }
    }
}

// The same step with the uniform grid: cells are walked in ray order (FP64
// 3D-DDA) and the walk stops once the best step lies before the exit of the
// cell just finished (with a relative margin of 2^-40): every daughter the
// track could still enter starts in a later cell.  Daughters arrive out of
// index order, so ties are resolved explicitly (mother, then lowest index).
__device__ __forceinline__ void nav_vox64(const VolView& v, const ShapeRec64* __restrict__ tab, double px,
                                          double py, double pz, double qx, double qy, double qz, double& best,
                                          int& h) {
    const double p[3] = {px, py, pz}, q[3] = {qx, qy, qz};
    best = dist_in64(v.m64, p, q);
    h = -1;
    const double dd = qx * qx + qy * qy + qz * qz;
    const double dn = sqrt(dd);
    int i0, i1, i2, s0, s1, s2;
    double m0, m1, m2, e0, e1, e2;
    auto setup = [&](int k, int& ii, int& st, double& tm, double& te) {
        const int g = v.grid[k];
        ii = int(floor((p[k] - v.lo[k]) * v.inv_cell[k]));
        ii = ii < 0 ? 0 : (ii >= g ? g - 1 : ii);
        if (q[k] > 0.0) {
            st = 1;
            tm = (v.lo[k] + (ii + 1) * v.cell[k] - p[k]) / q[k];
            te = v.cell[k] / q[k];
        } else if (q[k] < 0.0) {
            st = -1;
            tm = (v.lo[k] + ii * v.cell[k] - p[k]) / q[k];
            te = -v.cell[k] / q[k];
        } else {
            st = 0;
            tm = d_inf();
            te = d_inf();
        }
    };
    setup(0, i0, s0, m0, e0);
    setup(1, i1, s1, m1, e1);
    setup(2, i2, s2, m2, e2);
    const int g0 = v.grid[0], g1 = v.grid[1], g2 = v.grid[2];
    int mb0 = -1, mb1 = -1, mb2 = -1, mb3 = -1;
    const int maxit = g0 + g1 + g2 + 3;
    for (int it = 0; it < maxit; ++it) {
        const int c = (i0 * g1 + i1) * g2 + i2;
        const int q1 = v.vox_off[c + 1];
        for (int e = v.vox_off[c]; e < q1; ++e) {
            const int j = v.vox_ids[e];
            if (j == mb0 || j == mb1 || j == mb2 || j == mb3) continue;
            mb3 = mb2; mb2 = mb1; mb1 = mb0; mb0 = j;
            const ShapeRec64& r = tab[j];
            const double w0 = r.t[0] - px, w1 = r.t[1] - py, w2 = r.t[2] - pz;
            const double proj = w0 * qx + w1 * qy + w2 * qz;
            const double rb = r.brad * dn;
            if (proj + rb < 0.0) continue;
            if (proj - rb > best * dd) continue;
            const double ww = w0 * w0 + w1 * w1 + w2 * w2;
            if (ww * dd - proj * proj > rb * rb) continue;
            double x[3], u[3];
            to_local64(r, px, py, pz, qx, qy, qz, x, u);
            const double s = dist_out64(r, x, u);
            if (LT(s, best) || (BITS(s) == BITS(best) && h >= 0 && j < h)) {
                best = s;
                h = j;
            }
        }
        // the cell is left at min(m0, m1, m2): nothing entered later can win
        const double mn = fmin(m0, fmin(m1, m2));
        if (best < mn * (1.0 - 9.094947017729282e-13)) break;
        if (m0 <= m1 && m0 <= m2) {
            i0 += s0;
            if (i0 < 0 || i0 >= g0) break;
            m0 += e0;
        } else if (m1 <= m2) {
            i1 += s1;
            if (i1 < 0 || i1 >= g1) break;
            m1 += e1;
        } else {
            i2 += s2;
            if (i2 < 0 || i2 >= g2) break;
            m2 += e2;
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
