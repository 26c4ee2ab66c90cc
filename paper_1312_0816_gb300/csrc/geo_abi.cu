// geo_abi.cu -- host side of the C ABI declared in include/geo.h: argument
// validation, the volume builder (device tables of Fig. 1's mother and
// daughter volumes), and dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "geo_internal.h"

using namespace geonav;

struct geo_volume_s {
    int device = 0;
    VolView view{};
    ShapeRec64* d64 = nullptr;
    ShapeRec32* d32 = nullptr;
    int32_t* vox_off = nullptr;
    int32_t* vox_ids = nullptr;
    unsigned int* status = nullptr;
    double* planes = nullptr;         // polycone plane tables (device)
    std::vector<ShapeRec64> h64;      // host copy of the daughter records
    std::vector<double> h_planes;     // host copy of the plane tables
    std::vector<int64_t> pl_off;      // [nd + 1]: table offset of daughter j (last: the mother), -1 if none
    // staging workspace of geo_dist_to_boundary_host: kStageBufs buffers of
    // ws_tracks tracks, a copy-in and a copy-out stream, and events
    static constexpr int kStageBufs = 3;
    void* ws = nullptr;
    int64_t ws_tracks = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr, s_k2 = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in[kStageBufs] = {}, ev_k[kStageBufs] = {}, ev_out[kStageBufs] = {},
                ev_join = nullptr;
    std::mutex ws_mu;
};

struct geo_batch_s {
    int device = 0;
    int32_t n_vols = 0;
    int blocks_per_sm = 0;
    int tile_tracks = kTileTracks;
    int64_t ntiles = 0;
    int64_t max_end = 0;
    int32_t segs = 0;
    int32_t vox = 0;            // a volume has a uniform grid
    int64_t* d_idx = nullptr;   // track indices of packed tiles
    VolView* d_vols = nullptr;
    BatchTile* d_tiles = nullptr;
    unsigned int* d_words = nullptr;   // [0] tile counter, [1] status
};

namespace {

constexpr double kEps32 = 5.9604644775390625e-08;  // 2^-24, unit roundoff of FP32
constexpr double kPi = 3.14159265358979323846;

int num_sms_of(int dev) {
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 152;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        cache[dev] = n;
    }
    return cache[dev];
}

// shared memory of one SM
int sm_smem(int dev) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || v <= 0)
        v = 100 * 1024;
    return v;
}

int smem_budget(int dev) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
        v = 48 * 1024;
    return v - 1024;   // static shared memory of the kernels (mbarrier etc.)
}

bool finite_all(const double* a, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// number of planes of a polycone (its p[2])
int pcon_nz(const geo_placed_shape& s) { return int(s.p[2]); }

// Shape parameter validation (readings of the ROOT conventions, see geo.h).
geo_status check_shape(const geo_placed_shape& s, bool is_mother) {
    if (s.kind < GEO_BOX || s.kind > GEO_PCON) return GEO_ERR_INVALID_ARG;
    if (s.reserved != 0) return GEO_ERR_INVALID_ARG;
    if (!finite_all(s.p, 5) || !finite_all(s.rot, 9) || !finite_all(s.trans, 3)) return GEO_ERR_SHAPE_PARAMS;
    const double* p = s.p;
    if (s.kind == GEO_PCON) {
        if (!s.planes || !(p[2] >= 2 && p[2] <= kMaxPlanes && p[2] == std::floor(p[2]))) return GEO_ERR_INVALID_ARG;
        const int n = pcon_nz(s);
        const double *z = s.planes, *rn = z + n, *rx = rn + n;
        if (!finite_all(s.planes, 3 * n) || p[3] != 0 || p[4] != 0 || !(p[1] > 0 && p[1] <= 2.0 * kPi))
            return GEO_ERR_SHAPE_PARAMS;
        for (int k = 0; k < n; ++k) {
            if (!(rn[k] >= 0 && rn[k] <= rx[k])) return GEO_ERR_SHAPE_PARAMS;
            if (k + 1 < n && !(z[k + 1] > z[k] && rx[k] + rx[k + 1] > 0)) return GEO_ERR_SHAPE_PARAMS;
        }
    }
    switch (s.kind) {
        case GEO_PCON:
            break;
        case GEO_BOX:
            if (!(p[0] > 0 && p[1] > 0 && p[2] > 0)) return GEO_ERR_SHAPE_PARAMS;
            break;
        case GEO_TUBE:
            if (!(p[2] > 0 && p[0] >= 0 && p[1] > 0 && p[0] <= p[1])) return GEO_ERR_SHAPE_PARAMS;
            break;
        case GEO_TUBS:
            if (!(p[2] > 0 && p[0] >= 0 && p[1] > 0 && p[0] <= p[1] && p[4] > 0 && p[4] <= 2.0 * kPi))
                return GEO_ERR_SHAPE_PARAMS;
            break;
        default:
            if (!(p[0] > 0 && p[1] >= 0 && p[3] >= 0 && p[1] <= p[2] && p[3] <= p[4] && p[2] + p[4] > 0))
                return GEO_ERR_SHAPE_PARAMS;
    }
    // rotation: orthonormal with det +1 within 1e-12
    const double* R = s.rot;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double d = R[3 * a] * R[3 * b] + R[3 * a + 1] * R[3 * b + 1] + R[3 * a + 2] * R[3 * b + 2];
            if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-12) return GEO_ERR_SHAPE_PARAMS;
        }
    const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                       R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (std::fabs(det - 1.0) > 1e-12) return GEO_ERR_SHAPE_PARAMS;
    if (is_mother) {
        for (int k = 0; k < 9; ++k)
            if (R[k] != ((k % 4 == 0) ? 1.0 : 0.0)) return GEO_ERR_INVALID_ARG;
        if (s.trans[0] != 0 || s.trans[1] != 0 || s.trans[2] != 0) return GEO_ERR_INVALID_ARG;
    }
    return GEO_OK;
}

double bounding_radius(const geo_placed_shape& s) {
    const double* p = s.p;
    if (s.kind == GEO_BOX) return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if (s.kind == GEO_PCON) {
        const int n = pcon_nz(s);
        double r = 0;
        for (int k = 0; k < n; ++k) r = std::max(r, std::hypot(s.planes[2 * n + k], s.planes[k]));
        return r;
    }
    if (s.kind == GEO_TUBE || s.kind == GEO_TUBS) return std::sqrt(p[1] * p[1] + p[2] * p[2]);
    const double r = std::max(p[2], p[4]);
    return std::sqrt(r * r + p[0] * p[0]);
}

// The tube bounding a polycone: radii from the least inner to the largest
// outer radius over its z-range; placed at the range's centre (centered ==
// false), or about the shape's own origin with a half-length covering both
// ends (centered == true, for a mother, whose FP32 copies are used in its
// own frame).
geo_placed_shape bounding_tube(const geo_placed_shape& s, bool centered) {
    const int n = pcon_nz(s);
    const double *z = s.planes, *rn = z + n, *rx = rn + n;
    geo_placed_shape t = s;
    t.kind = GEO_TUBE;
    t.planes = nullptr;
    double lo = rn[0], hi = rx[0];
    for (int k = 1; k < n; ++k) {
        lo = std::min(lo, rn[k]);
        hi = std::max(hi, rx[k]);
    }
    const double zc = 0.5 * (z[0] + z[n - 1]);
    t.p[0] = lo;
    t.p[1] = hi;
    t.p[2] = centered ? std::max(std::fabs(z[0]), std::fabs(z[n - 1])) : 0.5 * (z[n - 1] - z[0]);
    t.p[3] = t.p[4] = 0.0;
    if (!centered)
        for (int k = 0; k < 3; ++k) t.trans[k] = s.trans[k] + s.rot[3 * k + 2] * zc;
    return t;
}

// A tube inside a whole-turn polycone, about its origin: radii from the
// largest inner to the least outer radius (every section's radii lie between
// its planes' values), half-length the smaller distance from the origin to an
// end plane.  false when there is none (a wedge, the origin outside the
// z-range, or no common radius).
bool inscribed_tube(const geo_placed_shape& s, geo_placed_shape& t) {
    const int n = pcon_nz(s);
    const double *z = s.planes, *rn = z + n, *rx = rn + n;
    if (s.p[1] < 2.0 * kPi || !(z[0] < 0.0 && z[n - 1] > 0.0)) return false;
    double lo = rn[0], hi = rx[0];
    for (int k = 1; k < n; ++k) {
        lo = std::max(lo, rn[k]);
        hi = std::min(hi, rx[k]);
    }
    if (!(lo < hi)) return false;
    t = s;
    t.kind = GEO_TUBE;
    t.planes = nullptr;
    t.p[0] = lo;
    t.p[1] = hi;
    t.p[2] = std::min(-z[0], z[n - 1]);
    t.p[3] = t.p[4] = 0.0;
    return true;
}

// plane table of a polycone (layout in geo_internal.h)
std::vector<double> pcon_table_host(const geo_placed_shape& s) {
    const int n = pcon_nz(s);
    std::vector<double> T(size_t(pcon_table_len(n)));
    std::copy(s.planes, s.planes + 3 * n, T.begin());
    const double *z = s.planes, *rn = z + n, *rx = rn + n;
    for (int k = 0; k + 1 < n; ++k) {
        T[3 * n + k] = (rn[k + 1] - rn[k]) / (z[k + 1] - z[k]);
        T[3 * n + (n - 1) + k] = (rx[k + 1] - rx[k]) / (z[k + 1] - z[k]);
    }
    return T;
}

// derived FP64 constants (layout in geo_internal.h); table: the device
// address of a polycone's plane table
ShapeRec64 make_rec64(const geo_placed_shape& s, const double* table = nullptr) {
    ShapeRec64 r;
    std::memset(&r, 0, sizeof r);
    std::memcpy(r.R, s.rot, sizeof r.R);
    std::memcpy(r.t, s.trans, sizeof r.t);
    std::memcpy(r.p, s.p, sizeof r.p);
    r.kind = s.kind;
    bool eye = true;
    for (int k = 0; k < 9; ++k) eye = eye && s.rot[k] == ((k % 4) == 0 ? 1.0 : 0.0);
    r.flags = eye ? kRec64Identity : 0;
    const double* p = s.p;
    if (s.kind == GEO_BOX) {
        r.d[0] = p[0]; r.d[1] = p[1]; r.d[2] = p[2];
    } else if (s.kind == GEO_TUBE || s.kind == GEO_TUBS || s.kind == GEO_PCON) {
        double sphi = p[3], dphi = p[4];
        if (s.kind == GEO_PCON) {
            const int n = pcon_nz(s);
            const double *rn = s.planes + n, *rx = rn + n;
            const long long bits = static_cast<long long>(reinterpret_cast<uintptr_t>(table));
            std::memcpy(&r.d[0], &bits, sizeof bits);
            r.d[1] = n;
            r.d[2] = rn[0] * rn[0]; r.d[3] = rx[0] * rx[0];
            r.d[4] = rn[n - 1] * rn[n - 1]; r.d[12] = rx[n - 1] * rx[n - 1];
            sphi = p[0];
            dphi = p[1];
        } else {
            r.d[0] = p[0]; r.d[1] = p[1]; r.d[2] = p[2];
            r.d[3] = p[0] * p[0]; r.d[4] = p[1] * p[1];
        }
        if (s.kind != GEO_TUBE) {
            const double f1 = sphi, f2 = sphi + dphi;
            r.d[5] = -std::sin(f1); r.d[6] = std::cos(f1);   // n1: wedge side of the face at sphi
            r.d[7] = std::sin(f2);  r.d[8] = -std::cos(f2);  // n2: wedge side of the face at sphi + dphi
            r.d[9] = dphi <= kPi ? 1.0 : 0.0;                // the wedge is n1 >= 0 AND n2 >= 0
            r.d[10] = dphi < 2.0 * kPi ? 0.0 : 1.0;          // a whole turn: no wedge
            r.d[11] = dphi == kPi ? 1.0 : 0.0;               // a half turn: the two planes coincide
        }
    } else {
        const double dz = p[0];
        r.d[0] = dz;
        r.d[1] = 0.5 * (p[2] + p[4]);
        r.d[2] = (p[4] - p[2]) / (2.0 * dz);
        r.d[3] = 0.5 * (p[1] + p[3]);
        r.d[4] = (p[3] - p[1]) / (2.0 * dz);
        r.d[5] = p[1] * p[1]; r.d[6] = p[2] * p[2]; r.d[7] = p[3] * p[3]; r.d[8] = p[4] * p[4];
        r.d[9] = 1.0 / std::sqrt(1.0 + r.d[2] * r.d[2]);
        r.d[10] = 1.0 / std::sqrt(1.0 + r.d[4] * r.d[4]);
        r.d[11] = (p[1] > 0.0 || p[3] > 0.0) ? 1.0 : 0.0;
    }
    const double br = bounding_radius(s);
    r.brad = br * (1.0 + 1e-12) + 1e-9;
    return r;
}

// FP32 record of a solid grown (grow > 0) or shrunk (grow < 0) by |grow| mm.
// Returns false when a shrunk solid degenerates.  A polycone is bounded by its
// tube (centered: about its origin, for a mother).
// The float nearest x from above / below.
float float_up(double x) {
    const float f = float(x);
    return double(f) < x ? std::nextafter(f, HUGE_VALF) : f;
}
float float_down(double x) {
    const float f = float(x);
    return double(f) > x ? std::nextafter(f, -HUGE_VALF) : f;
}

bool make_rec32(const geo_placed_shape& s, double grow, double delta, ShapeRec32& r, bool centered = false) {
    if (s.kind == GEO_PCON && grow >= 0) return make_rec32(bounding_tube(s, centered), grow, delta, r);
    geo_placed_shape in;
    // a shrunk polycone: its inscribed tube shrunk (when that survives)
    if (s.kind == GEO_PCON && inscribed_tube(s, in) && make_rec32(in, grow, delta, r)) return true;
    std::memset(&r, 0, sizeof r);
    for (int k = 0; k < 9; ++k) r.R[k] = float(s.rot[k]);
    bool eye = true;
    for (int k = 0; k < 9; ++k) eye = eye && s.rot[k] == ((k % 4) == 0 ? 1.0 : 0.0);
    r.flags = eye ? kRec32Identity : 0;
    for (int k = 0; k < 3; ++k) r.t[k] = float(s.trans[k]);
    r.kind = s.kind;
    r.delta = float(delta);
    const double* p = s.p;
    const double g = grow;
    if (s.kind == GEO_BOX) {
        for (int k = 0; k < 3; ++k) {
            r.e[k] = float(p[k] + g);
            if (!(p[k] + g > 0)) return false;
        }
    } else if ((s.kind == GEO_TUBS || s.kind == GEO_PCON) && g < 0) {
        // a shrunk whole tube is no subset of a segment (nor of a polycone
        // without an inscribed tube): an empty solid, so the filter never
        // decides "surely inside" there
        r.kind = GEO_TUBE;
        r.e[0] = 0.f; r.e[1] = -1.f; r.e[2] = -1.f; r.e[3] = 0.f;
    } else if (s.kind == GEO_TUBE || s.kind == GEO_TUBS) {
        // a segment is bounded by its whole tube (superset: valid lower bounds)
        r.kind = GEO_TUBE;
        const double rmin = p[0] - g, rmax = p[1] + g, dz = p[2] + g;
        if (!(rmax > 0 && dz > 0)) return false;
        const bool hole = p[0] > 0 && rmin > 0;
        r.e[0] = hole ? float(rmin * rmin) : 0.f;
        r.e[1] = float(rmax * rmax);
        r.e[2] = float(dz);
        r.e[3] = hole ? 1.f : 0.f;
        // acceptance limits of the filter's crossings, lenient by delta
        const double ro = rmax + delta, ri = rmin - delta;
        r.e[4] = float_up(ro * ro);
        r.e[5] = hole && ri > 0 ? float_down(ri * ri) : 0.f;
        r.e[6] = float_up(dz + delta);
    } else {
        const double dz = p[0], dzg = dz + g;
        if (!(dzg > 0)) return false;
        const double ao = 0.5 * (p[2] + p[4]), bo = (p[4] - p[2]) / (2.0 * dz);
        const double ai = 0.5 * (p[1] + p[3]), bi = (p[3] - p[1]) / (2.0 * dz);
        // offset the supporting lines of the slanted edges by g along their normals
        const double ao2 = ao + g * std::sqrt(1.0 + bo * bo);
        const double ai2 = ai - g * std::sqrt(1.0 + bi * bi);
        const double o_lo = ao2 - bo * dzg, o_hi = ao2 + bo * dzg;
        const double i_lo = ai2 - bi * dzg, i_hi = ai2 + bi * dzg;
        if (!(std::max(o_lo, o_hi) > 0)) return false;
        const bool hole = (p[1] > 0 || p[3] > 0) && i_lo > 0 && i_hi > 0;
        r.e[0] = float(dzg);
        r.e[1] = float(ao2);
        r.e[2] = float(bo);
        r.e[3] = hole ? float(ai2) : 0.f;
        r.e[4] = hole ? float(bi) : 0.f;
        r.e[5] = hole ? 1.f : 0.f;
        const double olo = std::max(o_lo, 0.0), ohi = std::max(o_hi, 0.0);
        r.e[6] = hole ? float(i_lo * i_lo) : 0.f;
        r.e[7] = float(olo * olo);
        r.e[8] = hole ? float(i_hi * i_hi) : 0.f;
        r.e[9] = float(ohi * ohi);
        // acceptance limits of the filter's end-plane crossings, lenient by delta
        r.e[10] = float_up((olo + delta) * (olo + delta));
        r.e[11] = float_up((ohi + delta) * (ohi + delta));
        const double ilo = hole ? i_lo - delta : 0.0, ihi = hole ? i_hi - delta : 0.0;
        r.e[12] = ilo > 0 ? float_down(ilo * ilo) : 0.f;
        r.e[13] = ihi > 0 ? float_down(ihi * ihi) : 0.f;
        r.e[14] = float_up(dzg + delta);
    }
    r.brad = float(bounding_radius(s) * (1.0 + 1e-6) + std::max(g, 0.0));
    r.brad2 = float_up(double(r.brad) * double(r.brad));
    return true;
}

// Extent of the mother: an upper bound of |p| for every point inside it.
double mother_scale(const geo_placed_shape& m) { return bounding_radius(m); }

// Inflation of one solid's FP32 copy (mm).  It covers the FP32 rounding of
//  - the inputs and the master->local transform, for positions up to the
//    mother scale S:                               48 eps32 S
//  - the shape arithmetic in the frame shifted to the closest approach
//    (magnitudes up to the bounding radius brad):  16 eps32 brad
//  - for a quadric of radius r and slope b, the rounding of its discriminant
//    expressed as a change of radius:              16 eps32 brad^2 (1+b^2) / r
//    with r taken no smaller than sqrt(eps32) brad / 2 (apexes, tiny holes).
double inflation(const geo_placed_shape& s, double S) {
    if (s.kind == GEO_PCON) return inflation(bounding_tube(s, false), S);
    const double br = bounding_radius(s);
    const double* p = s.p;
    double d = kEps32 * (48.0 * S + 16.0 * br);
    if (s.kind == GEO_BOX) return d;
    double rsmall = DBL_MAX, slope2 = 0.0;
    auto take = [&](double r) { rsmall = std::min(rsmall, r > 0 ? r : 0.0); };
    if (s.kind == GEO_TUBE || s.kind == GEO_TUBS) {
        take(p[1]);
        if (p[0] > 0) take(p[0]);
    } else {
        take(p[2]);
        take(p[4]);
        if (p[1] > 0 || p[3] > 0) {
            take(p[1]);
            take(p[3]);
        }
        const double bo = (p[4] - p[2]) / (2.0 * p[0]), bi = (p[3] - p[1]) / (2.0 * p[0]);
        slope2 = std::max(bo * bo, bi * bi);
    }
    const double floor_r = 0.5 * std::sqrt(kEps32) * br;
    d += 16.0 * kEps32 * br * br * (1.0 + slope2) / std::max(rsmall, floor_r);
    return d;
}

// A solid whose routines live in the kernels' second instantiation: tube
// segments, polycones, and cones with a zero radius at an end plane (an apex
// there, whose crossings are formed about it).
bool needs_segs_code(const geo_placed_shape& s) {
    if (s.kind == GEO_TUBS || s.kind == GEO_PCON) return true;
    if (s.kind != GEO_CONE) return false;
    const double* p = s.p;
    const bool hole = p[1] > 0.0 || p[3] > 0.0;
    return p[2] == 0.0 || p[4] == 0.0 || (hole && (p[1] == 0.0 || p[3] == 0.0));
}

geo_status cuda_status(cudaError_t e);

// Uniform grid over the mother's bounding box; every cell lists (CSR) the
// daughters whose world bounding box, grown by their FP32 inflation and by
// 1e-3 of a cell, overlaps it.  The growth keeps the lists conservative for
// an FP32 grid walk whose rounding can cut a corner between two cells.
geo_status build_voxels(const geo_placed_shape& m, const geo_placed_shape* d, int nd, double S,
                        const geo_build_opts* opts, cudaStream_t s, geo_volume v) {
    double half[3];
    const geo_placed_shape mb = m.kind == GEO_PCON ? bounding_tube(m, true) : m;
    const double* p = mb.p;
    if (mb.kind == GEO_BOX) { half[0] = p[0]; half[1] = p[1]; half[2] = p[2]; }
    else if (mb.kind == GEO_TUBE || mb.kind == GEO_TUBS) { half[0] = half[1] = p[1]; half[2] = p[2]; }
    else { half[0] = half[1] = std::max(p[2], p[4]); half[2] = p[0]; }
    int g[3];
    const int gauto = std::max(1, std::min(64, int(std::lround(2.0 * std::cbrt(double(std::max(nd, 1)))))));
    for (int k = 0; k < 3; ++k) g[k] = opts->grid[k] > 0 ? opts->grid[k] : gauto;
    const int64_t ncells = int64_t(g[0]) * g[1] * g[2];
    if (ncells > (int64_t(1) << 24)) return GEO_ERR_INVALID_ARG;
    VolView& vw = v->view;
    for (int k = 0; k < 3; ++k) {
        vw.grid[k] = g[k];
        vw.lo[k] = -half[k];
        vw.cell[k] = 2.0 * half[k] / g[k];
        vw.inv_cell[k] = 1.0 / vw.cell[k];
    }
    std::vector<std::vector<int32_t>> lists(static_cast<size_t>(ncells));
    for (int j = 0; j < nd; ++j) {
        const geo_placed_shape sh = d[j].kind == GEO_PCON ? bounding_tube(d[j], false) : d[j];
        double he[3];
        const double* q = sh.p;
        if (sh.kind == GEO_BOX) { he[0] = q[0]; he[1] = q[1]; he[2] = q[2]; }
        else if (sh.kind == GEO_TUBE || sh.kind == GEO_TUBS) { he[0] = he[1] = q[1]; he[2] = q[2]; }
        else { he[0] = he[1] = std::max(q[2], q[4]); he[2] = q[0]; }
        int i0[3], i1[3];
        for (int k = 0; k < 3; ++k) {
            const double ext = std::fabs(sh.rot[3 * k]) * he[0] + std::fabs(sh.rot[3 * k + 1]) * he[1] +
                               std::fabs(sh.rot[3 * k + 2]) * he[2];
            const double grow = inflation(sh, S) + 1e-3 * vw.cell[k] + 1e-9 * (1.0 + std::fabs(sh.trans[k]));
            const double a = (sh.trans[k] - ext - grow - vw.lo[k]) * vw.inv_cell[k];
            const double b = (sh.trans[k] + ext + grow - vw.lo[k]) * vw.inv_cell[k];
            i0[k] = int(std::max(0.0, std::min(double(g[k] - 1), std::floor(a))));
            i1[k] = int(std::max(0.0, std::min(double(g[k] - 1), std::floor(b))));
        }
        for (int a = i0[0]; a <= i1[0]; ++a)
            for (int b = i0[1]; b <= i1[1]; ++b)
                for (int c = i0[2]; c <= i1[2]; ++c) lists[(size_t(a) * g[1] + b) * g[2] + c].push_back(j);
    }
    std::vector<int32_t> off(static_cast<size_t>(ncells) + 1, 0), ids;
    for (int64_t c = 0; c < ncells; ++c) {
        off[c + 1] = off[c] + int32_t(lists[c].size());
        ids.insert(ids.end(), lists[c].begin(), lists[c].end());
    }
    if (ids.empty()) ids.push_back(0);
    cudaError_t e;
    if ((e = lib_malloc(&v->vox_off, sizeof(int32_t) * off.size())) != cudaSuccess ||
        (e = lib_malloc(&v->vox_ids, sizeof(int32_t) * ids.size())) != cudaSuccess ||
        (e = cudaMemcpyAsync(v->vox_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(v->vox_ids, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_status(e);
    vw.vox_off = v->vox_off;
    vw.vox_ids = v->vox_ids;
    vw.voxelized = 1;
    return GEO_OK;
}

geo_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GEO_OK;
    if (e == cudaErrorMemoryAllocation) return GEO_ERR_OOM;
    return GEO_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (cudaHostAlloc,
// cudaHostRegister), which kernels can read and write in place over the host
// link; nullptr for pageable memory.
const void* mapped_host_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

geo_status check_volume_device(geo_volume v) {
    if (!v) return GEO_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    return dev == v->device ? GEO_OK : GEO_ERR_INVALID_ARG;
}

geo_status check_basket(const double* x, const double* y, const double* z, int64_t n) {
    if (n < 0) return GEO_ERR_INVALID_ARG;
    if (n == 0) return GEO_OK;
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(z)) return GEO_ERR_INVALID_ARG;
    return GEO_OK;
}

// Reads and clears the device status word of earlier kernels (asynchronous
// copy would be ideal; a tiny synchronous read keeps the ABI simple and is
// only done in checked mode).
}  // namespace

namespace geonav {
const VolView* volume_view(geo_volume v) { return v ? &v->view : nullptr; }
const ShapeRec64* volume_host_daughters(geo_volume v) { return v ? v->h64.data() : nullptr; }
const double* volume_host_table(geo_volume v, int j) {
    if (!v || j < -1 || j >= v->view.nd) return nullptr;
    const int64_t o = v->pl_off[j < 0 ? size_t(v->view.nd) : size_t(j)];
    return o >= 0 ? v->h_planes.data() + o : nullptr;
}
int volume_device(geo_volume v) { return v ? v->device : -1; }
int sm_count(int device) { return num_sms_of(device); }

// geo_debug_fail_alloc: > 0 counts down the allocations; the one that brings
// it to zero fails
static std::atomic<int> g_fail_alloc{0};
bool lib_alloc_fails() {
    int n = g_fail_alloc.load();
    while (n > 0)
        if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 1;
    return false;
}
cudaError_t lib_malloc_raw(void** p, size_t bytes) {
    if (lib_alloc_fails()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
}  // namespace geonav

extern "C" {

const char* geo_status_string(geo_status s) {
    switch (s) {
        case GEO_OK: return "ok";
        case GEO_ERR_INVALID_ARG: return "invalid argument";
        case GEO_ERR_SHAPE_PARAMS: return "invalid shape parameters or placement";
        case GEO_ERR_OOM: return "device allocation failed";
        case GEO_ERR_CUDA: return "CUDA runtime error";
        case GEO_ERR_DEVICE_ASSERT: return "device-side check failed";
        case GEO_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

geo_status geo_build_volume(const geo_placed_shape* mother, const geo_placed_shape* daughters, int32_t n_daughters,
                            const geo_build_opts* opts, void* stream, geo_volume* out) {
    if (!out) return GEO_ERR_INVALID_ARG;
    *out = nullptr;
    if (!mother || n_daughters < 0 || (n_daughters > 0 && !daughters)) return GEO_ERR_INVALID_ARG;
    if (n_daughters > (1 << 20)) return GEO_ERR_INVALID_ARG;
    geo_status st = check_shape(*mother, true);
    if (st != GEO_OK) return st;
    for (int j = 0; j < n_daughters; ++j)
        if ((st = check_shape(daughters[j], false)) != GEO_OK) return st;
    if (opts && opts->voxelize) {
        for (int k = 0; k < 3; ++k)
            if (opts->grid[k] < 0 || opts->grid[k] > 256) return GEO_ERR_INVALID_ARG;
    }

    geo_volume v = lib_new<geo_volume_s>();
    if (!v) return GEO_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        delete v;
        return GEO_ERR_CUDA;
    }

    const double S = mother_scale(*mother);
    v->device = dev;
    // the polycones' plane tables, daughters first, then the mother
    v->pl_off.assign(size_t(n_daughters) + 1, -1);
    for (int j = 0; j <= n_daughters; ++j) {
        const geo_placed_shape& sh = j < n_daughters ? daughters[j] : *mother;
        if (sh.kind != GEO_PCON) continue;
        v->pl_off[j] = int64_t(v->h_planes.size());
        const std::vector<double> T = pcon_table_host(sh);
        v->h_planes.insert(v->h_planes.end(), T.begin(), T.end());
    }
    cudaError_t e = cudaSuccess;
    if (!v->h_planes.empty() && (e = lib_malloc(&v->planes, sizeof(double) * v->h_planes.size())) != cudaSuccess) {
        delete v;
        return cuda_status(e);
    }
    auto table_of = [&](int j) { return v->pl_off[j] >= 0 ? v->planes + v->pl_off[j] : nullptr; };

    std::vector<ShapeRec64> h64(n_daughters);
    std::vector<ShapeRec32> h32(n_daughters);
    for (int j = 0; j < n_daughters; ++j) {
        h64[j] = make_rec64(daughters[j], table_of(j));
        const double dl = inflation(daughters[j], S);
        if (!make_rec32(daughters[j], dl, dl, h32[j])) {
            geo_destroy_volume(v);
            return GEO_ERR_SHAPE_PARAMS;
        }
    }
    VolView& vw = v->view;
    std::memset(&vw, 0, sizeof vw);
    vw.m64 = make_rec64(*mother, table_of(n_daughters));
    const double dm = inflation(*mother, S);
    if (!make_rec32(*mother, -dm, dm, vw.m32) || !make_rec32(*mother, dm, dm, vw.m32u, true)) {
        geo_destroy_volume(v);
        return GEO_ERR_SHAPE_PARAMS;
    }
    vw.nd = n_daughters;
    // the kernels' instantiation with the out-of-line code of tube segments,
    // polycones and cones through an apex on an end plane
    vw.segs = needs_segs_code(*mother) ? 1 : 0;
    for (int j = 0; j < n_daughters; ++j)
        if (needs_segs_code(daughters[j])) vw.segs = 1;

    const size_t b64 = sizeof(ShapeRec64) * size_t(std::max(n_daughters, 1));
    const size_t b32 = sizeof(ShapeRec32) * size_t(std::max(n_daughters, 1));
    if ((e = lib_malloc(&v->d64, b64)) != cudaSuccess || (e = lib_malloc(&v->d32, b32)) != cudaSuccess ||
        (e = lib_malloc(&v->status, sizeof(unsigned int))) != cudaSuccess) {
        geo_destroy_volume(v);
        return cuda_status(e);
    }
    if (!v->h_planes.empty() &&
        (e = cudaMemcpyAsync(v->planes, v->h_planes.data(), sizeof(double) * v->h_planes.size(),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        geo_destroy_volume(v);
        return cuda_status(e);
    }
    if (n_daughters > 0) {
        if ((e = cudaMemcpyAsync(v->d64, h64.data(), sizeof(ShapeRec64) * n_daughters, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(v->d32, h32.data(), sizeof(ShapeRec32) * n_daughters, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess) {
            geo_destroy_volume(v);
            return cuda_status(e);
        }
    }
    if ((e = cudaMemsetAsync(v->status, 0, sizeof(unsigned int), s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        geo_destroy_volume(v);
        return cuda_status(e);
    }
    vw.d64 = v->d64;
    vw.d32 = v->d32;
    vw.status = v->status;
    v->h64 = std::move(h64);
    if (opts && opts->voxelize) {
        st = build_voxels(*mother, daughters, n_daughters, S, opts, s, v);
        if (st != GEO_OK) {
            geo_destroy_volume(v);
            return st;
        }
    }
    vw.smem64 = (int64_t(n_daughters) * int64_t(sizeof(ShapeRec64)) <= smem_budget(dev)) ? 1 : 0;
    // the refine kernel wants two blocks per SM: its staged tables get what
    // half of an SM's shared memory leaves beside its two stage buffers (less
    // the per-block reservation and static shared memory); larger tables are
    // read through L1 from global memory
    const int64_t stages = int64_t(refine_stage_bytes());
    vw.smem_refine = (int64_t(n_daughters) * int64_t(sizeof(ShapeRec64) + sizeof(ShapeRec32)) <=
                      std::min(int64_t(smem_budget(dev)) - stages, int64_t(sm_smem(dev)) / 2 - 2048 - stages))
                         ? 1
                         : 0;
    *out = v;
    return GEO_OK;
}

geo_status geo_destroy_volume(geo_volume v) {
    if (!v) return GEO_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != v->device) cudaSetDevice(v->device);
    cudaDeviceSynchronize();
    cudaFree(v->d64);
    cudaFree(v->d32);
    cudaFree(v->planes);
    cudaFree(v->vox_off);
    cudaFree(v->vox_ids);
    cudaFree(v->status);
    cudaFree(v->ws);
    if (v->s_in) cudaStreamDestroy(v->s_in);
    if (v->s_out) cudaStreamDestroy(v->s_out);
    if (v->s_k2) cudaStreamDestroy(v->s_k2);
    for (cudaEvent_t e : {v->ev_start, v->ev_join})
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < geo_volume_s::kStageBufs; ++k)
        for (cudaEvent_t e : {v->ev_in[k], v->ev_k[k], v->ev_out[k]})
            if (e) cudaEventDestroy(e);
    if (prev >= 0 && prev != v->device) cudaSetDevice(prev);
    delete v;
    return GEO_OK;
}

geo_status geo_volume_info(geo_volume v, int32_t* n_daughters, int32_t* voxelized, int32_t grid[3]) {
    if (!v) return GEO_ERR_INVALID_ARG;
    if (n_daughters) *n_daughters = v->view.nd;
    if (voxelized) *voxelized = v->view.voxelized;
    if (grid)
        for (int k = 0; k < 3; ++k) grid[k] = v->view.grid[k];
    return GEO_OK;
}

geo_status geo_dist_to_boundary(geo_volume v, const double* x, const double* y, const double* z, const double* dx,
                                const double* dy, const double* dz, int64_t n, double* step, int32_t* hit,
                                double* bpoint, int32_t mode, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if (mode != GEO_FP64 && mode != GEO_FP32_REFINE) return GEO_ERR_INVALID_ARG;
    if ((st = check_basket(x, y, z, n)) != GEO_OK) return st;
    if (n == 0) return GEO_OK;
    if (!is_device_ptr(dx) || !is_device_ptr(dy) || !is_device_ptr(dz) || !is_device_ptr(step) ||
        !is_device_ptr(hit) || (bpoint && !is_device_ptr(bpoint)))
        return GEO_ERR_INVALID_ARG;
    const Basket b{x, y, z, dx, dy, dz, n};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = num_sms_of(v->device);
    cudaError_t e = (mode == GEO_FP64) ? launch_dist_fp64(v->view, b, step, hit, bpoint, s, sms)
                                       : launch_dist_refine(v->view, b, step, hit, bpoint, s, sms);
    return cuda_status(e);
}

geo_status geo_contains(geo_volume v, const double* x, const double* y, const double* z, int64_t n, int32_t* where,
                        int32_t mode, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if (mode != GEO_FP64 && mode != GEO_FP32_REFINE) return GEO_ERR_INVALID_ARG;
    if ((st = check_basket(x, y, z, n)) != GEO_OK) return st;
    if (n == 0) return GEO_OK;
    if (!is_device_ptr(where)) return GEO_ERR_INVALID_ARG;
    const Basket b{x, y, z, nullptr, nullptr, nullptr, n};
    return cuda_status(launch_contains(v->view, b, where, mode, static_cast<cudaStream_t>(stream),
                                       num_sms_of(v->device)));
}

geo_status geo_safety(geo_volume v, const double* x, const double* y, const double* z, int64_t n, double* safety,
                      int32_t mode, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if (mode != GEO_FP64 && mode != GEO_FP32_REFINE && mode != GEO_SAFETY_ESTIMATE) return GEO_ERR_INVALID_ARG;
    if ((st = check_basket(x, y, z, n)) != GEO_OK) return st;
    if (n == 0) return GEO_OK;
    if (!is_device_ptr(safety)) return GEO_ERR_INVALID_ARG;
    const Basket b{x, y, z, nullptr, nullptr, nullptr, n};
    return cuda_status(
        launch_safety(v->view, b, safety, mode, static_cast<cudaStream_t>(stream), num_sms_of(v->device)));
}

geo_status geo_dist_to_boundary_host(geo_volume v, const double* x, const double* y, const double* z, const double* dx,
                                     const double* dy, const double* dz, int64_t n, double* step, int32_t* hit,
                                     int32_t mode, int64_t chunk, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if (mode != GEO_FP64 && mode != GEO_FP32_REFINE) return GEO_ERR_INVALID_ARG;
    if (n < 0 || chunk < 0) return GEO_ERR_INVALID_ARG;
    if (n == 0) return GEO_OK;
    if (!x || !y || !z || !dx || !dy || !dz || !step || !hit) return GEO_ERR_INVALID_ARG;
    const void* hp[8] = {x, y, z, dx, dy, dz, step, hit};
    const void* mp[8];
    bool mapped = true;
    for (int k = 0; k < 8; ++k) {
        if (is_device_ptr(hp[k])) return GEO_ERR_INVALID_ARG;
        mp[k] = mapped_host_ptr(hp[k]);
        mapped = mapped && mp[k] != nullptr;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = num_sms_of(v->device);
    cudaError_t e = cudaSuccess;
    if (mapped) {
        // every array page-locked: one step over the arrays in place (the
        // kernel's loads and stores cross the host link; no staging copies)
        const Basket b{static_cast<const double*>(mp[0]), static_cast<const double*>(mp[1]),
                       static_cast<const double*>(mp[2]), static_cast<const double*>(mp[3]),
                       static_cast<const double*>(mp[4]), static_cast<const double*>(mp[5]), n};
        double* ostep = const_cast<double*>(static_cast<const double*>(mp[6]));
        int32_t* ohit = const_cast<int32_t*>(static_cast<const int32_t*>(mp[7]));
        e = (mode == GEO_FP64) ? launch_dist_fp64(v->view, b, ostep, ohit, nullptr, s, sms)
                               : launch_dist_refine(v->view, b, ostep, ohit, nullptr, s, sms);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? GEO_OK : cuda_status(e);
    }
    if (chunk == 0) chunk = int64_t(1) << 18;
    if (chunk > n) chunk = n;
    std::lock_guard<std::mutex> lock(v->ws_mu);
    if (!v->s_in) {
        if ((e = cudaStreamCreateWithFlags(&v->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&v->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&v->s_k2, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_status(e);
        std::vector<cudaEvent_t*> evs = {&v->ev_start, &v->ev_join};
        for (int k = 0; k < geo_volume_s::kStageBufs; ++k) {
            evs.push_back(&v->ev_in[k]);
            evs.push_back(&v->ev_k[k]);
            evs.push_back(&v->ev_out[k]);
        }
        for (cudaEvent_t* ev : evs)
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
    }
    const size_t per_track = 7 * sizeof(double) + sizeof(int32_t);
    if (v->ws_tracks < chunk) {
        if (v->ws) {
            cudaFree(v->ws);
            v->ws = nullptr;
            v->ws_tracks = 0;
        }
        if ((e = lib_malloc(&v->ws, geo_volume_s::kStageBufs * size_t(chunk) * per_track)) != cudaSuccess)
            return cuda_status(e);
        v->ws_tracks = chunk;
    }
    const int64_t cap = v->ws_tracks;
    constexpr int NB = geo_volume_s::kStageBufs;
    double* f[NB][7];
    int32_t* whit[NB];
    for (int bfr = 0; bfr < NB; ++bfr) {
        double* w = reinterpret_cast<double*>(static_cast<char*>(v->ws) + bfr * size_t(cap) * per_track);
        for (int k = 0; k < 7; ++k) f[bfr][k] = w + k * cap;
        whit[bfr] = reinterpret_cast<int32_t*>(w + 7 * cap);
    }
    const double* src[6] = {x, y, z, dx, dy, dz};
    // three-stage pipeline over chunks and NB buffers: copy in (s_in), the
    // step, copy out (s_out); chunk c+1 is copied in while chunk c is stepped
    // and chunk c-1 copied out, and a buffer is refilled once its chunk has
    // been copied out (with three buffers the copy-in of chunk c+2 need not
    // wait for the step of chunk c).  The steps of even chunks run on the
    // caller's stream and those of odd chunks on a second internal stream, so
    // that a chunk's kernel can start on the SMs the previous one is leaving
    // (its tail) instead of waiting for it.
    if ((e = cudaEventRecord(v->ev_start, s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(v->s_in, v->ev_start, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(v->s_k2, v->ev_start, 0)) != cudaSuccess)
        return cuda_status(e);
    int64_t c = 0;
    for (int64_t off = 0; off < n; off += chunk, ++c) {
        const int bf = int(c % NB);
        const cudaStream_t ks = (c & 1) ? v->s_k2 : s;
        const int64_t m = std::min(chunk, n - off);
        if (c >= NB && (e = cudaStreamWaitEvent(v->s_in, v->ev_out[bf], 0)) != cudaSuccess) return cuda_status(e);
        for (int k = 0; k < 6; ++k)
            if ((e = cudaMemcpyAsync(f[bf][k], src[k] + off, size_t(m) * sizeof(double), cudaMemcpyHostToDevice,
                                     v->s_in)) != cudaSuccess)
                return cuda_status(e);
        if ((e = cudaEventRecord(v->ev_in[bf], v->s_in)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ks, v->ev_in[bf], 0)) != cudaSuccess)
            return cuda_status(e);
        const Basket b{f[bf][0], f[bf][1], f[bf][2], f[bf][3], f[bf][4], f[bf][5], m};
        e = (mode == GEO_FP64) ? launch_dist_fp64(v->view, b, f[bf][6], whit[bf], nullptr, ks, sms)
                               : launch_dist_refine(v->view, b, f[bf][6], whit[bf], nullptr, ks, sms);
        if (e != cudaSuccess) return cuda_status(e);
        if ((e = cudaEventRecord(v->ev_k[bf], ks)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(v->s_out, v->ev_k[bf], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(step + off, f[bf][6], size_t(m) * sizeof(double), cudaMemcpyDeviceToHost,
                                 v->s_out)) != cudaSuccess ||
            (e = cudaMemcpyAsync(hit + off, whit[bf], size_t(m) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 v->s_out)) != cudaSuccess ||
            (e = cudaEventRecord(v->ev_out[bf], v->s_out)) != cudaSuccess)
            return cuda_status(e);
    }
    // the caller's stream follows the whole call (the second stream joined)
    if ((e = cudaEventRecord(v->ev_join, v->s_k2)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, v->ev_join, 0)) != cudaSuccess ||
        (e = cudaStreamSynchronize(v->s_out)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_status(e);
    return GEO_OK;
}

geo_status geo_build_batch(const geo_volume* vols, int32_t n_vols, const geo_basket* baskets, int32_t n_baskets,
                           const geo_batch_opts* opts, void* stream, geo_batch* out) {
    if (!out) return GEO_ERR_INVALID_ARG;
    *out = nullptr;
    if (!vols || n_vols <= 0 || n_baskets < 0 || (n_baskets > 0 && !baskets)) return GEO_ERR_INVALID_ARG;
    const int order = opts ? opts->tile_order : 0;
    const int bps = opts ? opts->blocks_per_sm : 0;
    const int T = (opts && opts->tile_tracks != 0) ? opts->tile_tracks : kTileTracks;
    if ((order != 0 && order != 1) || bps < 0 || (T != kTileTracks && T != 256)) return GEO_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    for (int i = 0; i < n_vols; ++i)
        if (!vols[i] || vols[i]->device != dev) return GEO_ERR_INVALID_ARG;
    // Every basket's full T-track stretches become tiles of
    // consecutive tracks; the ragged tails of a volume's baskets are
    // gathered, in basket order, into packed tiles that list their tracks'
    // indices, so that baskets of a few tracks still fill the producer
    // threads.
    std::vector<BatchTile> tiles;
    std::vector<int64_t> cost;
    std::vector<std::vector<int64_t>> tails(static_cast<size_t>(n_vols));
    int64_t max_end = 0;
    for (int k = 0; k < n_baskets; ++k) {
        const geo_basket& bk = baskets[k];
        if (bk.reserved != 0 || bk.volume < 0 || bk.volume >= n_vols || bk.offset < 0 || bk.count < 0)
            return GEO_ERR_INVALID_ARG;
        max_end = std::max(max_end, bk.offset + bk.count);
        const int64_t full = bk.count / T * T;
        for (int64_t off = 0; off < full; off += T) {
            BatchTile t;
            t.vol = bk.volume;
            t.count = T;
            t.base = bk.offset + off;
            tiles.push_back(t);
            cost.push_back(int64_t(T) * (vols[bk.volume]->view.nd + 1));
        }
        for (int64_t q = bk.offset + full; q < bk.offset + bk.count; ++q) tails[size_t(bk.volume)].push_back(q);
    }
    std::vector<int64_t> idx;
    for (int v = 0; v < n_vols; ++v) {
        const std::vector<int64_t>& tv = tails[size_t(v)];
        for (size_t a = 0; a < tv.size(); a += size_t(T)) {
            const size_t m = std::min<size_t>(size_t(T), tv.size() - a);
            BatchTile t;
            t.vol = v;
            t.count = -int32_t(m);
            t.base = int64_t(idx.size());
            idx.insert(idx.end(), tv.begin() + std::ptrdiff_t(a), tv.begin() + std::ptrdiff_t(a + m));
            tiles.push_back(t);
            cost.push_back(int64_t(m) * (vols[v]->view.nd + 1));
        }
    }
    if (order == 0) {
        std::vector<size_t> idx(tiles.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
        std::vector<BatchTile> sorted(tiles.size());
        for (size_t i = 0; i < idx.size(); ++i) sorted[i] = tiles[idx[i]];
        tiles.swap(sorted);
    }
    std::vector<VolView> views(n_vols);
    for (int i = 0; i < n_vols; ++i) views[i] = vols[i]->view;
    geo_batch b = lib_new<geo_batch_s>();
    if (!b) return GEO_ERR_OOM;
    b->device = dev;
    b->n_vols = n_vols;
    b->blocks_per_sm = bps;
    b->tile_tracks = T;
    b->ntiles = int64_t(tiles.size());
    b->max_end = max_end;
    for (int i = 0; i < n_vols; ++i) {
        b->segs = b->segs || vols[i]->view.segs;
        b->vox = b->vox || vols[i]->view.voxelized;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = lib_malloc(&b->d_vols, sizeof(VolView) * n_vols)) != cudaSuccess ||
        (e = lib_malloc(&b->d_tiles, sizeof(BatchTile) * std::max<size_t>(tiles.size(), 1))) != cudaSuccess ||
        (e = lib_malloc(&b->d_words, 2 * sizeof(unsigned int))) != cudaSuccess ||
        (!idx.empty() && (e = lib_malloc(&b->d_idx, sizeof(int64_t) * idx.size())) != cudaSuccess) ||
        (!idx.empty() && (e = cudaMemcpyAsync(b->d_idx, idx.data(), sizeof(int64_t) * idx.size(),
                                              cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(b->d_vols, views.data(), sizeof(VolView) * n_vols, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (!tiles.empty() && (e = cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(),
                                                cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
        (e = cudaMemsetAsync(b->d_words, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        geo_destroy_batch(b);
        return cuda_status(e);
    }
    *out = b;
    return GEO_OK;
}

geo_status geo_destroy_batch(geo_batch b) {
    if (!b) return GEO_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    cudaFree(b->d_vols);
    cudaFree(b->d_tiles);
    cudaFree(b->d_words);
    cudaFree(b->d_idx);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    delete b;
    return GEO_OK;
}

geo_status geo_dist_to_boundary_batched(geo_batch b, const double* x, const double* y, const double* z,
                                        const double* dx, const double* dy, const double* dz, int64_t n_total,
                                        double* step, int32_t* hit, void* stream) {
    if (!b) return GEO_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    if (dev != b->device || n_total < b->max_end) return GEO_ERR_INVALID_ARG;
    if (b->ntiles == 0) return GEO_OK;
    if (!is_device_ptr(x) || !is_device_ptr(y) || !is_device_ptr(z) || !is_device_ptr(dx) || !is_device_ptr(dy) ||
        !is_device_ptr(dz) || !is_device_ptr(step) || !is_device_ptr(hit))
        return GEO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b->d_words, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_status(e);
    BatchView bv;
    bv.vols = b->d_vols;
    bv.tiles = b->d_tiles;
    bv.ntiles = b->ntiles;
    bv.counter = b->d_words;
    bv.status = b->d_words + 1;
    bv.segs = b->segs;
    bv.nvols = b->n_vols;
    bv.vox = b->vox;
    bv.pad_ = 0;
    bv.idx = b->d_idx;
    const Basket bk{x, y, z, dx, dy, dz, n_total};
    return cuda_status(
        launch_dist_batched(bv, bk, step, hit, b->blocks_per_sm, b->tile_tracks, s, num_sms_of(b->device)));
}

geo_status geo_adjoint_workspace_size(geo_volume v, int64_t n, uint64_t* bytes) {
    if (!v || !bytes || n < 0) return GEO_ERR_INVALID_ARG;
    *bytes = uint64_t(adjoint_workspace_bytes(v->view.nd, n, num_sms_of(v->device)));
    return GEO_OK;
}

geo_status geo_dist_to_boundary_adjoint(geo_volume v, const double* x, const double* y, const double* z,
                                        const double* dx, const double* dy, const double* dz, int64_t n,
                                        const int32_t* hit, const double* grad_step, double* grad_p, double* grad_d,
                                        double* grad_trans, double* grad_params, void* workspace,
                                        uint64_t workspace_bytes, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if ((st = check_basket(x, y, z, n)) != GEO_OK) return st;
    if (n == 0) return GEO_OK;
    if (!is_device_ptr(dx) || !is_device_ptr(dy) || !is_device_ptr(dz) || !is_device_ptr(hit) ||
        !is_device_ptr(grad_step) || !is_device_ptr(grad_p) || !is_device_ptr(grad_d) ||
        (grad_trans && !is_device_ptr(grad_trans)) || (grad_params && !is_device_ptr(grad_params)) ||
        !is_device_ptr(workspace))
        return GEO_ERR_INVALID_ARG;
    const int sms = num_sms_of(v->device);
    if (workspace_bytes < adjoint_workspace_bytes(v->view.nd, n, sms)) return GEO_ERR_INVALID_ARG;
    if (int64_t(adjoint_smem_bytes(v->view.nd)) > smem_budget(v->device)) return GEO_ERR_UNSUPPORTED;
    const Basket b{x, y, z, dx, dy, dz, n};
    return cuda_status(launch_adjoint(v->view, b, hit, grad_step, grad_p, grad_d, grad_trans, grad_params,
                                      static_cast<double*>(workspace), static_cast<cudaStream_t>(stream), sms));
}

geo_status geo_shape_query(const geo_placed_shape* shape, int32_t what, const double* x, const double* y,
                           const double* z, const double* dx, const double* dy, const double* dz, int64_t n,
                           double* out, int32_t* face, void* stream) {
    if (!shape) return GEO_ERR_INVALID_ARG;
    geo_status st = check_shape(*shape, false);
    if (st != GEO_OK) return st;
    if (what < GEO_Q_DIST_OUT || what > GEO_Q_CONTAINS) return GEO_ERR_INVALID_ARG;
    if ((st = check_basket(x, y, z, n)) != GEO_OK) return st;
    if (n == 0) return GEO_OK;
    const bool dist = what == GEO_Q_DIST_OUT || what == GEO_Q_DIST_IN;
    if (dist && (!is_device_ptr(dx) || !is_device_ptr(dy) || !is_device_ptr(dz))) return GEO_ERR_INVALID_ARG;
    if (!is_device_ptr(out) || (face && !is_device_ptr(face))) return GEO_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    ShapeArg a;
    std::memset(&a, 0, sizeof a);
    a.r = make_rec64(*shape);
    if (shape->kind == GEO_PCON) {
        const std::vector<double> T = pcon_table_host(*shape);
        std::copy(T.begin(), T.end(), a.table);
    }
    const Basket b{x, y, z, dist ? dx : nullptr, dist ? dy : nullptr, dist ? dz : nullptr, n};
    return cuda_status(launch_shape_query(a, what, b, out, face, static_cast<cudaStream_t>(stream),
                                          num_sms_of(dev)));
}

geo_status geo_dist_to_boundary_stats(geo_volume v, const double* x, const double* y, const double* z,
                                      const double* dx, const double* dy, const double* dz, int64_t n, double* step,
                                      int32_t* hit, int32_t* nref, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if ((st = check_basket(x, y, z, n)) != GEO_OK) return st;
    if (n == 0) return GEO_OK;
    if (!is_device_ptr(dx) || !is_device_ptr(dy) || !is_device_ptr(dz) || !is_device_ptr(step) ||
        !is_device_ptr(hit) || !is_device_ptr(nref))
        return GEO_ERR_INVALID_ARG;
    const Basket b{x, y, z, dx, dy, dz, n};
    return cuda_status(launch_dist_refine_stats(v->view, b, step, hit, nullptr, nref,
                                                static_cast<cudaStream_t>(stream), num_sms_of(v->device)));
}

geo_status geo_selftest_wait_timeout(geo_volume v, uint32_t polls, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    if (polls == 0 || polls > (1u << 20)) return GEO_ERR_INVALID_ARG;
    return cuda_status(launch_wait_selftest(v->status, polls, static_cast<cudaStream_t>(stream)));
}

geo_status geo_debug_fail_alloc(int32_t nth) {
    if (nth < 0) return GEO_ERR_INVALID_ARG;
    g_fail_alloc.store(nth);
    return GEO_OK;
}

geo_status geo_check_device_status(geo_volume v, uint32_t* word, void* stream) {
    geo_status st = check_volume_device(v);
    if (st != GEO_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int h = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&h, v->status, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(v->status, 0, sizeof h, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_status(e);
    if (word) *word = h;
    return h ? GEO_ERR_DEVICE_ASSERT : GEO_OK;
}

}  // extern "C"
