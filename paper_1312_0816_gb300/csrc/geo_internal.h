// geo_internal.h -- device table layout and launch interfaces shared by the
// CUDA translation units of the navigator library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <new>
#include <cuda_runtime.h>
#include "../../include/geo.h"

namespace geonav {

constexpr int KBOX = 0, KTUBE = 1, KCONE = 2, KTUBS = 3, KPCON = 4;
constexpr int kMaxPlanes = GEO_MAX_PLANES;
// tracks per tile of the FP32-filter kernels (one per producer thread)
constexpr int kTileTracks = GEO_TILE_TRACKS;

// Plane table of one polycone of n planes (m = n - 1 sections), FP64:
//  [0, n) z, [n, 2n) rmin, [2n, 3n) rmax, [3n, 3n+m) inner slopes b_in,
//  [3n+m, 3n+2m) outer slopes b_out; section k's radius lines are
//  R(z) = r[k] + b[k] (z - z[k]).
constexpr int pcon_table_len(int n) { return 3 * n + 2 * (n - 1); }
constexpr int kPconTableMax = pcon_table_len(kMaxPlanes);

// FP64 record of one placed solid, 256 B, read warp-uniformly (broadcast).
//  R: row-major local->mother rotation, t: translation.
//  p: raw parameters.  d: derived constants per kind:
//   box : d[0..2] = half-lengths
//   tube: d[0] rmin, d[1] rmax, d[2] dz, d[3] rmin^2, d[4] rmax^2
//   cone: d[0] dz, d[1] a_out, d[2] b_out, d[3] a_in, d[4] b_in,
//         d[5] rmin1^2, d[6] rmax1^2, d[7] rmin2^2, d[8] rmax2^2,
//         d[9] 1/sqrt(1+b_out^2), d[10] 1/sqrt(1+b_in^2), d[11] has_inner (0/1)
//   tube segment: d[0..4] as the tube, d[5], d[6] n1 = (-sin sphi, cos sphi),
//         d[7], d[8] n2 = (sin(sphi+dphi), -cos(sphi+dphi)): the wedge is
//         {n1.(x,y) >= 0} AND (d[9] = 1, dphi <= pi) or OR (d[9] = 0) the
//         same for n2; d[10] = 1 for a whole turn (no wedge); d[11] = 1 for
//         a half turn (both faces in one plane)
//   (radius lines R(z) = a + b z, R(-dz) = r1, R(+dz) = r2)
//   polycone: d[0] the device address of its plane table (bit pattern),
//         d[1] nz, d[2] rmin[0]^2, d[3] rmax[0]^2, d[4] rmin[nz-1]^2,
//         d[12] rmax[nz-1]^2, d[5..11] the wedge as for the tube segment;
//         p = (sphi, dphi, nz, 0, 0)
//  brad: bounding-sphere radius about t, enlarged by a relative 1e-12 + 1e-9 mm
//  so that the FP64 sphere cull is conservative.
//  flags: kRec64Identity when the rotation is exactly the identity: the
//  master->local transform is then x = p - t, u = d (3 FP64 operations
//  instead of 21; every kernel takes the same branch, so all agree bit for
//  bit).
constexpr int32_t kRec64Identity = 1;
struct __align__(16) ShapeRec64 {
    double R[9];
    double t[3];
    double p[5];
    double d[13];
    double brad;
    int32_t kind;
    int32_t flags;
};
static_assert(sizeof(ShapeRec64) == 256, "ShapeRec64 layout");

// FP32 record of one placed solid for the conservative filter, 128 B.
//  The shape is INFLATED by `delta` (mm) so that every FP32 rounding of the
//  transform and of the shape arithmetic is covered (see nav_refine.cu):
//   box : e[0..2] = h + delta
//   tube: e[0] rmin_in^2 (shrunk hole, 0 if none), e[1] rmax_out^2, e[2] dz + delta,
//         e[3] has_hole (0/1), e[4..6] acceptance limits (shapes32.cuh)
//   cone: e[0] dz + delta, e[1] a_out', e[2] b_out, e[3] a_in', e[4] b_in,
//         e[5] has_hole, e[6..9] inflated end radii squared (rmin1,rmax1,rmin2,rmax2),
//         e[10..14] acceptance limits (shapes32.cuh)
//  brad: inflated bounding radius; brad2 = brad^2 rounded up, beside t so
//  that the bounding-sphere test reads both with one 16-byte load.
//  flags: kRec32Identity when the rotation is exactly the identity (the
//  filter then skips the rotation: x = R^T w is w itself).
constexpr int32_t kRec32Identity = 1;
struct __align__(16) ShapeRec32 {
    float t[3];
    float brad2;
    float R[9];
    float e[15];
    float brad;
    float delta;
    int32_t kind;
    int32_t flags;
};
static_assert(sizeof(ShapeRec32) == 128, "ShapeRec32 layout");

// Everything a kernel needs about one volume, passed by value (or copied
// from a device array of views by the batched kernel).
struct __align__(16) VolView {
    ShapeRec64 m64;            // mother (identity placement)
    ShapeRec32 m32;            // mother, FP32 (deflated for lower bounds of the exit)
    ShapeRec32 m32u;           // mother, FP32 inflated (upper bound of the exit)
    const ShapeRec64* d64;     // [nd] device
    const ShapeRec32* d32;     // [nd] device
    int32_t nd;
    int32_t smem64;            // 1 if the FP64 table fits the shared-memory budget
    int32_t smem_refine;       // 1 if the FP32 + FP64 tables fit it together
    // voxel grid (uniform over the mother's bounding box)
    int32_t voxelized;
    int32_t grid[3];
    int32_t segs;              // 1 if the mother or a daughter is a tube segment or a polycone
    double lo[3];
    double cell[3];
    double inv_cell[3];
    const int32_t* vox_off;    // [ncells+1] CSR offsets
    const int32_t* vox_ids;    // daughter ids
    unsigned int* status;      // device error word (0 = ok)
};

struct Basket {
    const double *x, *y, *z, *dx, *dy, *dz;
    int64_t n;
};

// One tile of the batched launch: up to kTileTracks consecutive tracks of one
// basket, or (count < 0) up to kTileTracks tracks of one volume listed from
// BatchView::idx[base].
struct BatchTile {
    int32_t vol;
    int32_t count;
    int64_t base;
};
static_assert(sizeof(BatchTile) == 16, "BatchTile layout");

struct BatchView {
    const VolView* vols;      // device array of per-volume views
    const BatchTile* tiles;   // device array, in claim order
    int64_t ntiles;
    unsigned int* counter;    // next tile to claim (reset before every launch)
    unsigned int* status;     // device error word of the batch
    int32_t segs;             // 1 if a volume holds a tube segment or a polycone
    int32_t nvols;            // entries of vols
    int32_t vox;              // 1 if a volume has a uniform grid
    int32_t pad_;
    const int64_t* idx;       // track indices of packed tiles (count < 0), or null
};

// device error codes written to VolView::status
constexpr unsigned ST_TMA_TIMEOUT = 1u;
constexpr unsigned ST_BAD_INDEX = 2u;
constexpr unsigned ST_SYNC_TIMEOUT = 4u;

// the failure path of a bounded wait, run on purpose (tests)
cudaError_t launch_wait_selftest(unsigned int* status, uint32_t polls, cudaStream_t s);
// shared memory of the refine kernel's two stage buffers (host)
size_t refine_stage_bytes();
// the refine kernel in its latency configuration (small baskets)
cudaError_t launch_dist_refine_latency(const VolView& v, const Basket& b, double* step, int32_t* hit,
                                       double* bpoint, int32_t* nref, cudaStream_t s, int num_sms);

// small baskets in volumes of many daughters: the FP32 pass of a track split
// over the warps of a block
bool split_basket(const VolView& v, int64_t n, int num_sms);
cudaError_t launch_dist_refine_split(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                                     int32_t* nref, cudaStream_t s);

// launchers (host), each returns cudaGetLastError() of its launch
cudaError_t launch_dist_fp64(const VolView& v, const Basket& b, double* step, int32_t* hit,
                             double* bpoint, cudaStream_t s, int num_sms);
cudaError_t launch_dist_refine(const VolView& v, const Basket& b, double* step, int32_t* hit,
                               double* bpoint, cudaStream_t s, int num_sms);
// small baskets (at most 8 tracks per SM, at most 32 daughters, no voxels):
// one warp per track
bool small_basket(const VolView& v, int64_t n, int num_sms);
cudaError_t launch_dist_warp(const VolView& v, const Basket& b, double* step, int32_t* hit, double* bpoint,
                             cudaStream_t s, int num_sms);
cudaError_t launch_dist_refine_stats(const VolView& v, const Basket& b, double* step, int32_t* hit,
                                     double* bpoint, int32_t* nref, cudaStream_t s, int num_sms);
cudaError_t launch_dist_batched(const BatchView& bv, const Basket& b, double* step, int32_t* hit,
                                int blocks_per_sm, int tile_tracks, cudaStream_t s, int num_sms);
cudaError_t launch_contains(const VolView& v, const Basket& b, int32_t* where, int mode, cudaStream_t s,
                            int num_sms);
cudaError_t launch_safety(const VolView& v, const Basket& b, double* saf, int mode, cudaStream_t s,
                          int num_sms);
// FP32-filtered Contains and Safety (queries.cu); same answers as the FP64 ones
cudaError_t launch_contains_filter(const VolView& v, const Basket& b, int32_t* where, cudaStream_t s,
                                   int num_sms);
cudaError_t launch_safety_filter(const VolView& v, const Basket& b, double* saf, cudaStream_t s, int num_sms);
// the under-estimating safety (the FP32 lower bounds alone)
cudaError_t launch_safety_estimate(const VolView& v, const Basket& b, double* saf, cudaStream_t s, int num_sms);

// One solid for geo_shape_query: its record and, for a polycone, its plane
// table (the record's table address is not used: the kernel reads `table`).
struct ShapeArg {
    ShapeRec64 r;
    double table[kPconTableMax];
};
cudaError_t launch_shape_query(const ShapeArg& a, int what, const Basket& b, double* out, int32_t* face,
                               cudaStream_t s, int num_sms);
size_t adjoint_smem_bytes(int nd);
size_t adjoint_workspace_bytes(int nd, int64_t n, int num_sms);
cudaError_t launch_adjoint(const VolView& v, const Basket& b, const int32_t* hit, const double* gstep, double* gp,
                           double* gd, double* gtrans, double* gparams, double* workspace, cudaStream_t s,
                           int num_sms);

// The library's allocations go through these, so that geo_debug_fail_alloc()
// (host-side fault injection for the tests) can make one of them fail as if
// memory had run out (defined in geo_abi.cu).
bool lib_alloc_fails();
cudaError_t lib_malloc_raw(void** p, size_t bytes);
template <class T>
inline cudaError_t lib_malloc(T** p, size_t bytes) {
    return lib_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline T* lib_new() {
    return lib_alloc_fails() ? nullptr : new (std::nothrow) T;
}

// accessors of the opaque volume handle (defined in geo_abi.cu)
const VolView* volume_view(geo_volume v);
const ShapeRec64* volume_host_daughters(geo_volume v);   // host copy, nd records
const double* volume_host_table(geo_volume v, int j);    // host plane table of daughter j (-1: mother), or null
int volume_device(geo_volume v);
int sm_count(int device);

}  // namespace geonav
