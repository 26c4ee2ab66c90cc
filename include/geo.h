/*
 * geo.h -- C ABI of the GB300 vector navigator.
 *
 * The operations are those of the vector geometry navigator of "Vectorising
 * the detector geometry to optimize particle transport" (Apostolakis, Brun,
 * Carminati, Gheata, Wenzel):
 *   - Sec. 3 / Fig. 1: for a basket of tracks inside one mother volume, the
 *     geometrical step to the next boundary along the line of flight and the
 *     volume hit (mother DistFromInside, then per daughter a master->local
 *     transform and DistFromOutside, then min + index).
 *   - Sec. 3.1: the shape queries distance-to-enter, distance-to-leave,
 *     safety (minimum distance to any boundary) and inside/outside check for
 *     Box, Tube and Cone, and the coordinate transformation and min/max
 *     algorithms the navigator needs.
 *   - Sec. 2: tracks arrive as a "basket", a structure of contiguous arrays.
 *
 * Conventions (the paper defers all shape details to the ROOT geometry
 * library; these are the readings this library implements):
 *   - Units are mm.  Solids are closed sets.  Directions are NOT renormalised:
 *     steps are in units of |d|.
 *   - Box  p = (dx, dy, dz, -, -)               half-lengths
 *     Tube p = (rmin, rmax, dz, -, -)           rmin = 0 is a solid cylinder
 *     Cone p = (dz, rmin1, rmax1, rmin2, rmax2)  radii "1" at z=-dz, "2" at +dz
 *     Tube segment (GEO_TUBS) p = (rmin, rmax, dz, sphi, dphi): the tube cut
 *       to the closed wedge of azimuths [sphi, sphi + dphi], 0 < dphi <= 2 pi
 *       (2 pi: the whole tube); the wedge holds the z axis.  Its surfaces are
 *       tagged 8 (the face at sphi) and 9 (the face at sphi + dphi).
 *     Polycone (GEO_PCON; Sec. 3.1's sequence of connected cone and tube
 *       sections) p = (sphi, dphi, nz, 0, 0) with `planes` = nz plane
 *       heights z[k], then the nz inner radii rmin[k], then the nz outer
 *       radii rmax[k] (3 nz doubles): 2 <= nz <= GEO_MAX_PLANES, z strictly
 *       increasing, 0 <= rmin[k] <= rmax[k], rmax[k] + rmax[k+1] > 0.
 *       Section k (between planes k and k+1) is the cone whose radii vary
 *       linearly from plane k to plane k+1; the solid is the union of the
 *       sections cut to the wedge [sphi, sphi + dphi] as for the tube
 *       segment.  Inner planes are no surfaces.  Surfaces: 4 / 5 the planes
 *       z[0] / z[nz-1], 8 / 9 the phi faces, 16 + 2k the outer and 17 + 2k
 *       the inner surface of section k.  A cone segment (rmin1, rmax1,
 *       rmin2, rmax2, dz, sphi, dphi) is the polycone of the two planes
 *       -dz, +dz.
 *   - A daughter is placed by a rotation R (row-major, local -> mother) and a
 *     translation t:  p_mother = R p_local + t.  The mother's frame is the
 *     frame of the tracks (its rot must be the identity and trans zero).
 *   - Miss = +inf.  Ties between equal steps: the mother wins, then the lowest
 *     daughter index (the order of the sequential algorithm of Fig. 1a).
 *   - Track outside the mother: step 0, hit -2.  Non-finite position or
 *     direction, or a zero direction: step NaN, hit -2.
 *   - Safety is the exact Euclidean distance to the nearest boundary of the
 *     mother's exclusive region; 0 inside a daughter or outside the mother.
 *
 * Memory and streams:
 *   - Every basket and output pointer is DEVICE memory owned by the caller
 *     (e.g. torch.Tensor.data_ptr()), in structure-of-arrays layout, one FP64
 *     (or int32) element per track, no stride.  Host pointers are rejected
 *     with GEO_ERR_INVALID_ARG (except in geo_dist_to_boundary_host).
 *   - The library owns a volume's device tables from geo_build_volume until
 *     geo_destroy_volume.  Query calls allocate nothing.
 *   - Query calls are asynchronous on `stream` (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream) and never synchronise the host.
 *   - n == 0 returns GEO_OK and launches nothing.
 *   - Nothing throws across this boundary; every call returns a geo_status.
 *     geo_status_string() gives a static description.
 */
#ifndef GEONAV_GEO_H
#define GEONAV_GEO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GEO_OK = 0,
    GEO_ERR_INVALID_ARG = 1,    /* null/host pointer, n < 0, bad mode, bad kind     */
    GEO_ERR_SHAPE_PARAMS = 2,   /* non-finite or inconsistent shape / placement     */
    GEO_ERR_OOM = 3,            /* device allocation failed (builder only)          */
    GEO_ERR_CUDA = 4,           /* a CUDA runtime call failed                       */
    GEO_ERR_DEVICE_ASSERT = 5,  /* a kernel reported a failed internal check        */
    GEO_ERR_UNSUPPORTED = 6     /* valid request the library does not implement     */
} geo_status;

typedef enum { GEO_BOX = 0, GEO_TUBE = 1, GEO_CONE = 2, GEO_TUBS = 3, GEO_PCON = 4 } geo_kind;

#define GEO_MAX_PLANES 32

/* Tracks per tile of the FP32-filter kernels and of the batched launches
 * (geo_build_batch, geo_dist_to_boundary_batched_noalloc). */
#define GEO_TILE_TRACKS 384

/* GEO_FP64: every operation in FP64.
 * GEO_FP32_REFINE: a conservative FP32 pass bounds every candidate from below;
 * only candidates that can still win are recomputed with the same FP64
 * routines as GEO_FP64, so both modes return the same answers.
 * GEO_SAFETY_ESTIMATE (geo_safety only): the cheaper, under-estimating
 * safety (see geo_safety). */
typedef enum { GEO_FP64 = 0, GEO_FP32_REFINE = 1, GEO_SAFETY_ESTIMATE = 2 } geo_mode;

/* One placed solid.  kind: geo_kind.  p: shape parameters (see above).
 * rot: row-major 3x3 rotation local -> mother, orthonormal with det +1 within
 * 1e-12.  trans: translation (mm).  planes: for GEO_PCON a host array of
 * 3 * nz doubles (see above), read during the call that receives the struct
 * and not kept; ignored for the other kinds. */
typedef struct {
    int32_t kind;
    int32_t reserved;   /* must be 0 */
    double p[5];
    double rot[9];
    double trans[3];
    const double* planes;
} geo_placed_shape;

/* Build options.  voxelize != 0 builds a uniform-grid candidate list over the
 * mother's bounding box (grid[i] cells per axis; 0 = chosen from the daughter
 * count).  Daughter lists per voxel are used by geo_dist_to_boundary. */
typedef struct {
    int32_t voxelize;
    int32_t grid[3];
} geo_build_opts;

typedef struct geo_volume_s* geo_volume;

/* ---- one solid on its own (Sec. 3.1's per-shape algorithms, as measured
 * per shape in Fig. 2) ------------------------------------------------------ */
typedef enum {
    GEO_Q_DIST_OUT = 0,    /* DistFromOutside: inf{s >= 0 : x + s u in solid}; 0 inside; +inf miss */
    GEO_Q_DIST_IN = 1,     /* DistFromInside: end of the component of s = 0; 0 for x outside       */
    GEO_Q_SAFETY_OUT = 2,  /* distance from a point outside to the solid; 0 inside                 */
    GEO_Q_SAFETY_IN = 3,   /* distance from a point inside to the boundary; 0 outside              */
    GEO_Q_CONTAINS = 4     /* 1.0 if the closed solid contains the point, else 0.0                 */
} geo_shape_query_kind;

/* Evaluates one query of one placed solid for n tracks: positions x,y,z and
 * (for the two distances) directions dx,dy,dz are device FP64[n] in the frame
 * the solid is placed in (the placement's master->local transform is applied
 * per track; an identity placement queries the solid in its own frame).
 * Writes out[n] (device FP64) and, if face is not NULL, face[n] (device
 * int32): the surface crossed by a distance (box 0..5 = -x,+x,-y,+y,-z,+z;
 * tube and cone 4/5 = -z/+z planes, 6 outer, 7 inner; segments 8/9 the phi
 * faces; polycone sections 16 + 2k / 17 + 2k; -1 none), -1 for the other
 * queries.  A polycone's plane table travels in the kernel's parameters (the
 * call allocates nothing).  dx,dy,dz may be NULL for the safeties and Contains.
 * Non-finite input, or a zero direction for a distance: NaN.  The values are
 * those of the navigator's FP64 routines.  Errors: bad kind or parameters of
 * the solid (as geo_build_volume), bad query, host pointers. */
geo_status geo_shape_query(const geo_placed_shape* shape, int32_t what, const double* x, const double* y,
                           const double* z, const double* dx, const double* dy, const double* dz, int64_t n,
                           double* out, int32_t* face, void* stream);

/* Builds the device tables of one logical volume (Fig. 1: a mother and its
 * daughter volumes).  `mother` and `daughters[0..n_daughters)` are host
 * structs, copied; the caller may free them on return.  n_daughters may be 0.
 * Validation: kinds, finiteness, dz > 0, 0 <= rmin <= rmax (rmin1<=rmax1,
 * rmin2<=rmax2, rmax1+rmax2 > 0 for cones), 0 < dphi <= 2 pi for segments,
 * the polycone rules above (GEO_ERR_INVALID_ARG for planes == NULL or nz
 * out of range, GEO_ERR_SHAPE_PARAMS for the rest), orthonormal rotations.
 * Polycones' plane tables are copied to the device with the volume.  Allocates
 * device memory and copies on `stream`, then synchronises that stream.
 * On success *out owns the tables; on failure *out is NULL. */
geo_status geo_build_volume(const geo_placed_shape* mother, const geo_placed_shape* daughters,
                            int32_t n_daughters, const geo_build_opts* opts, void* stream,
                            geo_volume* out);

/* Frees the device tables (synchronises the device first).  NULL is a no-op. */
geo_status geo_destroy_volume(geo_volume v);

/* Number of daughters, and whether a voxel grid was built (1/0). */
geo_status geo_volume_info(geo_volume v, int32_t* n_daughters, int32_t* voxelized, int32_t grid[3]);

/* Fig. 1 navigator step for n tracks.  Inputs x,y,z (positions) and dx,dy,dz
 * (directions): device FP64 arrays of n elements.  Outputs: step[n] (FP64,
 * units of |d|), hit[n] (int32: -1 mother, j >= 0 daughter j, -2 outside or
 * invalid).  bpoint: NULL, or a device FP64 array of 3n elements receiving the
 * boundary point p + step*d as three consecutive SoA blocks (x[n], y[n], z[n]).
 * mode: geo_mode. */
geo_status geo_dist_to_boundary(geo_volume v, const double* x, const double* y, const double* z,
                                const double* dx, const double* dy, const double* dz, int64_t n,
                                double* step, int32_t* hit, double* bpoint, int32_t mode,
                                void* stream);

/* Inside/outside check of Sec. 3.1 at navigator level: where[i] = -2 outside
 * the mother, -1 in the mother's exclusive part, j = the lowest-index daughter
 * whose closed solid contains the point.  x,y,z device FP64[n]; where device
 * int32[n].  mode GEO_FP64 tests every daughter's bounding sphere and solid
 * in FP64; GEO_FP32_REFINE decides in FP32 on inflated (or, for the mother,
 * deflated) copies and tests in FP64 only the daughters the FP32 test cannot
 * exclude.  Both modes give the same answer for every point.  Other modes:
 * GEO_ERR_INVALID_ARG. */
geo_status geo_contains(geo_volume v, const double* x, const double* y, const double* z, int64_t n,
                        int32_t* where, int32_t mode, void* stream);

/* Safety of Sec. 3.1 at navigator level: min(mother inside-safety, min over
 * daughters of outside-safety), exact Euclidean; 0 outside the mother or
 * inside a daughter.  safety device FP64[n].  mode GEO_FP64 evaluates every
 * candidate not culled by its FP64 bounding sphere; GEO_FP32_REFINE bounds
 * every candidate from below in FP32 and evaluates in FP64 only those whose
 * bound does not exceed the smallest FP64 value found (usually one); both
 * modes return the same FP64 minimum.  GEO_SAFETY_ESTIMATE returns a cheaper
 * lower bound of the safety (never above it, 0 outside the mother or inside
 * a daughter), in the manner of ROOT's estimated safeties: every solid is
 * replaced by a simpler bound of its distance -- box and tube the exact
 * distance, cone the largest distance to a supporting half-plane of its
 * meridian trapezoid, tube segment and polycone the distance to the tube
 * enclosing them; the mother (box, tube, cone) its inside distance, a
 * segment or polycone mother 0 -- each evaluated in FP32 on a copy grown
 * (mother: shrunk) by the filter's inflation and lowered by a relative
 * 2^-18, with no FP64 work but the mother's containment test.  The value is
 * below that bound by at most about the inflation (a few 1e-5 of the
 * mother's extent). */
geo_status geo_safety(geo_volume v, const double* x, const double* y, const double* z, int64_t n,
                      double* safety, int32_t mode, void* stream);

/* Same as geo_dist_to_boundary but every array is HOST memory; a device
 * pointer among them gives GEO_ERR_INVALID_ARG.  When all eight arrays are
 * page-locked (cudaHostAlloc, cudaHostRegister; pinned torch tensors), one
 * step runs on them in place: the kernel reads the tracks and writes the
 * results across the host link, with no staging copies, and `chunk` is
 * unused.  Otherwise (pageable memory) the library stages the basket through a
 * device workspace of three buffers of `chunk` tracks (0 = 1<<18) as a
 * pipeline: chunk c+1 is copied in on an internal stream while chunk c is
 * stepped and chunk c-1 copied out on a second internal stream, and a buffer
 * is refilled as soon as its chunk has been copied out; even chunks
 * are stepped on `stream`, odd ones on a third internal stream (joined to
 * `stream` at the end), so that consecutive steps overlap.  Returns after
 * synchronising.  The workspace, streams and events are made
 * on the first call and kept with the volume (the buffers grow when `chunk`
 * grows); calls on one volume are serialised by a lock. */
geo_status geo_dist_to_boundary_host(geo_volume v, const double* x, const double* y,
                                     const double* z, const double* dx, const double* dy,
                                     const double* dz, int64_t n, double* step, int32_t* hit,
                                     int32_t mode, int64_t chunk, void* stream);

/* ---- many logical volumes in one launch -------------------------------
 * Tracks grouped by logical volume (the "basket" of Sec. 2: particles in the
 * same logical volume).  A batch is a list of baskets; basket k holds the
 * tracks [offset, offset + count) of shared SoA arrays, all inside volume
 * vols[volume]. */
typedef struct {
    int32_t volume;     /* index into the vols array of geo_build_batch      */
    int32_t reserved;   /* must be 0                                          */
    int64_t offset;     /* first track of the basket in the SoA arrays        */
    int64_t count;      /* number of tracks (>= 0)                            */
} geo_basket;

/* tile_order: 0 = largest estimated cost first (tracks x daughters), 1 = in
 * basket order (the packed tiles of ragged tails after the baskets' full
 * tiles, volume by volume).  blocks_per_sm: resident blocks of the persistent launch
 * (0 = as many as fit).  tile_tracks: the tile shape, 0 or GEO_TILE_TRACKS
 * (384 tracks per tile, 12 producer and 4 consumer warps) or 256 (8 producer
 * and 4 consumer warps).  Values other than these give GEO_ERR_INVALID_ARG. */
typedef struct {
    int32_t tile_order;
    int32_t blocks_per_sm;
    int32_t tile_tracks;
} geo_batch_opts;

typedef struct geo_batch_s* geo_batch;

/* Builds a batch: copies the baskets, splits them into tiles of
 * tile_tracks (default GEO_TILE_TRACKS) consecutive tracks, gathers the ragged
 * remainders of each volume's baskets into packed tiles of up to that many tracks (listing
 * their indices), orders the
 * tiles, and uploads the per-volume views, the tile list, the packed
 * indices and a tile counter to the device (the batch owns them).  The volumes must
 * stay alive while the batch is used.  All volumes must live on the current
 * device.  Synchronises `stream`. */
geo_status geo_build_batch(const geo_volume* vols, int32_t n_vols, const geo_basket* baskets,
                           int32_t n_baskets, const geo_batch_opts* opts, void* stream,
                           geo_batch* out);
geo_status geo_destroy_batch(geo_batch b);

/* Navigator step for every basket of the batch in ONE persistent launch
 * (GEO_FP32_REFINE; answers identical to geo_dist_to_boundary per basket).
 * x..dz: device FP64 SoA arrays of n_total tracks; step (FP64) and hit (int32)
 * device arrays of n_total, written for the tracks of the baskets only.
 * n_total must cover every basket (offset + count <= n_total).  Blocks claim
 * tiles from the batch's device counter, which the call resets with an
 * asynchronous memset on `stream` first; the call allocates nothing and does
 * not synchronise, so it can be captured in a CUDA graph.  Calls on the same
 * batch must not overlap on the GPU (they share the counter). */
geo_status geo_dist_to_boundary_batched(geo_batch b, const double* x, const double* y, const double* z,
                                        const double* dx, const double* dy, const double* dz,
                                        int64_t n_total, double* step, int32_t* hit, void* stream);

/* For callers that must not allocate device memory while they run (an
 * application whose allocator owns all device memory, a real-time loop that
 * forbids allocation after start-up).  The paper has no counterpart: this is
 * a service of the library.
 * Same step and answers as geo_build_batch + geo_dist_to_boundary_batched
 * (GEO_FP32_REFINE), but this call allocates nothing: the tile list, the
 * volume views, the tile counter and the status word are kept in a fixed
 * array of device memory owned by the library (about 0.55 MB, present on
 * every device that loads it until the process exits).  Limits: at most 64
 * volumes and 32768 tiles of GEO_TILE_TRACKS tracks (about 12.6 M tracks) per call; larger
 * requests return GEO_ERR_INVALID_ARG.  vols: volumes built earlier with
 * geo_build_volume, on the current device.  baskets: HOST array, as for
 * geo_build_batch.  x..dz, step, hit: device arrays as for
 * geo_dist_to_boundary_batched, n_total covering every basket.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and caches it.
 * Every call reuses the same array, so calls that overlap on the GPU (on
 * different streams, or from different host threads) race: serialise them.
 * The counter and status word are cleared by each call; the rest keeps the
 * last call's contents.  The tile list and the volume views are copied from
 * host memory that is not page-locked; such a copy waits for the work already
 * queued on `stream`, so the call may block the host until that work is done.
 * A wait of the kernel that runs out, or a tile index outside n_total, is
 * recorded in the status word of every volume of the call (read it with
 * geo_check_device_status). */
geo_status geo_dist_to_boundary_batched_noalloc(const geo_volume* vols, int32_t n_vols,
                                                const geo_basket* baskets, int32_t n_baskets,
                                                const double* x, const double* y, const double* z,
                                                const double* dx, const double* dy, const double* dz,
                                                int64_t n_total, double* step, int32_t* hit,
                                                void* stream);

/* ---- a tree of logical volumes: the step followed by final localisation -
 * The paper's navigator ends at the distance to the next boundary and the
 * volume hit; locating the track in the volume it then enters (or returns
 * to) is left out there.  These calls add it for a tree of logical volumes.
 *
 * Tree: volumes[v] are built logical volumes (geo_build_volume); daughter j
 * of volume v is an instance of volumes[child[o_v + j]], o_v = the number of
 * daughters of volumes 0..v-1; that volume's mother solid must equal the
 * daughter's solid (kind and parameters, else GEO_ERR_SHAPE_PARAMS).  The
 * frame of volumes[root] is the frame of the tracks.  Placed volumes (nodes)
 * are numbered breadth first from the root (node 0): the children of a node
 * are consecutive in daughter order, nodes expanded in number order.  At
 * most 2^24 nodes and 64 levels (else GEO_ERR_INVALID_ARG).  The world keeps
 * pointers to the volumes' device tables: destroy the world before them.
 *
 * Track state: a node (-1 outside the root) and a flag: j >= 0 when the
 * track has just left daughter j of its node (its next step takes j's
 * re-entry distance instead of DistFromOutside, which would be 0 on j's
 * surface), -2 when it has just entered its node through the node's surface
 * (a start point a rounding outside the node is accepted and the mother's
 * exit is that of the part being entered), -1 otherwise (after Locate). */
typedef struct geo_world_s* geo_world;

geo_status geo_build_world(const geo_volume* volumes, int32_t n_volumes, const int32_t* child, int32_t root,
                           void* stream, geo_world* out);
geo_status geo_destroy_world(geo_world w);
/* Number of nodes and depth of the deepest node (root = 0). */
geo_status geo_world_info(geo_world w, int32_t* n_nodes, int32_t* max_depth);
/* Host arrays of n_nodes: logical volume, parent (-1 for the root), slot in
 * the parent's daughters (-1), first child's node number.  Any may be NULL. */
geo_status geo_world_nodes(geo_world w, int32_t* lv, int32_t* parent, int32_t* slot, int32_t* first_child);

/* Locate: node[i] = the deepest node whose closed solid contains point i,
 * choosing at every level the lowest-index daughter that contains it; -1
 * outside the root's solid, -2 non-finite.  Device arrays. */
geo_status geo_world_locate(geo_world w, const double* x, const double* y, const double* z, int64_t n,
                            int32_t* node, void* stream);

/* One step of every track: the step of Fig. 1 in the logical volume of its
 * node (mode as in geo_dist_to_boundary; both modes give the same answers),
 * then relocation at the boundary point:
 *   a daughter hit: that child, then down while a daughter contains the
 *   point (lowest index first); flag_out -2;
 *   the node's own boundary: up to the parent, where the lowest-index
 *   daughter other than the one left that contains the point is entered
 *   (then down; flag -2), else the parent itself if its solid contains the
 *   point (flag = the slot left), else up again; leaving the root: node -1.
 * A track not inside its node's solid (flag != -2), with an invalid node or
 * invalid input gets node -2 (step 0, or NaN for invalid input).
 * Inputs: positions and directions in the root frame, node_in, flag_in
 * (NULL = all -1); outputs step[n] (units of |d|), node_out[n], flag_out[n]
 * (may be NULL).  The caller moves the track: p + step * d.  Device arrays.
 * The tracks are first grouped by the logical volume of their node (in a
 * scratch array the world owns, allocated on the first call and grown when
 * n grows: such a call synchronises `stream`); calls on one world must not
 * overlap on the GPU. */
geo_status geo_world_step(geo_world w, const double* x, const double* y, const double* z, const double* dx,
                          const double* dy, const double* dz, int64_t n, const int32_t* node_in,
                          const int32_t* flag_in, double* step, int32_t* node_out, int32_t* flag_out, int32_t mode,
                          void* stream);

/* ---- gradients of the step (the paper has no gradients; this supports a
 * differentiable use of the navigator) ----------------------------------
 * For loss L with dL/dstep = grad_step (device FP64[n]) and the forward
 * answers hit (device int32[n], from geo_dist_to_boundary on the same
 * inputs, either mode), writes
 *   grad_p (device FP64[3n], SoA x|y|z blocks)  dL/dposition per track,
 *   grad_d (device FP64[3n], SoA)               dL/ddirection per track,
 *   grad_trans (device FP64[3*nd] or NULL)      dL/dt_j summed over tracks,
 *   grad_params (device FP64[5*(nd+1)] or NULL) dL/dp_j[0..4] summed over
 *       tracks, daughters first then the mother's parameters at 5*nd,
 * by the implicit-function rule on the surface the winning solid's FP64
 * routine crossed.  Tracks without a defined surface (inside a daughter,
 * outside the mother, invalid) get 0; so does a hit index >= nd, which also
 * sets the volume's device status word (geo_check_device_status).  The sums over tracks are deterministic
 * (fixed-order two-pass reduction) and need a caller-provided device
 * workspace of geo_adjoint_workspace_size() bytes. */
geo_status geo_adjoint_workspace_size(geo_volume v, int64_t n, uint64_t* bytes);
geo_status geo_dist_to_boundary_adjoint(geo_volume v, const double* x, const double* y, const double* z,
                                        const double* dx, const double* dy, const double* dz, int64_t n,
                                        const int32_t* hit, const double* grad_step, double* grad_p,
                                        double* grad_d, double* grad_trans, double* grad_params,
                                        void* workspace, uint64_t workspace_bytes, void* stream);

/* Same as geo_dist_to_boundary in GEO_FP32_REFINE mode, and also writes, per
 * track, the number of FP64 solid evaluations the refine stage performed
 * (mother and daughters; 1000 is added when the track fell back to the full
 * FP64 loop) into nref (device int32[n]).  For measurement of the filter. */
geo_status geo_dist_to_boundary_stats(geo_volume v, const double* x, const double* y, const double* z,
                                      const double* dx, const double* dy, const double* dz, int64_t n,
                                      double* step, int32_t* hit, int32_t* nref, void* stream);

/* Reads and clears the volume's device status word (errors recorded by
 * kernels: 1 a bulk-copy wait that ran out of polls, 2 a track index outside
 * the basket, 4 a pipeline wait that ran out of polls; the batched launches
 * record theirs in every volume of the batch).  Synchronises `stream`.
 * Returns GEO_ERR_DEVICE_ASSERT if any was recorded; *word gets the raw bits
 * when non-NULL. */
geo_status geo_check_device_status(geo_volume v, uint32_t* word, void* stream);

/* ---- test support: failure detection without a GPU fault ----------------
 * The paper has no counterpart; these exercise the library's failure paths.
 *
 * geo_selftest_wait_timeout: launches one warp that waits, with `polls`
 * (1 .. 2^20) polls of the pipeline's bounded wait, on a shared-memory
 * barrier that no thread arrives at --
 * the failure path of every bounded wait of the pipeline kernels -- and
 * records bit 4 in the volume's status word; the kernel then returns, so the
 * context stays usable.  Asynchronous on `stream`; read the word with
 * geo_check_device_status.
 *
 * geo_debug_fail_alloc: host-side fault injection.  With nth > 0, the nth
 * allocation the library makes from now on (host objects of volumes, batches
 * and trees, and their device memory) fails as if memory had run out: the
 * building call frees what it had taken and returns GEO_ERR_OOM.  0 turns it
 * off; negative values give GEO_ERR_INVALID_ARG.  Process-wide. */
geo_status geo_selftest_wait_timeout(geo_volume v, uint32_t polls, void* stream);
geo_status geo_debug_fail_alloc(int32_t nth);

/* Measurement support (not part of the navigator): issue rate in operations
 * per second of one arithmetic operation over the whole GPU: what = 0 FP32
 * FMA, 1 FP64 FMA, 2 FP64 divide, 3 FP64 square root, 4 FP32 divide, 5 FP32
 * square root.  scratch: device buffer of >= 256 doubles.  Synchronises. */
geo_status geo_probe_pipe(int32_t what, int64_t iters, int32_t blocks, void* scratch, void* stream,
                          double* ops_per_s);

const char* geo_status_string(geo_status s);

#ifdef __cplusplus
}
#endif

#endif /* GEONAV_GEO_H */
