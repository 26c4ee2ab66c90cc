// world.cuh -- a tree of logical volumes and the final localisation after a
// step, the part of the navigator that the paper leaves out (after the
// distance to the next boundary and the volume hit, the track must be
// located in the volume it enters or returns to).
//
// Layout.  Placed volumes (nodes) are numbered breadth first from the root:
// the children of a node are consecutive, in daughter order.  Per node the
// device holds its logical volume, parent, slot in the parent and first child
// (int32 structure of arrays), and its world transform (R row-major, t: 12
// doubles; p_world = R p_node + t), composed on the host when the tree is
// built.  The logical volumes keep their own tables (geo_volume); the world
// holds a device array of their views.
//
// A step of track i in node N: world -> N's frame with N's transform, the
// step of Fig. 1 in N's logical volume (plain FP64 or FP32 filter + FP64
// refine), then relocation at the boundary point b (in N's frame, FP64):
//   hit j >= 0   -> child j, then down while a daughter's closed solid
//                   contains the point (lowest index first);
//   hit -1       -> up: in the parent the lowest daughter other than the one
//                   just left that contains b is entered (then down), else
//                   the parent itself if its solid contains b, else up again;
//                   leaving the root gives -1.
// The track carries a flag: j >= 0 after leaving daughter j into its node
// (the next step takes j's re-entry distance instead of DistFromOutside,
// which would be 0 on j's surface), -2 after entering its node through the
// node's surface (its start may lie a rounding outside; the mother's exit is
// that of the part being entered), -1 after Locate.
#pragma once
#include "geo_internal.h"
#include "nav_common.cuh"
#include "nav_refine.cuh"
#include "queries.cuh"
#include "shapes64.cuh"

namespace geonav {

constexpr int kMaxWorldDepth = 64;
constexpr int64_t kMaxWorldNodes = int64_t(1) << 24;

// device view of the node table
struct WorldView {
    const VolView* vols;
    const int32_t* lv;
    const int32_t* parent;
    const int32_t* slot;
    const int32_t* first;
    const double* xf;   // [12 * nnodes]
    int32_t nnodes;
};

cudaError_t launch_world_locate(const WorldView& w, const Basket& b, int32_t* node, cudaStream_t s, int num_sms);
// counting sort of the track indices by the logical volume of their node:
// cnt holds nlv + 1 ints of scratch, perm n ints (the order)
cudaError_t launch_world_group(const WorldView& w, int64_t n, const int32_t* node_in, int nlv, int32_t* cnt,
                               int32_t* perm, cudaStream_t s, int num_sms);
cudaError_t launch_world_step(const WorldView& w, const Basket& b, const int32_t* perm, const int32_t* node_in,
                              const int32_t* flag_in, double* step, int32_t* node_out, int32_t* flag_out, int mode,
                              cudaStream_t s, int num_sms);

// x in N's frame: R^T (p - t)
__device__ __forceinline__ void world_to_node(const double* G, double px, double py, double pz, double qx,
                                              double qy, double qz, double* x, double* u) {
    const double w0 = SUB(px, G[9]), w1 = SUB(py, G[10]), w2 = SUB(pz, G[11]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        x[k] = FMA(G[6 + k], w2, FMA(G[3 + k], w1, MUL(G[k], w0)));
        u[k] = FMA(G[6 + k], qz, FMA(G[3 + k], qy, MUL(G[k], qx)));
    }
}

// The first daughter of v from index `from` on, other than `skip`, whose
// inflated FP32 copy holds the FP32 point (-1: none).  A daughter is excluded
// when the point lies outside its inflated bounding sphere or its inflated
// copy (then the exact point is outside by more than the FP64 rounding).
__device__ __forceinline__ int next_candidate(const VolView& v, const float* p32, int skip, int from) {
    for (int j = from; j < v.nd; ++j) {
        if (j == skip) continue;
        const ShapeRec32& r = v.d32[j];
        float o[3], xs[3];
        const float c2 = offset32(r, p32, o);
        if (c2 > r.brad * r.brad * (1.f + kSafMargin)) continue;
        local32(r, o, xs);
        if (contains32(r, xs)) return j;
    }
    return -1;
}

// The lowest-index daughter of v other than `skip` whose closed solid holds
// the point x (v's frame), -1 if none: the candidates of the FP32 tests are
// tested in FP64 in index order (as Contains in queries.cuh).  The FP64 test
// sits outside the candidate search, so the lanes of a warp take it together
// instead of once for every daughter at which one of them stops.
__device__ __forceinline__ int first_containing(const VolView& v, const double* x, int skip, double* xl) {
    const float p32[3] = {f64_to_f32_trunc(x[0]), f64_to_f32_trunc(x[1]), f64_to_f32_trunc(x[2])};
    for (int j = next_candidate(v, p32, skip, 0); j >= 0; j = next_candidate(v, p32, skip, j + 1)) {
        const ShapeRec64& r64 = v.d64[j];
        point_to_local64(r64, x[0], x[1], x[2], xl);
        if (contains64(r64, xl)) return j;
    }
    return -1;
}

// Down from `node` (x in its frame) while a daughter contains the point.
static __device__ int world_descend(const WorldView& w, int node, double* x) {
    for (int level = 0; level < kMaxWorldDepth; ++level) {
        double xn[3];
        const int next = first_containing(w.vols[w.lv[node]], x, -1, xn);
        if (next < 0) return node;
        node = w.first[node] + next;
        x[0] = xn[0];
        x[1] = xn[1];
        x[2] = xn[2];
    }
    return node;
}

// Relocation after the step; b is the boundary point in node's frame.
static __device__ void world_relocate(const WorldView& w, int node, int hit, double* b, int& nout, int& fout) {
    const VolView& v = w.vols[w.lv[node]];
    if (hit >= 0) {
        double xl[3];
        point_to_local64(v.d64[hit], b[0], b[1], b[2], xl);
        nout = world_descend(w, w.first[node] + hit, xl);
        fout = -2;
        return;
    }
    int m = node;
    for (int level = 0; level < kMaxWorldDepth && m != 0; ++level) {
        const int P = w.parent[m], left = w.slot[m];
        const VolView& vp = w.vols[w.lv[P]];
        const ShapeRec64& rl = vp.d64[left];
        double xp[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            xp[k] = FMA(rl.R[3 * k], b[0], FMA(rl.R[3 * k + 1], b[1], FMA(rl.R[3 * k + 2], b[2], rl.t[k])));
        double xl[3];
        const int j = first_containing(vp, xp, left, xl);
        if (j >= 0) {
            nout = world_descend(w, w.first[P] + j, xl);
            fout = -2;
            return;
        }
        if (contains64(vp.m64, xp)) {
            nout = P;
            fout = left;
            return;
        }
        b[0] = xp[0];
        b[1] = xp[1];
        b[2] = xp[2];
        m = P;
    }
    nout = -1;   // left the root
    fout = -1;
}

// The step of Fig. 1 in one logical volume with the world flags, all FP64:
// mother first, daughters in index order, strict '<'; the daughter `skip`
// just left takes its re-entry distance.  Out of line: in the filter path
// it is the rare fallback, and inlined its FP64 code spilled registers of
// the FP32 pass (world step 0.368 -> 0.364 ms).
static __device__ __noinline__ void world_nav64(const VolView& v, const double* x, const double* u, int skip,
                                                bool entered, double& best, int& h) {
    if (!valid_track(x[0], x[1], x[2], u[0], u[1], u[2])) {
        best = d_nan();
        h = -2;
        return;
    }
    if (!entered && !contains64(v.m64, x)) {
        best = 0.0;
        h = -2;
        return;
    }
    best = dist_in64(v.m64, x, u);
    h = -1;
    const double dd = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double dn = sqrt(dd);
    for (int j = 0; j < v.nd; ++j) {
        const ShapeRec64& r = v.d64[j];
        const double w0 = r.t[0] - x[0], w1 = r.t[1] - x[1], w2 = r.t[2] - x[2];
        const double proj = w0 * u[0] + w1 * u[1] + w2 * u[2];
        const double rb = r.brad * dn;
        if (proj + rb < 0.0) continue;
        if (proj - rb >= best * dd) continue;
        const double ww = w0 * w0 + w1 * w1 + w2 * w2;
        if (ww * dd - proj * proj > rb * rb) continue;
        double xl[3], ul[3];
        to_local64(r, x[0], x[1], x[2], u[0], u[1], u[2], xl, ul);
        const double s = j == skip ? reentry64(r, xl, ul) : dist_out64(r, xl, ul);
        if (LT(s, best)) {
            best = s;
            h = j;
        }
    }
}

// The same answer with the FP32 filter: bounds for every daughter but
// `skip`, FP64 refinement of the candidates, then `skip`'s re-entry distance
// merged with the order of the sequential loop.  A track whose candidate
// list overflowed takes the FP64 loop.  In three parts, so that the kernel can
// run the first FP64 evaluation of many tracks binned by solid kind:
// world_pass1 (FP32; st.status 1: best/h final), the first task's FP64 value
// (eval64 of first_task(st)), world_finish (s_re: the re-entry distance of
// `skip` when the caller has it already).
static __device__ __forceinline__ void world_pass1(const VolView& v, const double* x, const double* u, int skip,
                                                   bool entered, RefineState& st, double& best, int& h) {
    st.status = 1;
    st.c.n = 0;
    st.c.dropped = f_inf();
#pragma unroll
    for (int k = 0; k < kCand; ++k) {
        st.c.L[k] = f_inf();
        st.c.j[k] = 0;
    }
    st.Lm = 0.f;
    if (!valid_track(x[0], x[1], x[2], u[0], u[1], u[2])) {
        best = d_nan();
        h = -2;
        return;
    }
    const float p32[3] = {f64_to_f32_trunc(x[0]), f64_to_f32_trunc(x[1]), f64_to_f32_trunc(x[2])};
    const float d32[3] = {f64_to_f32_trunc(u[0]), f64_to_f32_trunc(u[1]), f64_to_f32_trunc(u[2])};
    const float dd = fmaf(d32[0], d32[0], fmaf(d32[1], d32[1], d32[2] * d32[2]));
    if (!(dd > 1e-30f && dd < 1e30f)) {
        world_nav64(v, x, u, skip, entered, best, h);
        return;
    }
    const float inv_dd = __frcp_rn(dd);
    const float inv_dn = rsqrtf(dd) * (1.f + 4.f * kEps32f);
    bool in_shrunk;
    const float e_lo = exit32(v.m32, p32, d32, in_shrunk);
    const bool inside = in_shrunk || entered || contains64_cold<true>(v.m64, x[0], x[1], x[2]);
    if (!inside) {
        best = 0.0;
        h = -2;
        return;
    }
    st.Lm = in_shrunk ? fmaxf(lower_bound(e_lo, v.m32.delta, inv_dn), 0.f) : 0.f;
    bool dummy;
    const float e_hi = exit32(v.m32u, p32, d32, dummy);
    const float Um = e_hi + 16.f * kEps32f * e_hi + v.m32u.delta * inv_dn;
    for (int j = 0; j < v.nd; ++j)
        if (j != skip) bound_daughter(v.d32[j], j, p32, d32, inv_dd, inv_dn, Um, st.c);
    st.status = 0;
}

static __device__ __forceinline__ void world_finish(const VolView& v, const double* x, const double* u, int skip,
                                                    bool entered, const RefineState& st, double s1, double& best,
                                                    int& h, const double* s_re = nullptr) {
    if (!refine_fast(st, s1, best, h)) {
        int nev;
        refine_rest(v, v.d64, st, s1, x[0], x[1], x[2], u[0], u[1], u[2], best, h, nev);
        if (nev >= 1000) {   // the candidate list overflowed: the loop over every daughter
            world_nav64(v, x, u, skip, entered, best, h);
            return;
        }
    }
    if (skip >= 0) {
        double s;
        if (s_re) {
            s = *s_re;
        } else {
            const ShapeRec64& r = v.d64[skip];
            double xl[3], ul[3];
            to_local64(r, x[0], x[1], x[2], u[0], u[1], u[2], xl, ul);
            s = reentry64(r, xl, ul);
        }
        if (LT(s, best) || (BITS(s) == BITS(best) && h >= 0 && skip < h)) {
            best = s;
            h = skip;
        }
    }
}

}  // namespace geonav
