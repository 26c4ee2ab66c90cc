// shape_query.cu -- the elementary per-shape algorithms of Sec. 3.1 on their
// own (the vectorised DistFromOutside / DistFromInside / Safety / Contains of
// one solid that Fig. 2 measures per shape), for a basket of points or tracks.
//
// The solid's FP64 record travels in the kernel parameters (every lane reads
// the same constants), and so does a polycone's plane table (read through
// the address of the __grid_constant__ parameter, so the call allocates
// nothing); each thread takes one track, applies the placement's
// master->local transform and the FP64 routine of the navigator kernels
// (shapes64.cuh), so the values are the ones the navigator computes for that
// solid.  Grid-stride over the basket, blocks sized by occupancy.
#include <cuda_runtime.h>

#include "geo_internal.h"
#include "launch.cuh"
#include "nav_common.cuh"
#include "shapes64.cuh"

namespace geonav {

template <int WHAT>
__global__ void __launch_bounds__(256) k_shape(const __grid_constant__ ShapeArg a, Basket b, double* __restrict__ out,
                                               int32_t* __restrict__ face) {
    const ShapeRec64& r = a.r;
    const bool pc = r.kind == KPCON;
    const double* T = a.table;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const double px = b.x[i], py = b.y[i], pz = b.z[i];
        double v;
        int f = -1;
        if (WHAT == GEO_Q_DIST_OUT || WHAT == GEO_Q_DIST_IN) {
            const double qx = b.dx[i], qy = b.dy[i], qz = b.dz[i];
            if (!valid_track(px, py, pz, qx, qy, qz)) {
                v = d_nan();
            } else {
                double x[3], u[3];
                to_local64(r, px, py, pz, qx, qy, qz, x, u);
                if (WHAT == GEO_Q_DIST_OUT) {
                    v = pc ? pcon_out64_call<true, false>(r.d, T, x[0], x[1], x[2], u[0], u[1], u[2], &f)
                           : dist_out64<true>(r, x, u, &f);
                } else if (pc ? pcon_contains64(r.d, T, x[0], x[1], x[2]) : contains64(r, x)) {
                    v = pc ? pcon_in64_call<true>(r.d, T, x[0], x[1], x[2], u[0], u[1], u[2], &f)
                           : dist_in64<true>(r, x, u, &f);
                } else {
                    v = 0.0;   // DistFromInside of a point outside
                }
            }
        } else {
            const bool fin = finite64(px) && finite64(py) && finite64(pz);
            double x[3];
            point_to_local64(r, px, py, pz, x);
            const bool in = fin && (pc ? pcon_contains64(r.d, T, x[0], x[1], x[2]) : contains64(r, x));
            if (!fin) v = d_nan();
            else if (WHAT == GEO_Q_CONTAINS) v = in ? 1.0 : 0.0;
            else if (pc) v = in == (WHAT == GEO_Q_SAFETY_IN) ? pcon_safety64(r.d, T, x[0], x[1], x[2], in) : 0.0;
            else v = safety64(r, x, WHAT == GEO_Q_SAFETY_IN);
        }
        out[i] = v;
        if (face) face[i] = f;
    }
}

template <int WHAT>
static cudaError_t launch_shape_q(const ShapeArg& a, const Basket& b, double* out, int32_t* face, cudaStream_t s,
                                  int num_sms) {
    k_shape<WHAT><<<blocks_for(k_shape<WHAT>, b.n, 0, num_sms), 256, 0, s>>>(a, b, out, face);
    return cudaGetLastError();
}

cudaError_t launch_shape_query(const ShapeArg& a, int what, const Basket& b, double* out, int32_t* face,
                               cudaStream_t s, int num_sms) {
    switch (what) {
        case GEO_Q_DIST_OUT: return launch_shape_q<GEO_Q_DIST_OUT>(a, b, out, face, s, num_sms);
        case GEO_Q_DIST_IN: return launch_shape_q<GEO_Q_DIST_IN>(a, b, out, face, s, num_sms);
        case GEO_Q_SAFETY_OUT: return launch_shape_q<GEO_Q_SAFETY_OUT>(a, b, out, face, s, num_sms);
        case GEO_Q_SAFETY_IN: return launch_shape_q<GEO_Q_SAFETY_IN>(a, b, out, face, s, num_sms);
        case GEO_Q_CONTAINS: return launch_shape_q<GEO_Q_CONTAINS>(a, b, out, face, s, num_sms);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace geonav
