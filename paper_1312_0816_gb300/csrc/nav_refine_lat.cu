// nav_refine_lat.cu -- the refine kernel in its latency configuration (8
// producer + 4 consumer warps, tiles of 256 tracks) for baskets of at most
// two tiles per resident block; a translation unit of its own so that the
// two configurations compile in parallel.
#include "refine_kernel.cuh"

namespace geonav {

cudaError_t launch_dist_refine_latency(const VolView& v, const Basket& b, double* step, int32_t* hit,
                                       double* bpoint, int32_t* nref, cudaStream_t s, int num_sms) {
    return launch_refine_cfg<kLatProd, kLatCons>(v, b, step, hit, bpoint, nref, s, num_sms);
}

}  // namespace geonav
