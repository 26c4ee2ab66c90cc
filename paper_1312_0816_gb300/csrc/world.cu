// world.cu -- kernels of the geometry tree: Locate, and the step followed by
// final localisation (the per-track routines are in world.cuh).  One thread
// per track, grid-stride; the volumes' tables are read through L1.
#include <cuda_runtime.h>

#include "launch.cuh"
#include "world.cuh"

namespace geonav {

template <int MODE>
__global__ void __launch_bounds__(256) k_world_step(WorldView w, Basket b, const int32_t* __restrict__ node_in,
                                                    const int32_t* __restrict__ flag_in, double* __restrict__ step,
                                                    int32_t* __restrict__ node_out, int32_t* __restrict__ flag_out) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        const int node = node_in[i];
        const int flag = flag_in ? flag_in[i] : -1;
        double best = d_nan();
        int nout = -2, fout = -1;
        if (node >= 0 && node < w.nnodes) {
            double x[3], u[3];
            world_to_node(w.xf + 12 * size_t(node), b.x[i], b.y[i], b.z[i], b.dx[i], b.dy[i], b.dz[i], x, u);
            const VolView& v = w.vols[w.lv[node]];
            const int skip = flag >= 0 && flag < v.nd ? flag : -1;
            const bool entered = flag == -2;
            int h;
            if (MODE == GEO_FP64) world_nav64(v, x, u, skip, entered, best, h);
            else world_refine(v, x, u, skip, entered, best, h);
            if (h >= -1) {
                double bp[3] = {FMA(best, u[0], x[0]), FMA(best, u[1], x[1]), FMA(best, u[2], x[2])};
                world_relocate(w, node, h, bp, nout, fout);
            }
        }
        step[i] = best;
        node_out[i] = nout;
        if (flag_out) flag_out[i] = fout;
    }
}

__global__ void __launch_bounds__(256) k_world_locate(WorldView w, Basket b, int32_t* __restrict__ node) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < b.n; i += stride) {
        double x[3] = {b.x[i], b.y[i], b.z[i]};
        int n;
        if (!(finite64(x[0]) && finite64(x[1]) && finite64(x[2]))) n = -2;
        else if (!contains64(w.vols[w.lv[0]].m64, x)) n = -1;
        else n = world_descend(w, 0, x);
        node[i] = n;
    }
}


cudaError_t launch_world_locate(const WorldView& w, const Basket& b, int32_t* node, cudaStream_t s, int num_sms) {
    k_world_locate<<<blocks_for(k_world_locate, b.n, 0, num_sms), 256, 0, s>>>(w, b, node);
    return cudaGetLastError();
}

cudaError_t launch_world_step(const WorldView& w, const Basket& b, const int32_t* node_in, const int32_t* flag_in,
                              double* step, int32_t* node_out, int32_t* flag_out, int mode, cudaStream_t s,
                              int num_sms) {
    if (mode == GEO_FP64)
        k_world_step<GEO_FP64><<<blocks_for(k_world_step<GEO_FP64>, b.n, 0, num_sms), 256, 0, s>>>(
            w, b, node_in, flag_in, step, node_out, flag_out);
    else
        k_world_step<GEO_FP32_REFINE><<<blocks_for(k_world_step<GEO_FP32_REFINE>, b.n, 0, num_sms), 256, 0, s>>>(
            w, b, node_in, flag_in, step, node_out, flag_out);
    return cudaGetLastError();
}

}  // namespace geonav
