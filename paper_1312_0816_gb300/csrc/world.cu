// world.cu -- kernels of the geometry tree: Locate, and the step followed by
// final localisation (the per-track routines are in world.cuh).  One thread
// per track, grid-stride; the volumes' tables are read through L1.
//
// Before a step the tracks are grouped by the logical volume of their node
// (a counting sort of track indices: histogram, scan, scatter), and the step
// kernel takes them in that order, so that the lanes of a warp navigate the
// same volume: the daughter loops, the shape code and the relocation then
// diverge far less (a warp pays for every path its lanes take, and the FP64
// pipe charges a warp instruction whatever the number of active lanes).
// This is the basket of Sec. 2 -- tracks in the same logical volume --
// formed on the device.  The order within a group depends on atomics; the
// answer of a track does not depend on it.
#include <cuda_runtime.h>

#include "launch.cuh"
#include "world.cuh"

namespace geonav {

// group key of a track: its node's logical volume; invalid nodes last
__device__ __forceinline__ int world_key(const WorldView& w, int nlv, int node) {
    return node >= 0 && node < w.nnodes ? w.lv[node] : nlv;
}

// histogram of the keys: per block in shared memory (one global add per
// block and key) when the keys fit, else straight into global memory
constexpr int kHistSmemKeys = 8192;

template <bool SMEM>
__global__ void __launch_bounds__(256) k_world_hist(WorldView w, int64_t n, const int32_t* __restrict__ node_in,
                                                    int nkeys, int32_t* __restrict__ cnt) {
    extern __shared__ int32_t h_smem[];
    int32_t* h = SMEM ? h_smem : cnt;
    if (SMEM) {
        for (int k = threadIdx.x; k < nkeys; k += blockDim.x) h_smem[k] = 0;
        __syncthreads();
    }
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&h[world_key(w, nkeys - 1, node_in[i])], 1);
    if (SMEM) {
        __syncthreads();
        for (int k = threadIdx.x; k < nkeys; k += blockDim.x)
            if (h_smem[k]) atomicAdd(&cnt[k], h_smem[k]);
    }
}

// exclusive scan of nkeys counts in place, one block of 1024 threads: each
// thread scans a contiguous chunk, the chunk totals are scanned in shared
// memory, then added back
__global__ void __launch_bounds__(1024) k_world_scan(int nkeys, int32_t* __restrict__ cnt) {
    __shared__ int32_t tot[1024];
    const int t = threadIdx.x;
    const int chunk = (nkeys + 1023) / 1024;
    const int a = t * chunk, e = min(nkeys, a + chunk);
    int32_t sum = 0;
    for (int k = a; k < e; ++k) sum += cnt[k];
    tot[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = t >= off ? tot[t - off] : 0;
        __syncthreads();
        tot[t] += v;
        __syncthreads();
    }
    int32_t run = tot[t] - sum;   // exclusive prefix of this chunk
    for (int k = a; k < e; ++k) {
        const int32_t c = cnt[k];
        cnt[k] = run;
        run += c;
    }
}

// scatter the track indices to their group's next slots (one atomic per
// group of equal keys in a warp)
__global__ void __launch_bounds__(256) k_world_scatter(WorldView w, int64_t n, const int32_t* __restrict__ node_in,
                                                       int nkeys, int32_t* __restrict__ off,
                                                       int32_t* __restrict__ perm) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool live = i < n;
        const int key = live ? world_key(w, nkeys - 1, node_in[i]) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(same) - 1;
        int pos = 0;
        if (live && lane == leader) pos = atomicAdd(&off[key], __popc(same));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (live) perm[pos + __popc(same & ((1u << lane) - 1u))] = int32_t(i);
    }
}

// One thread per track over the grouped order.  Three resident blocks per SM
// (80 registers, some spills) instead of two at 124: the toy world's
// filtered step 0.44 -> 0.41 ms.
template <int MODE>
__global__ void __launch_bounds__(256, 3) k_world_step(WorldView w, Basket b, const int32_t* __restrict__ perm,
                                                    const int32_t* __restrict__ node_in,
                                                    const int32_t* __restrict__ flag_in, double* __restrict__ step,
                                                    int32_t* __restrict__ node_out, int32_t* __restrict__ flag_out) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < b.n; t += stride) {
        const int64_t i = perm ? perm[t] : t;
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

cudaError_t launch_world_group(const WorldView& w, int64_t n, const int32_t* node_in, int nlv, int32_t* cnt,
                               int32_t* perm, cudaStream_t s, int num_sms) {
    const int nkeys = nlv + 1;
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nkeys, s)) != cudaSuccess) return e;
    if (nkeys <= kHistSmemKeys) {
        const int hsmem = int(sizeof(int32_t)) * nkeys;
        k_world_hist<true><<<blocks_for(k_world_hist<true>, n, hsmem, num_sms), 256, hsmem, s>>>(w, n, node_in,
                                                                                                nkeys, cnt);
    } else {
        k_world_hist<false><<<blocks_for(k_world_hist<false>, n, 0, num_sms), 256, 0, s>>>(w, n, node_in, nkeys,
                                                                                          cnt);
    }
    k_world_scan<<<1, 1024, 0, s>>>(nkeys, cnt);
    k_world_scatter<<<blocks_for(k_world_scatter, n, 0, num_sms), 256, 0, s>>>(w, n, node_in, nkeys, cnt, perm);
    return cudaGetLastError();
}

cudaError_t launch_world_step(const WorldView& w, const Basket& b, const int32_t* perm, const int32_t* node_in,
                              const int32_t* flag_in, double* step, int32_t* node_out, int32_t* flag_out, int mode,
                              cudaStream_t s, int num_sms) {
    if (mode == GEO_FP64)
        k_world_step<GEO_FP64><<<blocks_for(k_world_step<GEO_FP64>, b.n, 0, num_sms), 256, 0, s>>>(
            w, b, perm, node_in, flag_in, step, node_out, flag_out);
    else
        k_world_step<GEO_FP32_REFINE><<<blocks_for(k_world_step<GEO_FP32_REFINE>, b.n, 0, num_sms), 256, 0, s>>>(
            w, b, perm, node_in, flag_in, step, node_out, flag_out);
    return cudaGetLastError();
}

}  // namespace geonav
