// world.cu -- kernels of the geometry tree: Locate, and the step followed by
// final localisation (the per-track routines are in world.cuh).  Grid-stride
// over the tracks (the filtered step by tiles of 256); the volumes' tables
// are read through L1.
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
#include "refine_kernel.cuh"
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

// The plain FP64 step (GEO_FP64), one thread per track over the grouped
// order.  Three resident blocks per SM (80 registers, some spills) instead of
// two at 124 (measured on the filtered step when it ran this way: 0.44 ->
// 0.41 ms on the toy world).
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
            world_nav64(v, x, u, skip, entered, best, h);
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

// The filtered step (GEO_FP32_REFINE) by tiles of 256 tracks of the grouped
// order, with the FP64 evaluations every track needs binned by solid kind:
// the FP32 pass per track; then each track's first FP64 task and, after it
// left a daughter, that daughter's re-entry distance, run by whole warps over
// the binned list (32 tasks of one kind each: a warp pays for every code path
// its lanes take); then per track the rest of the refinement, the merge of
// the re-entry and the relocation.  The same answers as one thread per track
// (the same routines on the same values).  Toy world, the bench's four
// states: 0.366 ms per step with one thread per track, 0.350 with the first
// tasks binned, 0.332 with the re-entries binned too (two blocks per SM
// instead of three: 0.401).
constexpr int kWorldTile = 256;
struct WorldTile {
    double x[3][kWorldTile];   // the track in its node's frame
    double u[3][kWorldTile];
    double s1[kWorldTile];     // the first task's FP64 value (a final answer's step)
    float L[kCand][kWorldTile];
    int j[kCand][kWorldTile];
    float Lm[kWorldTile];
    float dropped[kWorldTile];
    int n[kWorldTile];         // candidate count; -1: the FP32 pass's answer is final
    int h[kWorldTile];         // a final answer's hit
    int lv[kWorldTile];        // logical volume
    double sre[kWorldTile];    // the re-entry distance of the daughter just left
    int task[2 * kWorldTile + 256];   // binned tasks (8 bins, each padded to a multiple of 32)
    int cnt[8];                       // bins 0-3: first tasks by kind, 4-7: re-entries by kind
    int next;                         // the next chunk of 32 tasks to claim
};

// start of bin `bin` of the tile's task list
__device__ __forceinline__ int bin_start8(const int* cnt, int bin) {
    int start = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (q < bin) start += (cnt[q] + 31) & ~31;
    return start;
}
constexpr int kReentryTask = 1 << 30;   // task flag: the re-entry of the daughter just left

__global__ void __launch_bounds__(kWorldTile, 3)
    k_world_step_binned(WorldView w, Basket b, const int32_t* __restrict__ perm, const int32_t* __restrict__ node_in,
                        const int32_t* __restrict__ flag_in, double* __restrict__ step,
                        int32_t* __restrict__ node_out, int32_t* __restrict__ flag_out) {
    __shared__ WorldTile T;
    const int t = threadIdx.x, lane = t & 31;
    const int64_t ntiles = (b.n + kWorldTile - 1) / kWorldTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t q = tile * kWorldTile + t;
        int bin = -1, task = 0, bin2 = -1, task2 = 0;
        {
            // FP32 pass of this thread's track
            const bool live = q < b.n;
            const int64_t i = live ? (perm ? perm[q] : q) : 0;
            const int node = live ? node_in[i] : -1;
            const int flag = live && flag_in ? flag_in[i] : -1;
            RefineState st;
            st.status = 1;
            double best = d_nan(), x[3] = {0, 0, 0}, u[3] = {0, 0, 0};
            int h = -2, lvi = 0;
            if (live && node >= 0 && node < w.nnodes) {
                world_to_node(w.xf + 12 * size_t(node), b.x[i], b.y[i], b.z[i], b.dx[i], b.dy[i], b.dz[i], x, u);
                lvi = w.lv[node];
                const VolView& v = w.vols[lvi];
                world_pass1(v, x, u, flag >= 0 && flag < v.nd ? flag : -1, flag == -2, st, best, h);
                if (st.status == 0) {
                    task = first_task(st);
                    bin = task < 0 ? 0 : kind_bin(v.d64[task].kind);
                    if (flag >= 0 && flag < v.nd) {
                        task2 = flag;
                        bin2 = 4 + kind_bin(v.d64[flag].kind);
                    }
                }
            }
            __syncthreads();   // the previous tile's tracks are done with the tile's memory
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T.x[k][t] = x[k];
                T.u[k][t] = u[k];
            }
#pragma unroll
            for (int c = 0; c < kCand; ++c) {
                T.L[c][t] = st.c.L[c];
                T.j[c][t] = st.c.j[c];
            }
            T.Lm[t] = st.Lm;
            T.dropped[t] = st.c.dropped;
            T.n[t] = st.status == 0 ? st.c.n : -1;
            T.s1[t] = best;
            T.h[t] = h;
            T.lv[t] = lvi;
            if (t < 8) T.cnt[t] = 0;
            if (t == 8) T.next = 0;
        }
        __syncthreads();
        const int slot = bin >= 0 ? atomicAdd(&T.cnt[bin], 1) : 0;
        const int slot2 = bin2 >= 0 ? atomicAdd(&T.cnt[bin2], 1) : 0;
        __syncthreads();
        if (bin >= 0) T.task[bin_start8(T.cnt, bin) + slot] = t | ((task + 1) << kOwnerBits);
        if (bin2 >= 0) T.task[bin_start8(T.cnt, bin2) + slot2] = kReentryTask | t | ((task2 + 1) << kOwnerBits);
        {   // -1 between the bins (each starts on a multiple of 32)
            const int bb = t >> 5, c = T.cnt[bb];
            if ((t & 31) < ((c + 31) & ~31) - c) T.task[bin_start8(T.cnt, bb) + c + (t & 31)] = -1;
        }
        __syncthreads();
        // the first FP64 tasks and the re-entries, 32 of one kind per warp
        const int total = bin_start8(T.cnt, 8);
        for (;;) {
            int q0 = 0;
            if (lane == 0) q0 = atomicAdd(&T.next, 32);
            q0 = __shfl_sync(0xffffffffu, q0, 0);
            if (q0 >= total) break;
            const int e = T.task[q0 + lane];
            if (e >= 0) {
                const int o = e & ((1 << kOwnerBits) - 1), jj = ((e & ~kReentryTask) >> kOwnerBits) - 1;
                const VolView& v = w.vols[T.lv[o]];
                if (e & kReentryTask) {
                    const ShapeRec64& r = v.d64[jj];
                    double xl[3], ul[3];
                    to_local64(r, T.x[0][o], T.x[1][o], T.x[2][o], T.u[0][o], T.u[1][o], T.u[2][o], xl, ul);
                    T.sre[o] = reentry64(r, xl, ul);
                } else {
                    T.s1[o] = eval64(v, v.d64, jj, T.x[0][o], T.x[1][o], T.x[2][o], T.u[0][o], T.u[1][o], T.u[2][o]);
                }
            }
        }
        __syncthreads();
        // the rest of each track: refinement, re-entry, relocation
        if (q < b.n) {
            const int64_t i = perm ? perm[q] : q;
            const int node = node_in[i];
            const int flag = flag_in ? flag_in[i] : -1;
            double best = d_nan();
            int nout = -2, fout = -1;
            if (node >= 0 && node < w.nnodes) {
                const double x[3] = {T.x[0][t], T.x[1][t], T.x[2][t]}, u[3] = {T.u[0][t], T.u[1][t], T.u[2][t]};
                int h = T.h[t];
                best = T.s1[t];
                if (T.n[t] >= 0) {
                    const VolView& v = w.vols[T.lv[t]];
                    RefineState st;
                    st.status = 0;
                    st.c.n = T.n[t];
#pragma unroll
                    for (int c = 0; c < kCand; ++c) {
                        st.c.L[c] = T.L[c][t];
                        st.c.j[c] = T.j[c][t];
                    }
                    st.c.dropped = T.dropped[t];
                    st.Lm = T.Lm[t];
                    const double s1 = best;
                    world_finish(v, x, u, flag >= 0 && flag < v.nd ? flag : -1, flag == -2, st, s1, best, h, &T.sre[t]);
                }
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
        k_world_step<<<blocks_for(k_world_step, b.n, 0, num_sms), 256, 0, s>>>(w, b, perm, node_in, flag_in, step,
                                                                            node_out, flag_out);
    else
        k_world_step_binned<<<blocks_for(k_world_step_binned, b.n, 0, num_sms), kWorldTile, 0, s>>>(
            w, b, perm, node_in, flag_in, step, node_out, flag_out);
    return cudaGetLastError();
}

}  // namespace geonav
