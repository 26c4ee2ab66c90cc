// world_abi.cu -- host side of the geometry tree: validation, breadth-first
// expansion of the placed volumes with their world transforms, upload, and
// the C ABI entry points (include/geo.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "geo_internal.h"
#include "world.cuh"

using namespace geonav;

// ------------------------------------------------------------------ host ---

struct geo_world_s {
    int device = 0;
    int32_t nnodes = 0;
    int32_t max_depth = 0;
    int32_t nlv = 0;
    // grouping scratch of geo_world_step (grown on demand)
    int32_t* d_cnt = nullptr;
    int32_t* d_perm = nullptr;
    int64_t perm_cap = 0;
    std::mutex mu;
    std::vector<int32_t> h_lv, h_parent, h_slot, h_first;
    VolView* d_vols = nullptr;
    int32_t* d_node = nullptr;   // lv | parent | slot | first, nnodes each
    double* d_xf = nullptr;
};

namespace {

geo_status world_cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GEO_OK;
    if (e == cudaErrorMemoryAllocation) return GEO_ERR_OOM;
    return GEO_ERR_CUDA;
}

bool device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

WorldView world_view(const geo_world_s* w) {
    WorldView v;
    v.vols = w->d_vols;
    v.lv = w->d_node;
    v.parent = w->d_node + w->nnodes;
    v.slot = w->d_node + 2 * size_t(w->nnodes);
    v.first = w->d_node + 3 * size_t(w->nnodes);
    v.xf = w->d_xf;
    v.nnodes = w->nnodes;
    return v;
}

geo_status world_check(geo_world w) {
    if (!w) return GEO_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    return dev == w->device ? GEO_OK : GEO_ERR_INVALID_ARG;
}

}  // namespace

extern "C" {

geo_status geo_build_world(const geo_volume* volumes, int32_t n_volumes, const int32_t* child, int32_t root,
                           void* stream, geo_world* out) {
    if (!out) return GEO_ERR_INVALID_ARG;
    *out = nullptr;
    if (!volumes || n_volumes <= 0 || root < 0 || root >= n_volumes) return GEO_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    std::vector<int64_t> off(static_cast<size_t>(n_volumes) + 1, 0);
    for (int v = 0; v < n_volumes; ++v) {
        if (!volumes[v] || volume_device(volumes[v]) != dev) return GEO_ERR_INVALID_ARG;
        off[v + 1] = off[v] + volume_view(volumes[v])->nd;
    }
    if (off[n_volumes] > 0 && !child) return GEO_ERR_INVALID_ARG;
    // every daughter is an instance of a logical volume whose mother solid is
    // that daughter's solid
    for (int v = 0; v < n_volumes; ++v) {
        const ShapeRec64* d = volume_host_daughters(volumes[v]);
        for (int j = 0; j < volume_view(volumes[v])->nd; ++j) {
            const int c = child[off[v] + j];
            if (c < 0 || c >= n_volumes) return GEO_ERR_INVALID_ARG;
            const ShapeRec64& m = volume_view(volumes[c])->m64;
            if (m.kind != d[j].kind || std::memcmp(m.p, d[j].p, sizeof m.p) != 0) return GEO_ERR_SHAPE_PARAMS;
            if (m.kind == KPCON) {   // and the same planes
                const double *a = volume_host_table(volumes[c], -1), *b = volume_host_table(volumes[v], j);
                if (!a || !b || std::memcmp(a, b, sizeof(double) * 3 * size_t(m.d[1])) != 0)
                    return GEO_ERR_SHAPE_PARAMS;
            }
        }
    }
    // breadth-first expansion with world transforms
    std::vector<int32_t> lv{root}, parent{-1}, slot{-1}, first, depth{0};
    std::vector<double> xf = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
    int32_t maxd = 0;
    for (size_t head = 0; head < lv.size(); ++head) {
        const int v = lv[head];
        first.push_back(int32_t(lv.size()));
        const ShapeRec64* d = volume_host_daughters(volumes[v]);
        const int nd = volume_view(volumes[v])->nd;
        if (nd > 0 && depth[head] + 1 > kMaxWorldDepth) return GEO_ERR_INVALID_ARG;
        if (int64_t(lv.size()) + nd > kMaxWorldNodes) return GEO_ERR_INVALID_ARG;
        double G[12];
        std::copy(xf.begin() + 12 * head, xf.begin() + 12 * head + 12, G);
        for (int j = 0; j < nd; ++j) {
            const double* R = d[j].R;
            const double* t = d[j].t;
            double Rc[9], tc[3];
            for (int a = 0; a < 3; ++a) {
                for (int bb = 0; bb < 3; ++bb)
                    Rc[3 * a + bb] = G[3 * a] * R[bb] + G[3 * a + 1] * R[3 + bb] + G[3 * a + 2] * R[6 + bb];
                tc[a] = G[3 * a] * t[0] + G[3 * a + 1] * t[1] + G[3 * a + 2] * t[2] + G[9 + a];
            }
            lv.push_back(child[off[v] + j]);
            parent.push_back(int32_t(head));
            slot.push_back(j);
            depth.push_back(depth[head] + 1);
            maxd = std::max(maxd, depth[head] + 1);
            xf.insert(xf.end(), Rc, Rc + 9);
            xf.insert(xf.end(), tc, tc + 3);
        }
    }
    geo_world w = lib_new<geo_world_s>();
    if (!w) return GEO_ERR_OOM;
    w->device = dev;
    w->nlv = n_volumes;
    w->nnodes = int32_t(lv.size());
    w->max_depth = maxd;
    w->h_lv = lv;
    w->h_parent = parent;
    w->h_slot = slot;
    w->h_first = first;
    std::vector<VolView> views(static_cast<size_t>(n_volumes));
    for (int v = 0; v < n_volumes; ++v) views[v] = *volume_view(volumes[v]);
    std::vector<int32_t> node(static_cast<size_t>(4) * w->nnodes);
    std::copy(lv.begin(), lv.end(), node.begin());
    std::copy(parent.begin(), parent.end(), node.begin() + w->nnodes);
    std::copy(slot.begin(), slot.end(), node.begin() + 2 * size_t(w->nnodes));
    std::copy(first.begin(), first.end(), node.begin() + 3 * size_t(w->nnodes));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = lib_malloc(&w->d_vols, sizeof(VolView) * views.size())) != cudaSuccess ||
        (e = lib_malloc(&w->d_node, sizeof(int32_t) * node.size())) != cudaSuccess ||
        (e = lib_malloc(&w->d_xf, sizeof(double) * xf.size())) != cudaSuccess ||
        (e = cudaMemcpyAsync(w->d_vols, views.data(), sizeof(VolView) * views.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(w->d_node, node.data(), sizeof(int32_t) * node.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(w->d_xf, xf.data(), sizeof(double) * xf.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        geo_destroy_world(w);
        return world_cuda_status(e);
    }
    *out = w;
    return GEO_OK;
}

geo_status geo_destroy_world(geo_world w) {
    if (!w) return GEO_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != w->device) cudaSetDevice(w->device);
    cudaDeviceSynchronize();
    cudaFree(w->d_vols);
    cudaFree(w->d_node);
    cudaFree(w->d_xf);
    cudaFree(w->d_cnt);
    cudaFree(w->d_perm);
    if (prev >= 0 && prev != w->device) cudaSetDevice(prev);
    delete w;
    return GEO_OK;
}

geo_status geo_world_info(geo_world w, int32_t* n_nodes, int32_t* max_depth) {
    if (!w) return GEO_ERR_INVALID_ARG;
    if (n_nodes) *n_nodes = w->nnodes;
    if (max_depth) *max_depth = w->max_depth;
    return GEO_OK;
}

geo_status geo_world_nodes(geo_world w, int32_t* lv, int32_t* parent, int32_t* slot, int32_t* first_child) {
    if (!w) return GEO_ERR_INVALID_ARG;
    if (lv) std::copy(w->h_lv.begin(), w->h_lv.end(), lv);
    if (parent) std::copy(w->h_parent.begin(), w->h_parent.end(), parent);
    if (slot) std::copy(w->h_slot.begin(), w->h_slot.end(), slot);
    if (first_child) std::copy(w->h_first.begin(), w->h_first.end(), first_child);
    return GEO_OK;
}

geo_status geo_world_locate(geo_world w, const double* x, const double* y, const double* z, int64_t n,
                            int32_t* node, void* stream) {
    geo_status st = world_check(w);
    if (st != GEO_OK) return st;
    if (n < 0) return GEO_ERR_INVALID_ARG;
    if (n == 0) return GEO_OK;
    if (!device_ptr(x) || !device_ptr(y) || !device_ptr(z) || !device_ptr(node)) return GEO_ERR_INVALID_ARG;
    const Basket b{x, y, z, nullptr, nullptr, nullptr, n};
    return world_cuda_status(
        launch_world_locate(world_view(w), b, node, static_cast<cudaStream_t>(stream), sm_count(w->device)));
}

geo_status geo_world_step(geo_world w, const double* x, const double* y, const double* z, const double* dx,
                          const double* dy, const double* dz, int64_t n, const int32_t* node_in,
                          const int32_t* flag_in, double* step, int32_t* node_out, int32_t* flag_out, int32_t mode,
                          void* stream) {
    geo_status st = world_check(w);
    if (st != GEO_OK) return st;
    if (mode != GEO_FP64 && mode != GEO_FP32_REFINE) return GEO_ERR_INVALID_ARG;
    if (n < 0) return GEO_ERR_INVALID_ARG;
    if (n == 0) return GEO_OK;
    if (!device_ptr(x) || !device_ptr(y) || !device_ptr(z) || !device_ptr(dx) || !device_ptr(dy) ||
        !device_ptr(dz) || !device_ptr(node_in) || !device_ptr(step) || !device_ptr(node_out) ||
        (flag_in && !device_ptr(flag_in)) || (flag_out && !device_ptr(flag_out)))
        return GEO_ERR_INVALID_ARG;
    const Basket b{x, y, z, dx, dy, dz, n};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = sm_count(w->device);
    std::lock_guard<std::mutex> lock(w->mu);
    if (n > w->perm_cap) {
        // grow the grouping scratch (the only allocation of the call)
        cudaError_t e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return world_cuda_status(e);
        cudaFree(w->d_perm);
        cudaFree(w->d_cnt);
        w->d_perm = nullptr;
        w->d_cnt = nullptr;
        w->perm_cap = 0;
        if ((e = lib_malloc(&w->d_perm, sizeof(int32_t) * size_t(n))) != cudaSuccess ||
            (e = lib_malloc(&w->d_cnt, sizeof(int32_t) * (size_t(w->nlv) + 1))) != cudaSuccess)
            return world_cuda_status(e);
        w->perm_cap = n;
    }
    const WorldView wv = world_view(w);
    cudaError_t e = launch_world_group(wv, n, node_in, w->nlv, w->d_cnt, w->d_perm, s, sms);
    if (e != cudaSuccess) return world_cuda_status(e);
    return world_cuda_status(launch_world_step(wv, b, w->d_perm, node_in, flag_in, step, node_out, flag_out, mode, s,
                                               sms));
}

}  // extern "C"
