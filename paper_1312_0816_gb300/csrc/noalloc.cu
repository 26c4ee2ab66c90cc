// noalloc.cu -- a navigator entry point for callers that must not allocate
// device memory.
//
// Some programs cannot let a library call cudaMalloc once they are running:
// an application whose framework owns all device memory through its own
// allocator, or a real-time pipeline that forbids allocation after start-up
// so that a step can neither fail for lack of memory nor stall the device
// (cudaMalloc and cudaFree synchronise it).  For them,
// geo_dist_to_boundary_batched_noalloc runs the batched persistent launch
// with its scratch -- the tile list, the per-volume views, the tile counter
// and the status word -- in one fixed array of device memory that belongs to
// this library (NoAllocScratch below, about 0.55 MB, held on every device
// that loads the library until the process exits).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "geo_internal.h"

using namespace geonav;

namespace {

constexpr int kNoAllocMaxVolumes = 64;
constexpr int kNoAllocMaxTiles = 32768;   // tiles of at most kTileTracks tracks

struct NoAllocScratch {
    VolView vols[kNoAllocMaxVolumes];
    BatchTile tiles[kNoAllocMaxTiles];
    unsigned int words[4];   // [0] tile counter, [1] status word
};

// The scratch itself.  In host code `g_noalloc_scratch` is only a stand-in
// for the symbol, not a device address: its device address is obtained once
// per device with cudaGetSymbolAddress and cached in g_dev_ptr.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoAllocScratch* g_dev_ptr[kMaxDevices] = {nullptr};
BatchTile g_host_tiles[kNoAllocMaxTiles];   // host staging of the tile list (under g_mu)

// Device address of the scratch on the current device (set-up on first use).
geo_status scratch_on(int dev, NoAllocScratch** out) {
    if (dev < 0 || dev >= kMaxDevices) return GEO_ERR_UNSUPPORTED;
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GEO_ERR_CUDA;
        }
        g_dev_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_dev_ptr[dev];
    return GEO_OK;
}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" geo_status geo_dist_to_boundary_batched_noalloc(const geo_volume* vols, int32_t n_vols,
                                                          const geo_basket* baskets, int32_t n_baskets,
                                                          const double* x, const double* y, const double* z,
                                                          const double* dx, const double* dy, const double* dz,
                                                          int64_t n_total, double* step, int32_t* hit,
                                                          void* stream) {
    if (!vols || n_vols <= 0 || n_baskets < 0 || (n_baskets > 0 && !baskets) || n_total < 0)
        return GEO_ERR_INVALID_ARG;
    if (n_vols > kNoAllocMaxVolumes) return GEO_ERR_INVALID_ARG;   // beyond the scratch
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GEO_ERR_CUDA;
    for (int i = 0; i < n_vols; ++i)
        if (!vols[i] || volume_device(vols[i]) != dev) return GEO_ERR_INVALID_ARG;
    int64_t ntiles = 0;
    for (int k = 0; k < n_baskets; ++k) {
        const geo_basket& bk = baskets[k];
        if (bk.reserved != 0 || bk.volume < 0 || bk.volume >= n_vols || bk.offset < 0 || bk.count < 0 ||
            bk.offset + bk.count > n_total)
            return GEO_ERR_INVALID_ARG;
        ntiles += (bk.count + kTileTracks - 1) / kTileTracks;
    }
    if (ntiles > kNoAllocMaxTiles) return GEO_ERR_INVALID_ARG;     // beyond the scratch
    if (ntiles == 0) return GEO_OK;
    if (!on_device(x) || !on_device(y) || !on_device(z) || !on_device(dx) || !on_device(dy) || !on_device(dz) ||
        !on_device(step) || !on_device(hit))
        return GEO_ERR_INVALID_ARG;

    std::lock_guard<std::mutex> lock(g_mu);
    NoAllocScratch* d = nullptr;
    geo_status st = scratch_on(dev, &d);
    if (st != GEO_OK) return st;
    // tiles of at most kTileTracks tracks, largest estimated cost (tracks x daughters) first
    int64_t m = 0;
    for (int k = 0; k < n_baskets; ++k) {
        const geo_basket& bk = baskets[k];
        for (int64_t off = 0; off < bk.count; off += kTileTracks) {
            BatchTile& t = g_host_tiles[m++];
            t.vol = bk.volume;
            t.count = int32_t(std::min<int64_t>(kTileTracks, bk.count - off));
            t.base = bk.offset + off;
        }
    }
    std::stable_sort(g_host_tiles, g_host_tiles + m, [&](const BatchTile& a, const BatchTile& b) {
        return int64_t(a.count) * (volume_view(vols[a.vol])->nd + 1) >
               int64_t(b.count) * (volume_view(vols[b.vol])->nd + 1);
    });
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    // Copies from pageable host memory: the runtime has read the source (into
    // its staging memory) when such a call returns, so the shared host tile
    // list can be rewritten by the next call; it also waits for the work
    // already queued on the stream before it starts the copy, so this call may
    // block the host until then.
    for (int i = 0; i < n_vols && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(&d->vols[i], volume_view(vols[i]), sizeof(VolView), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d->tiles, g_host_tiles, sizeof(BatchTile) * size_t(m), cudaMemcpyHostToDevice, s);
    // the counter and the status word must start at zero on every call
    if (e == cudaSuccess) e = cudaMemsetAsync(d->words, 0, sizeof(d->words), s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GEO_ERR_OOM : GEO_ERR_CUDA;
    BatchView bv;
    bv.vols = d->vols;
    bv.tiles = d->tiles;
    bv.ntiles = m;
    bv.counter = &d->words[0];
    bv.status = &d->words[1];
    bv.segs = 0;
    bv.nvols = n_vols;
    bv.vox = 0;
    bv.pad_ = 0;
    bv.idx = nullptr;   // plain tiles only
    for (int i = 0; i < n_vols; ++i) {
        bv.segs = bv.segs || volume_view(vols[i])->segs;
        bv.vox = bv.vox || volume_view(vols[i])->voxelized;
    }
    const Basket bk{x, y, z, dx, dy, dz, n_total};
    e = launch_dist_batched(bv, bk, step, hit, 0, kTileTracks, s, sm_count(dev));
    return e == cudaSuccess ? GEO_OK : GEO_ERR_CUDA;
}
