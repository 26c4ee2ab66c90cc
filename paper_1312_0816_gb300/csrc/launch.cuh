// launch.cuh -- grid sizing for the persistent grid-stride kernels: as many
// resident 256-thread blocks as the SMs hold (a multiple of the SM count),
// never more blocks than tiles of 256 tracks.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace geonav {

template <typename K>
static inline int blocks_for(K kernel, int64_t n, int smem, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t need = (n + 255) / 256;
    const int64_t cap = int64_t(per_sm) * num_sms;
    return int(need < cap ? need : cap);
}

template <typename K>
static inline cudaError_t prep(K kernel, int smem) {
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return cudaSuccess;
}

}  // namespace geonav
