// Launchers of the plain sweep variants (FP64 Euclidean / p-norm, FP64 and
// FP32 z-normalised).
#pragma once

#include <cuda_runtime.h>

#include "mp_simple.cuh"

namespace mpk {

inline int *device_error_ptr() {
    void *p = nullptr;
    cudaGetSymbolAddress(&p, mp_device_error);
    return static_cast<int *>(p);
}

template <class V>
inline cudaError_t launch_simple(const TileGrid &g, const V &v, int B, cudaStream_t st) {
    if (g.tiles <= 0) return cudaSuccess;
    simple_sweep_kernel<V><<<static_cast<unsigned>(g.tiles), SM_NT, 0, st>>>(g, v, B);
    return cudaGetLastError();
}

}  // namespace mpk
