// The generic FP32 sweep (any m the two-stream kernel does not take, real p,
// float64 input carried as hi + lo) for single series and batch queues.
#include "mp_kernels.h"

namespace mpk {

template <int KIND, bool SPLIT>
static cudaError_t launch(const SweepArgs &a, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<KIND, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sweep_kernel<KIND, SPLIT><<<static_cast<unsigned>(a.tiles), SW_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t generic_launch(int kind, bool split, const SweepArgs &a, size_t smem, cudaStream_t st) {
    switch (kind * 2 + (split ? 1 : 0)) {
        case 0: return launch<K_P2, false>(a, smem, st);
        case 1: return launch<K_P2, true>(a, smem, st);
        case 2: return launch<K_P1, false>(a, smem, st);
        case 3: return launch<K_P1, true>(a, smem, st);
        case 4: return launch<K_P3, false>(a, smem, st);
        case 5: return launch<K_P3, true>(a, smem, st);
        case 6: return launch<K_PG, false>(a, smem, st);
        default: return launch<K_PG, true>(a, smem, st);
    }
}

template <int KIND>
static cudaError_t bsetup(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(sweep_batch_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sweep_batch_kernel<KIND>, SW_NT, smem);
}

template <int KIND>
static cudaError_t blaunch(int grid, size_t smem, const BatchData &d, const BatchQueue &q, int *err,
                           cudaStream_t st) {
    sweep_batch_kernel<KIND><<<grid, SW_NT, smem, st>>>(d, q, err);
    return cudaGetLastError();
}

cudaError_t batchg_setup(int kind, size_t smem, int *per_sm) {
    switch (kind) {
        case K_P1: return bsetup<K_P1>(smem, per_sm);
        case K_P3: return bsetup<K_P3>(smem, per_sm);
        case K_PG: return bsetup<K_PG>(smem, per_sm);
        default: return bsetup<K_P2>(smem, per_sm);
    }
}

cudaError_t batchg_launch(int kind, int grid, size_t smem, const BatchData &d, const BatchQueue &q, int *err,
                          cudaStream_t st) {
    switch (kind) {
        case K_P1: return blaunch<K_P1>(grid, smem, d, q, err, st);
        case K_P3: return blaunch<K_P3>(grid, smem, d, q, err, st);
        case K_PG: return blaunch<K_PG>(grid, smem, d, q, err, st);
        default: return blaunch<K_P2>(grid, smem, d, q, err, st);
    }
}

MPK_ERROR_WORD_ACCESSOR(generic_error_word)

}  // namespace mpk
