// Batch queues of the two-stream sweep: persistent CTAs taking tiles of many
// series (p = 2 with or without the block filter, p = 1, p = 3).
#include "mp_kernels.h"

namespace mpk {

template <int KIND, bool FILTER>
static cudaError_t setup(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(sweep2_batch_kernel<KIND, FILTER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sweep2_batch_kernel<KIND, FILTER>, V2_NT, smem);
}

template <int KIND, bool FILTER>
static cudaError_t launch(int grid, size_t smem, const BatchData &d, const BatchQueue &q, cudaStream_t st) {
    sweep2_batch_kernel<KIND, FILTER><<<grid, V2_NT, smem, st>>>(d, q);
    return cudaGetLastError();
}

cudaError_t batch2_setup(int kind, bool filter, size_t smem, int *per_sm) {
    if (kind == K_P1) return setup<K_P1, false>(smem, per_sm);
    if (kind == K_P3) return setup<K_P3, false>(smem, per_sm);
    return filter ? setup<K_P2, true>(smem, per_sm) : setup<K_P2, false>(smem, per_sm);
}

cudaError_t batch2_launch(int kind, bool filter, int grid, size_t smem, const BatchData &d, const BatchQueue &q,
                          cudaStream_t st) {
    if (kind == K_P1) return launch<K_P1, false>(grid, smem, d, q, st);
    if (kind == K_P3) return launch<K_P3, false>(grid, smem, d, q, st);
    return filter ? launch<K_P2, true>(grid, smem, d, q, st) : launch<K_P2, false>(grid, smem, d, q, st);
}

MPK_ERROR_WORD_ACCESSOR(batch2_error_word)

}  // namespace mpk
