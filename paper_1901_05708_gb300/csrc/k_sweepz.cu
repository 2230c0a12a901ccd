// Tall float-float tiles: the z-normalised sweep (Algorithm 2, Lemma 3, on the
// centred covariance) and the Euclidean / p-norm sweeps of long windows, for
// single series and for the batch queue of z-normalised series.
#include "mp_kernels.h"

namespace mpk {

template <int MODE, int FILTER>
static cudaError_t launch(const SweepZArgs &a, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweepz_kernel<MODE, FILTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sweepz_kernel<MODE, FILTER><<<static_cast<unsigned>(a.tiles), Z_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sweepz_launch(int mode, int filter, const SweepZArgs &a, size_t smem, cudaStream_t st) {
    switch (mode) {
        case K_Z:
            return filter == 2 ? launch<K_Z, 2>(a, smem, st) : filter ? launch<K_Z, 1>(a, smem, st)
                                                                     : launch<K_Z, 0>(a, smem, st);
        case K_P1: return launch<K_P1, 0>(a, smem, st);
        case K_P3: return launch<K_P3, 0>(a, smem, st);
        default: return filter ? launch<K_P2, 1>(a, smem, st) : launch<K_P2, 0>(a, smem, st);
    }
}

cudaError_t batchz_setup(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(sweepz_batch_kernel<K_Z>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sweepz_batch_kernel<K_Z>, Z_NT, smem);
}

cudaError_t batchz_launch(int grid, size_t smem, const BatchData &d, const BatchQueue &q, cudaStream_t st) {
    sweepz_batch_kernel<K_Z><<<grid, Z_NT, smem, st>>>(d, q);
    return cudaGetLastError();
}

MPK_ERROR_WORD_ACCESSOR(sweepz_error_word)

}  // namespace mpk
