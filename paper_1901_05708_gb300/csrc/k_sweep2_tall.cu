// The two-stream Euclidean sweep (Algorithm 1, Lemma 1) for single series in
// tall tiles (several sub-tiles of V2_HT rows per stream), with and without
// the block filter.
#include "mp_kernels.h"

namespace mpk {

template <bool FILTER>
static cudaError_t launch(const Sweep2Args &a, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweep2_kernel<K_P2, FILTER, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sweep2_kernel<K_P2, FILTER, true><<<static_cast<unsigned>(a.tiles), V2_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sweep2_p2_tall_launch(bool filter, const Sweep2Args &a, size_t smem, cudaStream_t st) {
    return filter ? launch<true>(a, smem, st) : launch<false>(a, smem, st);
}

MPK_ERROR_WORD_ACCESSOR(sweep2_tall_error_word)

}  // namespace mpk
