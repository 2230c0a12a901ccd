// The two-stream Euclidean sweep (Algorithm 1, Lemma 1) for single series,
// with and without the block filter, in one-step tiles of V2_R rows.
#include "mp_kernels.h"

namespace mpk {

template <bool FILTER>
static cudaError_t launch(const Sweep2Args &a, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweep2_kernel<K_P2, FILTER, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sweep2_kernel<K_P2, FILTER, false><<<static_cast<unsigned>(a.tiles), V2_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sweep2_p2_launch(bool filter, const Sweep2Args &a, size_t smem, cudaStream_t st) {
    if (a.R > V2_R) return sweep2_p2_tall_launch(filter, a, smem, st);
    return filter ? launch<true>(a, smem, st) : launch<false>(a, smem, st);
}

MPK_ERROR_WORD_ACCESSOR(sweep2_p2_error_word)

}  // namespace mpk
