// The two-stream p-norm sweep (Algorithm 3, Lemma 2) for p = 1 and p = 3 on
// single series, in one-step or tall tiles.
#include "mp_kernels.h"

namespace mpk {

template <int KIND, bool TALL>
static cudaError_t launch(const Sweep2Args &a, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweep2_kernel<KIND, false, TALL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sweep2_kernel<KIND, false, TALL><<<static_cast<unsigned>(a.tiles), V2_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sweep2_p13_launch(int kind, const Sweep2Args &a, size_t smem, cudaStream_t st) {
    if (a.R > V2_R) return kind == K_P1 ? launch<K_P1, true>(a, smem, st) : launch<K_P3, true>(a, smem, st);
    return kind == K_P1 ? launch<K_P1, false>(a, smem, st) : launch<K_P3, false>(a, smem, st);
}

MPK_ERROR_WORD_ACCESSOR(sweep2_p13_error_word)

}  // namespace mpk
