// The two-stream p-norm sweep (Algorithm 3, Lemma 2) for p = 1 and p = 3 on
// single series.
#include "mp_kernels.h"

namespace mpk {

template <int KIND>
static cudaError_t launch(const Sweep2Args &a, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sweep2_kernel<KIND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    sweep2_kernel<KIND, false><<<static_cast<unsigned>(a.tiles), V2_NT, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t sweep2_p13_launch(int kind, const Sweep2Args &a, size_t smem, cudaStream_t st) {
    return kind == K_P1 ? launch<K_P1>(a, smem, st) : launch<K_P3>(a, smem, st);
}

MPK_ERROR_WORD_ACCESSOR(sweep2_p13_error_word)

}  // namespace mpk
