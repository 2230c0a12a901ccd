// Device-side helpers shared by the matrix-profile kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// Device-side error word: kernels OR mpk::ERR_* bits into it; mp_sync_status
// reads and clears it.  The library is several translation units compiled
// without relocatable device code, so each one that holds kernels has its own
// word (internal linkage) and exports its address through an accessor
// (MPK_ERROR_WORD_ACCESSOR); mp_sync_status reads every word.
static __device__ int mp_device_error;

// Defines `int *fn()`: the device address of this translation unit's error word.
#define MPK_ERROR_WORD_ACCESSOR(fn)                                               \
    int *fn() {                                                                   \
        void *p = nullptr;                                                        \
        return cudaGetSymbolAddress(&p, mp_device_error) == cudaSuccess           \
                   ? static_cast<int *>(p) : nullptr;                             \
    }

namespace mpk {

// Term of the distance carried by the Euclidean / p-norm sweeps:
// e^2 (p = 2, Lemma 1), |e| (p = 1), |e|^3 (p = 3), |e|^p (other real p; Lemma 2).
enum Kind { K_P2 = 0, K_P1 = 1, K_P3 = 2, K_PG = 3, K_Z = 4 };  // K_Z: the z-normalised sweep

// Error bits written to the device error word (read back by mp_sync_status).
enum : int {
    ERR_CAS_SPIN = 1,   // a bounded compare-and-swap loop gave up
    ERR_BAD_TILE = 2,   // tile decoding produced an out-of-range tile
};

// A 64-bit profile key orders candidates the way the strict '<' of the
// paper's loops does: high word = non-negative FP32 score bits (monotone as
// an unsigned integer), low word = 2k + [neighbour on the right].  The
// smallest key is the smallest score, then the smallest |i - j|, then the
// left neighbour.  The all-ones key means "no candidate yet".
constexpr unsigned long long KEY_NONE = ~0ull;

__device__ __forceinline__ unsigned long long make_key(unsigned value_bits, long long k, int right) {
    return (static_cast<unsigned long long>(value_bits) << 32) |
           static_cast<unsigned>(2 * k + right);
}

// 128-bit key for the FP64 sweep: (FP64 score bits, 2k + side), compared
// lexicographically.  Stored as two u64 words, high word first.
struct alignas(16) Key128 {
    unsigned long long hi, lo;
};

// atomicMin on a Key128 through a bounded 128-bit compare-and-swap loop.  The
// 128-bit operand {a, b} has a in its low half, which is the word at the
// lower address (little endian), i.e. Key128::hi.
// Returns false if the loop gave up (the caller flags ERR_CAS_SPIN).
__device__ __forceinline__ bool atomic_min_key128(Key128 *addr, unsigned long long hi,
                                                  unsigned long long lo) {
    unsigned long long ohi = addr->hi, olo = addr->lo;  // may be torn; CAS fixes it
    for (int it = 0; it < 4096; ++it) {
        if (ohi < hi || (ohi == hi && olo <= lo)) return true;
        unsigned long long rhi, rlo;
        asm volatile(
            "{ .reg .b128 cmp, swp, old;\n\t"
            "mov.b128 cmp, {%2, %3};\n\t"
            "mov.b128 swp, {%4, %5};\n\t"
            "atom.global.cas.b128 old, [%6], cmp, swp;\n\t"
            "mov.b128 {%0, %1}, old; }"
            : "=l"(rhi), "=l"(rlo)
            : "l"(ohi), "l"(olo), "l"(hi), "l"(lo), "l"(addr)
            : "memory");
        if (rhi == ohi && rlo == olo) return true;
        ohi = rhi;
        olo = rlo;
    }
    return false;
}

// Smallest FP32 not below x (x >= 0): a float threshold that never rejects a
// double candidate that is <= x.
__device__ __forceinline__ float float_up(double x) { return __double2float_ru(x); }

}  // namespace mpk
