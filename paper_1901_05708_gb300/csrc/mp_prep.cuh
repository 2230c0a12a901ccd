// Pre- and post-processing kernels around the diagonal sweep:
//   a1  convert   series -> FP32 (hi[, lo]) or FP64 copy in the workspace
//   a2  stats     FP64 window means / centred sums of squares (z-norm)
//   a6  finalize  keys -> I, P (optionally polished in FP64 at I)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"

namespace mpk {

constexpr int PREP_NT = 256;

// ---- deterministic FP64 sum of the input (two passes, fixed order) -----------
// Pass 1: block b sums elements b, b + G, b + 2G, ... (grid-stride) into part[b].
template <typename Tin>
__global__ void __launch_bounds__(PREP_NT) sum_partial_kernel(const Tin *__restrict__ T, long long n,
                                                              double *__restrict__ part) {
    __shared__ double red[PREP_NT];
    double acc = 0.0;
    for (long long x = blockIdx.x * (long long)PREP_NT + threadIdx.x; x < n;
         x += (long long)gridDim.x * PREP_NT)
        acc += static_cast<double>(T[x]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = PREP_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Pass 2: one block adds the partials in a fixed order; out = sum / n.
__global__ void __launch_bounds__(PREP_NT) sum_final_kernel(const double *__restrict__ part, int nparts,
                                                            long long n, double *__restrict__ out) {
    __shared__ double red[PREP_NT];
    double acc = 0.0;
    for (int x = threadIdx.x; x < nparts; x += PREP_NT) acc += part[x];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = PREP_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] / static_cast<double>(n);
}

// ---- a1: conversion for the FP32 sweep ----------------------------------------
// FP32 input: hi = t exactly (the differences t_i - t_j the sweep needs are
// then as exact as FP32 allows); lo = 0.
// FP64 input: hi + lo represents t - shift to ~2^-48 relative, where shift is
// the series mean (distances are shift-invariant, Eq. def-euclidean-distance,
// and z-normalisation removes any offset, Eq. def-z-normalized-distance).
// Elements in [n, n + pad) are zero so that tile loads may run past the end.
template <typename Tin>
__global__ void __launch_bounds__(PREP_NT) convert_f32_kernel(const Tin *__restrict__ T, long long n,
                                                              long long padded,
                                                              const double *__restrict__ shift_ptr,
                                                              float *__restrict__ hi,
                                                              float *__restrict__ lo) {
    const double shift = shift_ptr ? shift_ptr[0] : 0.0;
    for (long long x = blockIdx.x * (long long)PREP_NT + threadIdx.x; x < padded;
         x += (long long)gridDim.x * PREP_NT) {
        if (x < n) {
            const double v = static_cast<double>(T[x]) - shift;
            const float h = static_cast<float>(v);
            hi[x] = h;
            if (lo) lo[x] = static_cast<float>(v - static_cast<double>(h));
        } else {
            hi[x] = 0.f;
            if (lo) lo[x] = 0.f;
        }
    }
}

template <typename Tin>
__global__ void __launch_bounds__(PREP_NT) convert_f64_kernel(const Tin *__restrict__ T, long long n,
                                                              long long padded,
                                                              double *__restrict__ out) {
    for (long long x = blockIdx.x * (long long)PREP_NT + threadIdx.x; x < padded;
         x += (long long)gridDim.x * PREP_NT)
        out[x] = x < n ? static_cast<double>(T[x]) : 0.0;
}

__global__ void __launch_bounds__(PREP_NT) fill_u64_kernel(unsigned long long *__restrict__ p, long long count,
                                                           unsigned long long v) {
    for (long long x = blockIdx.x * (long long)PREP_NT + threadIdx.x; x < count;
         x += (long long)gridDim.x * PREP_NT)
        p[x] = v;
}

// ---- a2: window statistics for the z-normalised distance ----------------------
// For every window i (Sec. 4.1's A_i and the definition of mu_i, sigma_i):
//   mu_i  = (1/m) sum_l t_{i+l}
//   S_i   = sum_l (t_{i+l} - mu_i)^2          (= m sigma_i^2, population)
//   flat_i: S_i <= 2^-40 sum_l t_{i+l}^2     (sigma = 0 up to rounding)
// Two passes per window in FP64 over the (shifted) FP64 series x.  One
// thread per window; neighbouring threads read overlapping windows through
// the cache.  O(n m) FP64 work, a small share of the sweep for m <= 512.
// One window (X = double, or float for an FP32 series read directly).
// Sums over a window are taken as four interleaved partial sums (independent
// FP64 chains and loads in flight), combined pairwise.
template <typename X>
__device__ __forceinline__ void window_stats_at(const X *__restrict__ x, long long i, int m, double &mean,
                                                double &S, unsigned char &flat) {
    const X *w = x + i;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int l = 0;
    for (; l + 4 <= m; l += 4) {
        a0 += static_cast<double>(w[l]);
        a1 += static_cast<double>(w[l + 1]);
        a2 += static_cast<double>(w[l + 2]);
        a3 += static_cast<double>(w[l + 3]);
    }
    for (; l < m; ++l) a0 += static_cast<double>(w[l]);
    mean = ((a0 + a1) + (a2 + a3)) / m;
    double q0 = 0.0, q1 = 0.0, r0 = 0.0, r1 = 0.0;
    l = 0;
    for (; l + 2 <= m; l += 2) {
        const double v0 = static_cast<double>(w[l]), v1 = static_cast<double>(w[l + 1]);
        const double d0 = v0 - mean, d1 = v1 - mean;
        q0 = fma(d0, d0, q0);
        q1 = fma(d1, d1, q1);
        r0 = fma(v0, v0, r0);
        r1 = fma(v1, v1, r1);
    }
    if (l < m) {
        const double v = static_cast<double>(w[l]), d = v - mean;
        q0 = fma(d, d, q0);
        r0 = fma(v, v, r0);
    }
    const double q = q0 + q1, r = r0 + r1;
    S = q;
    flat = q <= 0x1p-40 * r;
}

__global__ void __launch_bounds__(PREP_NT) window_stats_kernel(const double *__restrict__ x, long long N, int m,
                                                               double *__restrict__ mu,
                                                               double *__restrict__ S,
                                                               unsigned char *__restrict__ flat) {
    for (long long i = blockIdx.x * (long long)PREP_NT + threadIdx.x; i < N;
         i += (long long)gridDim.x * PREP_NT)
        window_stats_at(x, i, m, mu[i], S[i], flat[i]);
}

// FP32 operands of the centred-covariance sweep (derived in FP64):
//   df_i = (t_{i+m} - t_i) / 2
//   dg_i = (t_{i+m} - mu_{i+1}) + (t_i - mu_i)
//   inv_i = 1 / sqrt(S_i)  (NaN for a flat window: every score it touches is NaN
//                          and never wins a minimum)
// so that cov_{i+1,j+1} = cov_{i,j} + df_i dg_j + df_j dg_i and
// rho_{i,j} = cov_{i,j} inv_i inv_j (Lemma 3 with A = m mu, C = cov + m mu_i mu_j).
template <typename X>
__device__ __forceinline__ void znorm_operands_at(const X *__restrict__ x, long long i, long long N, int m,
                                                  const double *__restrict__ mu, const double *__restrict__ S,
                                                  const unsigned char *__restrict__ flat, double shift,
                                                  float *__restrict__ df, float *__restrict__ dg,
                                                  float *__restrict__ inv, float *__restrict__ muf,
                                                  float *__restrict__ mul) {
    inv[i] = flat[i] ? __int_as_float(0x7fc00000) : static_cast<float>(1.0 / sqrt(S[i]));
    const double ms = mu[i] - shift;
    muf[i] = static_cast<float>(ms);
    if (mul) mul[i] = static_cast<float>(ms - static_cast<double>(muf[i]));  // float-float mean
    if (i + 1 < N) {
        const double xe = static_cast<double>(x[i + m]), xl = static_cast<double>(x[i]);
        df[i] = static_cast<float>(0.5 * (xe - xl));
        dg[i] = static_cast<float>((xe - mu[i + 1]) + (xl - mu[i]));
    } else {
        df[i] = 0.f;
        dg[i] = 0.f;
    }
}

__global__ void __launch_bounds__(PREP_NT) znorm_operands_kernel(const double *__restrict__ x, long long N, int m,
                                                                 const double *__restrict__ mu,
                                                                 const double *__restrict__ S,
                                                                 const unsigned char *__restrict__ flat,
                                                                 float *__restrict__ df, float *__restrict__ dg,
                                                                 float *__restrict__ inv, float *__restrict__ muf,
                                                                 float *__restrict__ mul,
                                                                 const double *__restrict__ shift_ptr,
                                                                 long long padded) {
    const double shift = shift_ptr ? shift_ptr[0] : 0.0;  // the offset removed from the FP32 series
    for (long long i = blockIdx.x * (long long)PREP_NT + threadIdx.x; i < padded;
         i += (long long)gridDim.x * PREP_NT) {
        if (i < N) {
            znorm_operands_at(x, i, N, m, mu, S, flat, shift, df, dg, inv, muf, mul);
        } else {
            inv[i] = __int_as_float(0x7fc00000);
            muf[i] = 0.f;
            if (mul) mul[i] = 0.f;
            df[i] = 0.f;
            dg[i] = 0.f;
        }
    }
}

// ---- a6: finalize ----------------------------------------------------------------
enum { FIN_EUCLID = 0, FIN_PNORM = 1, FIN_ZNORM = 2 };

template <typename X>
struct FinalizeArgsT {
    const unsigned long long *keys;  // FP32 sweep keys, or
    const Key128 *keys128;           // FP64 sweep keys
    const X *x;                      // the series for the polish (FP64, or FP32 read as FP64)
    const double *mu, *S;            // z-norm stats (FP64)
    long long N;
    int m;
    int dist;
    double p;
    int polish;
    int fkey;                        // z-norm keys hold the order image of F (Sec. 4.3), not 1 - rho
    double *P;
    long long *I;
};
using FinalizeArgs = FinalizeArgsT<double>;

// Inverse of the order-preserving images f_order_bits (mp_simple.cuh).
__device__ __forceinline__ float f_from_order_bits(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ double f_from_order_bits(unsigned long long u) {
    return __longlong_as_double(static_cast<long long>((u >> 63) ? (u & ~(1ull << 63)) : ~u));
}

// DZ^2 from F = -m^2 rho |rho|: 2m + 2 sign(F) sqrt(|F|) (Sec. 4.3, Appendix A).
__device__ __forceinline__ double dz2_from_f(double F, int m) {
    const double r = sqrt(fabs(F));
    return 2.0 * m + 2.0 * (F < 0 ? -r : r);
}

// |v|^p; the products are rounded one by one (no contraction into the caller's
// sum), so every kernel that polishes gets the same bits.
__device__ __forceinline__ double pow_abs(double v, double p) {
    v = fabs(v);
    if (p == 1.0) return v;
    if (p == 2.0) return __dmul_rn(v, v);
    if (p == 3.0) return __dmul_rn(__dmul_rn(v, v), v);
    return pow(v, p);
}

// d(i, j) from the definitions (Sec. 2) in FP64, as four interleaved partial
// sums combined pairwise (independent chains keep loads in flight).
template <typename X>
__device__ double exact_score(const FinalizeArgsT<X> &a, long long i, long long j) {
    const X *xi = a.x + i, *xj = a.x + j;
    const int m = a.m;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (a.dist == FIN_EUCLID) {
        int l = 0;
        for (; l + 4 <= m; l += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double d = static_cast<double>(xi[l + u]) - static_cast<double>(xj[l + u]);
                acc[u] = fma(d, d, acc[u]);
            }
        }
        for (; l < m; ++l) {
            const double d = static_cast<double>(xi[l]) - static_cast<double>(xj[l]);
            acc[0] = fma(d, d, acc[0]);
        }
    } else if (a.dist == FIN_PNORM) {
        int l = 0;
        for (; l + 4 <= m; l += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                acc[u] = __dadd_rn(acc[u], pow_abs(static_cast<double>(xi[l + u]) - static_cast<double>(xj[l + u]), a.p));
        }
        for (; l < m; ++l) acc[0] = __dadd_rn(acc[0], pow_abs(static_cast<double>(xi[l]) - static_cast<double>(xj[l]), a.p));
    } else {
        const double mi = a.mu[i], mj = a.mu[j];
        const double si = 1.0 / sqrt(a.S[i] / m), sj = 1.0 / sqrt(a.S[j] / m);
        int l = 0;
        for (; l + 4 <= m; l += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double d = __dsub_rn(__dmul_rn(static_cast<double>(xi[l + u]) - mi, si),
                                           __dmul_rn(static_cast<double>(xj[l + u]) - mj, sj));
                acc[u] = fma(d, d, acc[u]);
            }
        }
        for (; l < m; ++l) {
            const double d = __dsub_rn(__dmul_rn(static_cast<double>(xi[l]) - mi, si),
                                       __dmul_rn(static_cast<double>(xj[l]) - mj, sj));
            acc[0] = fma(d, d, acc[0]);
        }
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

template <typename X>
__device__ __forceinline__ double finish_score(const FinalizeArgsT<X> &a, double s) {
    if (s < 0) s = 0;
    if (a.dist == FIN_PNORM) {
        if (a.p == 1.0) return s;
        if (a.p == 2.0) return sqrt(s);
        return pow(s, 1.0 / a.p);
    }
    return sqrt(s);
}

// Window x: key -> I[x]; P[x] from the sweep value or, polished, from d(x, I[x]).
template <typename X>
__device__ __forceinline__ void finalize_at(const FinalizeArgsT<X> &a, long long x) {
    unsigned long long lo;
    double sweep_score;
    bool none;
    if (a.keys) {
        const unsigned long long key = a.keys[x];
        none = key == KEY_NONE;
        lo = key & 0xffffffffull;
        const unsigned vb = static_cast<unsigned>(key >> 32);
        const float v = __uint_as_float(vb);
        // z-norm keys hold 1 - rho; DZ^2 = 2m(1 - rho) (Lemma 3); or F
        if (a.fkey) sweep_score = dz2_from_f(static_cast<double>(f_from_order_bits(vb)), a.m);
        else sweep_score = a.dist == FIN_ZNORM ? 2.0 * a.m * static_cast<double>(v) : static_cast<double>(v);
    } else {
        const Key128 key = a.keys128[x];
        none = key.hi == KEY_NONE;
        lo = key.lo;
        const double v = __longlong_as_double(static_cast<long long>(key.hi));
        if (a.fkey) sweep_score = dz2_from_f(f_from_order_bits(key.hi), a.m);
        else sweep_score = a.dist == FIN_ZNORM ? 2.0 * a.m * v : v;
    }
    if (none) {
        a.P[x] = __longlong_as_double(0x7ff0000000000000ll);  // +inf
        a.I[x] = -1;
        return;
    }
    const long long k = static_cast<long long>(lo >> 1);
    const long long j = (lo & 1) ? x + k : x - k;
    a.I[x] = j;
    double s = a.polish ? exact_score(a, x, j) : sweep_score;
    if (a.dist == FIN_ZNORM) s = fmin(fmax(s, 0.0), 4.0 * a.m);
    a.P[x] = finish_score(a, s);
}

__global__ void __launch_bounds__(PREP_NT) finalize_kernel(FinalizeArgs a) {
    for (long long x = blockIdx.x * (long long)PREP_NT + threadIdx.x; x < a.N;
         x += (long long)gridDim.x * PREP_NT)
        finalize_at(a, x);
}

}  // namespace mpk
