// A plain diagonal sweep shared by the FP64 variants (Algorithms 1/3 in FP64,
// Algorithm 2 in FP64) and by the FP32 z-normalised sweep.
//
// Same tiling as the FP32 Euclidean kernel (bands of NT * D diagonals cut
// into R-row tiles, one CTA per tile, D adjacent diagonals per thread), but
// the series is read through the cache, the score is re-anchored from a
// direct O(m) window sum every B rows, and minima keep an explicit
// (value, slot) pair compared exactly in the score's own precision.
//
// A variant V supplies:
//   using Real;                                 score type
//   struct State;                               per-diagonal running state
//   State anchor(i, k)                          exact state of cell (i, i+k)
//   void  step(State&, i, k)                    state of (i, i+k) from (i-1, i+k-1)
//   Real  score(const State&, i, k)             value to minimise (NaN = excluded)
//   void  emit(target, value, k, right)         offer a candidate to P[target]
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"

namespace mpk {

constexpr int SM_NT = 128;
constexpr int SM_D = 4;
constexpr int SM_KW = SM_NT * SM_D;

struct TileGrid {
    long long N, k_first, k_end, L, C, tiles, nb;
    int R, q;  // q = KW / R
};

inline TileGrid make_grid(long long N, long long k_first, long long k_end, int KW, int R) {
    TileGrid g{};
    g.N = N;
    g.k_first = k_first;
    g.k_end = k_end;
    g.R = R;
    g.q = KW / R;
    g.L = N - k_first;
    g.C = (g.L + R - 1) / R;
    const long long nb = (k_end - k_first + KW - 1) / KW;
    g.nb = nb;
    g.tiles = nb * g.C - static_cast<long long>(g.q) * nb * (nb - 1) / 2;
    return g;
}

__device__ __forceinline__ long long grid_prefix(const TileGrid &g, long long b) {
    return b * g.C - static_cast<long long>(g.q) * b * (b - 1) / 2;
}

__device__ __forceinline__ void grid_decode(const TileGrid &g, long long t, long long &b, long long &r) {
    const double cq = static_cast<double>(g.C) + 0.5 * g.q;
    const double disc = cq * cq - 2.0 * g.q * static_cast<double>(t);
    long long bb = static_cast<long long>((cq - sqrt(fmax(disc, 0.0))) / g.q);
    if (bb < 0) bb = 0;
    if (bb > g.nb - 1) bb = g.nb - 1;
    while (bb > 0 && grid_prefix(g, bb) > t) --bb;
    while (bb + 1 < g.nb && grid_prefix(g, bb + 1) <= t) ++bb;
    b = bb;
    r = t - grid_prefix(g, bb);
}

template <class V>
__global__ void __launch_bounds__(SM_NT) simple_sweep_kernel(const TileGrid g, const V v, const int B) {
    using Real = typename V::Real;
    using State = typename V::State;
    long long band, rt;
    grid_decode(g, blockIdx.x, band, rt);
    if (rt < 0 || rt >= g.C - static_cast<long long>(g.q) * band) {
        if (threadIdx.x == 0) atomicOr(&mp_device_error, ERR_BAD_TILE);
        return;
    }
    const long long k0 = g.k_first + band * SM_KW;
    const long long r0 = rt * g.R;
    const long long kt = k0 + static_cast<long long>(threadIdx.x) * SM_D;
    const long long nd_ll = g.k_end - kt;
    const int nd = nd_ll <= 0 ? 0 : (nd_ll >= SM_D ? SM_D : static_cast<int>(nd_ll));
    const long long lim = g.N - kt - r0;  // cell (u, d) valid iff u + d < lim
    const int rows = nd == 0 || lim <= 0 ? 0 : (lim < g.R ? static_cast<int>(lim) : g.R);
    if (rows == 0) return;

    State st[SM_D];
    Real colv[SM_D];
    int cold[SM_D];
    const Real inf = V::inf();
#pragma unroll
    for (int d = 0; d < SM_D; ++d) { colv[d] = inf; cold[d] = -1; }

    int ulast = 0;
    for (int ub = 0; ub < rows; ub += SM_D) {
#pragma unroll
        for (int ul = 0; ul < SM_D; ++ul) {
            const int u = ub + ul;
            if (u >= rows) break;
            const long long i = r0 + u;
            Real sc[SM_D];
#pragma unroll
            for (int d = 0; d < SM_D; ++d) {
                const long long k = kt + d;
                const bool ok = d < nd && u + d < lim;
                if (ok) {
                    if (u % B == 0) st[d] = v.anchor(i, k);
                    else v.step(st[d], i, k);
                    sc[d] = v.score(st[d], i, k);
                } else {
                    sc[d] = inf;
                }
            }
            // row: first strictly smaller wins (smallest k among equals)
            Real rv = inf;
            int rd = -1;
#pragma unroll
            for (int d = 0; d < SM_D; ++d)
                if (sc[d] < rv) { rv = sc[d]; rd = d; }
            if (rd >= 0) v.emit(i, rv, kt + rd, 1);
            // columns: slot (ul + d) % D holds column r0 + kt + u + d; a later
            // row brings a smaller d, so '<=' keeps the smallest k among equals
#pragma unroll
            for (int d = SM_D - 1; d >= 0; --d) {
                const int sl = (ul + d) % SM_D;
                if (sc[d] <= colv[sl]) { colv[sl] = sc[d]; cold[sl] = d; }
            }
            if (cold[ul] >= 0) v.emit(r0 + kt + u, colv[ul], kt + cold[ul], 0);
            colv[ul] = inf;
            cold[ul] = -1;
            ulast = u;
        }
    }
#pragma unroll
    for (int sl = 0; sl < SM_D; ++sl) {
        if (cold[sl] < 0) continue;
        const int delta = ((sl - ulast) % SM_D + SM_D) % SM_D;
        v.emit(r0 + kt + ulast + delta, colv[sl], kt + cold[sl], 0);
    }
}

// ---- FP64 Euclidean / p-norm (Algorithms 1 and 3 in FP64) -------------------------
struct VarF64Lp {
    using Real = double;
    struct State { double s; };
    const double *x;  // FP64 series
    int m;
    double p;
    Key128 *keys;
    int *err;
    __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    __device__ double tm(double e) const {
        e = fabs(e);
        if (p == 2.0) return e * e;
        if (p == 1.0) return e;
        if (p == 3.0) return e * e * e;
        return pow(e, p);
    }
    __device__ State anchor(long long i, long long k) const {
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc += tm(x[i + l] - x[i + k + l]);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        s.s = (s.s + tm(x[i + m - 1] - x[i + k + m - 1])) - tm(x[i - 1] - x[i + k - 1]);
    }
    __device__ double score(const State &s, long long, long long) const { return s.s < 0 ? 0.0 : s.s; }
    __device__ void emit(long long target, double val, long long k, int right) const {
        const double cur = __longlong_as_double(static_cast<long long>(keys[target].hi));
        if (!(val <= cur) && keys[target].hi != KEY_NONE) return;
        if (!atomic_min_key128(&keys[target], static_cast<unsigned long long>(__double_as_longlong(val)),
                               static_cast<unsigned long long>(2 * k + right)))
            atomicOr(err, ERR_CAS_SPIN);
    }
};

// ---- z-normalised (Algorithm 2 on the centred covariance) --------------------------
// cov_{i,j} = sum_l (t_{i+l} - mu_i)(t_{j+l} - mu_j), carried along the diagonal
// with cov_{i,j} = cov_{i-1,j-1} + df_{i-1} dg_{j-1} + df_{j-1} dg_{i-1}, and the
// score q = 1 - rho = 1 - cov / sqrt(S_i S_j) (DZ^2 = 2 m q, Lemma 3).
struct VarF64Z {
    using Real = double;
    struct State { double cov; };
    const double *x, *mu, *S;
    const unsigned char *flat;
    int m;
    Key128 *keys;
    int *err;
    __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    __device__ State anchor(long long i, long long k) const {
        const double mi = mu[i], mj = mu[i + k];
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(x[i + l] - mi, x[i + k + l] - mj, acc);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        const long long a = i - 1, b = i + k - 1;
        const double dfa = 0.5 * (x[a + m] - x[a]), dfb = 0.5 * (x[b + m] - x[b]);
        const double dga = (x[a + m] - mu[a + 1]) + (x[a] - mu[a]);
        const double dgb = (x[b + m] - mu[b + 1]) + (x[b] - mu[b]);
        s.cov = fma(dfa, dgb, fma(dfb, dga, s.cov));
    }
    __device__ double score(const State &s, long long i, long long k) const {
        if (flat[i] || flat[i + k]) return __longlong_as_double(0x7ff8000000000000ll);  // NaN
        const double q = 1.0 - s.cov / sqrt(S[i] * S[i + k]);
        return q < 0 ? 0.0 : (q > 2.0 ? 2.0 : q);
    }
    __device__ void emit(long long target, double val, long long k, int right) const {
        const double cur = __longlong_as_double(static_cast<long long>(keys[target].hi));
        if (!(val <= cur) && keys[target].hi != KEY_NONE) return;
        if (!atomic_min_key128(&keys[target], static_cast<unsigned long long>(__double_as_longlong(val)),
                               static_cast<unsigned long long>(2 * k + right)))
            atomicOr(err, ERR_CAS_SPIN);
    }
};

// FP32 z-normalised sweep: FP32 covariance recurrence on FP32 operands
// (df, dg, inv from the FP64 statistics), FP32 anchors on FP32-centred values
// (cov = sum (t_i - mu~_i)(t_j - mu~_j) is insensitive to the rounding of the
// means to first order), 64-bit keys holding the FP32 score q = 1 - rho.
struct VarF32Z {
    using Real = float;
    struct State { float cov; };
    const float *t;            // FP32 series
    const float *muf;          // FP32 window means
    const float *df, *dg, *inv;  // inv = NaN for a flat window
    int m;
    unsigned long long *keys;
    __device__ static float inf() { return __int_as_float(0x7f800000); }
    __device__ State anchor(long long i, long long k) const {
        const float mi = muf[i], mj = muf[i + k];
        float acc = 0.f;
        for (int l = 0; l < m; ++l) acc = fmaf(t[i + l] - mi, t[i + k + l] - mj, acc);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        const long long a = i - 1, b = i + k - 1;
        s.cov = fmaf(df[a], dg[b], fmaf(df[b], dg[a], s.cov));
    }
    __device__ float score(const State &s, long long i, long long k) const {
        const float q = fmaf(-s.cov, inv[i] * inv[i + k], 1.0f);  // NaN if flat
        return q < 0.f ? 0.f : q;
    }
    __device__ void emit(long long target, float val, long long k, int right) const {
        if (!(val < __int_as_float(0x7f800000))) return;
        atomicMin(&keys[target], make_key(__float_as_uint(val), k, right));
    }
};

// ---- z-normalised, raw sums (Algorithm 2 as printed; an ablation) -------------------
// The paper's form of Lemma 3: the dot product C_{i,j} = sum_l t_{i+l} t_{j+l}
// carried with C_{i,j} = C_{i-1,j-1} + t_{i+m-1} t_{j+m-1} - t_{i-1} t_{j-1}, and
// rho = (C - A_i A_j / m) / sqrt(S_i S_j) with the window sums A = m mu.  The
// numerator cancels when a window's mean is large against its spread; the
// centred covariance of VarF64Z / VarF32Z avoids that.  Both precisions take
// the same denominators and flat rule as the centred variants, so only the
// form of the sum differs.
struct VarF64ZRaw {
    using Real = double;
    struct State { double c; };
    const double *x, *mu, *S;
    const unsigned char *flat;
    int m;
    Key128 *keys;
    int *err;
    __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    __device__ State anchor(long long i, long long k) const {
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(x[i + l], x[i + k + l], acc);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        const long long a = i - 1, b = i + k - 1;
        s.c = fma(x[a + m], x[b + m], fma(-x[a], x[b], s.c));
    }
    __device__ double score(const State &s, long long i, long long k) const {
        if (flat[i] || flat[i + k]) return __longlong_as_double(0x7ff8000000000000ll);  // NaN
        const double num = s.c - static_cast<double>(m) * mu[i] * mu[i + k];
        const double q = 1.0 - num / sqrt(S[i] * S[i + k]);
        return q < 0 ? 0.0 : (q > 2.0 ? 2.0 : q);
    }
    __device__ void emit(long long target, double val, long long k, int right) const {
        const double cur = __longlong_as_double(static_cast<long long>(keys[target].hi));
        if (!(val <= cur) && keys[target].hi != KEY_NONE) return;
        if (!atomic_min_key128(&keys[target], static_cast<unsigned long long>(__double_as_longlong(val)),
                               static_cast<unsigned long long>(2 * k + right)))
            atomicOr(err, ERR_CAS_SPIN);
    }
};

struct VarF32ZRaw {
    using Real = float;
    struct State { float c; };
    const float *t;    // FP32 series
    const float *muf;  // FP32 window means
    const float *inv;  // 1 / sqrt(S) from the FP64 statistics; NaN for a flat window
    int m;
    unsigned long long *keys;
    __device__ static float inf() { return __int_as_float(0x7f800000); }
    __device__ State anchor(long long i, long long k) const {
        float acc = 0.f;
        for (int l = 0; l < m; ++l) acc = fmaf(t[i + l], t[i + k + l], acc);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        const long long a = i - 1, b = i + k - 1;
        s.c = fmaf(t[a + m], t[b + m], fmaf(-t[a], t[b], s.c));
    }
    __device__ float score(const State &s, long long i, long long k) const {
        const float num = fmaf(-static_cast<float>(m) * muf[i], muf[i + k], s.c);
        const float q = fmaf(-num, inv[i] * inv[i + k], 1.0f);  // NaN if flat
        return q < 0.f ? 0.f : q;
    }
    __device__ void emit(long long target, float val, long long k, int right) const {
        if (!(val < __int_as_float(0x7f800000))) return;
        atomicMin(&keys[target], make_key(__float_as_uint(val), k, right));
    }
};

}  // namespace mpk

namespace mpk {

// ---- z-normalised, raw sums compared through F (Sec. 4.3, Appendix A; an ablation) ---
// The paper's cheaper comparison: instead of DZ^2, each candidate is ordered by
//   F_{i,j} = (A_i B_j - m C_{i,j}) |A_i B_j - m C_{i,j}| / (S_i S_j)
// with Lemma 3's window sums A = m mu, the dot product C carried along the
// diagonal as in VarF64ZRaw / VarF32ZRaw, and S the centred sums of squares
// (the denominator read as (B_j - B_j^2 / m), the square Lemma 3 has).  F is
// -m^2 rho |rho|, increasing in DZ, and needs no square root per cell; the
// winner's distance is DZ^2 = 2m + 2 sign(F) sqrt(|F|) (that formula's left
// side read as DZ^2).  F is signed, so keys hold an order-preserving map of its
// bits (f_order_bits) and the finalize inverts it (FinalizeArgs::fkey).

// Unsigned image of a float / double that orders like the value (negative
// values: all bits flipped; others: the sign bit set).
__device__ __forceinline__ unsigned f_order_bits(float f) {
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long f_order_bits(double f) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(f));
    return (b >> 63) ? ~b : (b | (1ull << 63));
}

struct VarF64ZF {
    using Real = double;
    struct State { double c; };
    const double *x, *mu, *S;
    const unsigned char *flat;
    int m;
    Key128 *keys;
    int *err;
    __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    __device__ State anchor(long long i, long long k) const {
        double acc = 0.0;
        for (int l = 0; l < m; ++l) acc = fma(x[i + l], x[i + k + l], acc);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        const long long a = i - 1, b = i + k - 1;
        s.c = fma(x[a + m], x[b + m], fma(-x[a], x[b], s.c));
    }
    __device__ double score(const State &s, long long i, long long k) const {
        if (flat[i] || flat[i + k]) return __longlong_as_double(0x7ff8000000000000ll);  // NaN
        const double A = m * mu[i], B = m * mu[i + k];
        const double num = fma(A, B, -static_cast<double>(m) * s.c);  // A_i B_j - m C
        return num * fabs(num) / (S[i] * S[i + k]);
    }
    __device__ void emit(long long target, double val, long long k, int right) const {
        const unsigned long long hi = f_order_bits(val);
        if (keys[target].hi != KEY_NONE && hi > keys[target].hi) return;
        if (!atomic_min_key128(&keys[target], hi, static_cast<unsigned long long>(2 * k + right)))
            atomicOr(err, ERR_CAS_SPIN);
    }
};

struct VarF32ZF {
    using Real = float;
    struct State { float c; };
    const float *t;    // FP32 series
    const float *muf;  // FP32 window means
    const float *inv;  // 1 / sqrt(S); NaN for a flat window
    int m;
    unsigned long long *keys;
    __device__ static float inf() { return __int_as_float(0x7f800000); }
    __device__ State anchor(long long i, long long k) const {
        float acc = 0.f;
        for (int l = 0; l < m; ++l) acc = fmaf(t[i + l], t[i + k + l], acc);
        return State{acc};
    }
    __device__ void step(State &s, long long i, long long k) const {
        const long long a = i - 1, b = i + k - 1;
        s.c = fmaf(t[a + m], t[b + m], fmaf(-t[a], t[b], s.c));
    }
    __device__ float score(const State &s, long long i, long long k) const {
        const float fm = static_cast<float>(m);
        const float num = fmaf(fm * muf[i], fm * muf[i + k], -fm * s.c);  // A_i B_j - m C
        const float w = inv[i] * inv[i + k];                                // NaN if flat
        return num * fabsf(num) * (w * w);
    }
    __device__ void emit(long long target, float val, long long k, int right) const {
        if (!(val < __int_as_float(0x7f800000))) return;
        atomicMin(&keys[target], make_key(f_order_bits(val), k, right));
    }
};

}  // namespace mpk
