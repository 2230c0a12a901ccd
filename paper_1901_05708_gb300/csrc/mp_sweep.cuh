// a3-a5: the diagonal sweep of Algorithms 1 (Euclidean) and 3 (p-norm).
//
// Work decomposition.  The candidate pairs (i, j = i + k) with
// k_first <= k < k_end and i + k < N form a triangle in (row i, diagonal k).
// It is cut into bands of KW = NT * D consecutive diagonals and each band
// into row tiles of R rows; one CTA sweeps one tile.  Thread t owns the D
// adjacent diagonals k0 + tD .. k0 + tD + D - 1 of its band and walks the
// tile's rows top to bottom, carrying one running score per diagonal
// (Lemma 1 / Lemma 2: drop the leaving term, add the entering one).
//
// Precision.  An FP32 running score drifts by about eps times the largest
// score seen since its last exact value, which is far above the small
// scores that matter (nearest neighbours).  The score is therefore replaced
// every B rows by an exact sum of its window, built from block sums: each
// thread keeps, per diagonal, the sums of the last Q = m / B blocks of B
// entering terms (a ring in shared memory); they are sums of non-negative
// terms, accurate relative to themselves, and their total is the window's
// score.  Cost: one extra FMA per cell plus Q adds every B rows.
//
// Minima.  Each cell is offered to its row (P[i], neighbour i + k on the
// right) and its column (P[j], neighbour j - k on the left).  A cell's
// 32-bit key is its score's bits with the low log2(D) bits replaced by the
// thread-local diagonal slot d; integer minima over these keys give the
// best slot with the paper's tie-break (smaller k first) for free.  Row keys
// are reduced over the D slots of a row; column keys are reduced in D
// rotating registers, since column c = i + k receives slot d from row
// c - k0 - tD - d.  A reduced key that can beat the tile's cached best
// (shared-memory thresholds loaded from the global keys) lowers that
// threshold and, if it was still the tile's best, goes to a global 64-bit
// atomicMin.
//
// Shared-memory layout.  The j-side series values of the entering and the
// leaving terms are kept in two copies offset by m, so that a thread's
// window starts at a multiple of D in both; each copy is padded with one
// word per D words so that the 32 lanes (stride D) hit 32 different banks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"

namespace mpk {

constexpr int SW_NT = 256;           // threads per CTA
constexpr int SW_D = 8;              // diagonals per thread
constexpr int SW_KW = SW_NT * SW_D;  // diagonals per band
constexpr int SW_QMAX = 8;           // ring blocks per diagonal
constexpr int SW_W = 2 * SW_D - 1;   // window values per D-row block


struct SweepArgs {
    const float *hi;  // series (FP32 part), zero beyond n
    const float *lo;  // low part for FP64 input, else nullptr
    unsigned long long *keys;
    int *err;
    long long n, N;
    long long k_first, k_end;  // diagonals [k_first, k_end)
    long long L;               // N - k_first: rows of band 0
    long long C;               // ceil(L / R): row tiles of band 0
    long long tiles;           // total number of tiles
    long long nb;              // number of bands
    int m, B, Q, R, q;         // q = KW / R
    int RL;                    // rows of the leaving copies: max(R, m + 1) rounded up to D
    float p;                   // exponent for K_PG
};

// Tiles are numbered band by band; band b has C - q b row tiles, so the
// first tile of band b is prefix(b) = b C - q b (b - 1) / 2.
__device__ __forceinline__ long long tile_prefix(const SweepArgs &a, long long b) {
    return b * a.C - static_cast<long long>(a.q) * b * (b - 1) / 2;
}

__device__ __forceinline__ void decode_tile(const SweepArgs &a, long long t, long long &b, long long &r) {
    const double cq = static_cast<double>(a.C) + 0.5 * a.q;
    const double disc = cq * cq - 2.0 * a.q * static_cast<double>(t);
    long long bb = static_cast<long long>((cq - sqrt(fmax(disc, 0.0))) / a.q);
    if (bb < 0) bb = 0;
    if (bb > a.nb - 1) bb = a.nb - 1;
    while (bb > 0 && tile_prefix(a, bb) > t) --bb;
    while (bb + 1 < a.nb && tile_prefix(a, bb + 1) <= t) ++bb;
    b = bb;
    r = t - tile_prefix(a, bb);
}

template <int KIND>
__device__ __forceinline__ float term(float x, float p) {
    if constexpr (KIND == K_P2) return x * x;
    else if constexpr (KIND == K_P1) return fabsf(x);
    else if constexpr (KIND == K_P3) { const float a = fabsf(x); return a * a * a; }
    else return __powf(fabsf(x), p);
}

__device__ __forceinline__ int cell_key(float s, int d) {
    return (__float_as_int(s) & ~(SW_D - 1)) | d;
}

// Non-negative score bits of a reduced key (negative drift -> 0).
__device__ __forceinline__ unsigned key_value(int key) {
    const int v = key & ~(SW_D - 1);
    return v < 0 ? 0u : static_cast<unsigned>(v);
}

// padded position of x in a j-side copy: one pad word after every D words
__host__ __device__ __forceinline__ int jpos(int x) { return x + x / SW_D; }

// One tile (band, rt) of one problem.  Every thread of the CTA calls it; it
// synchronises once (after staging) and may return early per thread after that.
template <int KIND, bool SPLIT>
__device__ __forceinline__ void sweep_tile(const SweepArgs &a, long long band, long long rt, unsigned char *smem) {
    const int R = a.R, m = a.m, B = a.B, Q = a.Q, RL = a.RL;
    const int tid = threadIdx.x;
    const long long k0 = a.k_first + band * SW_KW;
    const long long r0 = rt * R;

    // ---- shared memory
    //  TiE[u] = T[r0 + m - 1 + u]   u in [0, R)        entering, i side
    //  TiL[u] = T[r0 - 1 + u]       u in [0, RL)       leaving, i side (TiL[x + 1] = T[r0 + x])
    //  TjE[jpos(x)] = T[r0 + k0 + m - 1 + x], x in [0, KW + R)
    //  TjL[jpos(x)] = T[r0 + k0 - 1 + x],     x in [0, KW + RL)
    const int njE = jpos(SW_KW + R), njL = jpos(SW_KW + RL);
    float *TiE = reinterpret_cast<float *>(smem);
    float *TiL = TiE + R;
    float *TjE = TiL + RL;
    float *TjL = TjE + njE;
    float *TiEl = TjL + njL;  // low parts (SPLIT)
    float *TiLl = TiEl + (SPLIT ? R : 0);
    float *TjEl = TiLl + (SPLIT ? RL : 0);
    float *TjLl = TjEl + (SPLIT ? njE : 0);
    unsigned *thr_r = reinterpret_cast<unsigned *>(TjLl + (SPLIT ? njL : 0));
    unsigned *thr_c = thr_r + R;
    float *ring = reinterpret_cast<float *>(thr_c + SW_KW + R);

    auto ld = [&](long long g, float &h, float &l) {
        if (g >= 0 && g < a.n) {
            h = a.hi[g];
            if constexpr (SPLIT) l = a.lo[g];
        } else {
            h = 0.f;
            l = 0.f;
        }
    };
    for (int u = tid; u < R; u += SW_NT) {
        float h, l = 0.f;
        ld(r0 + m - 1 + u, h, l);
        TiE[u] = h;
        if constexpr (SPLIT) TiEl[u] = l;
    }
    for (int u = tid; u < RL; u += SW_NT) {
        float h, l = 0.f;
        ld(r0 - 1 + u, h, l);
        TiL[u] = h;
        if constexpr (SPLIT) TiLl[u] = l;
    }
    for (int x = tid; x < SW_KW + R; x += SW_NT) {
        float h, l = 0.f;
        ld(r0 + k0 + m - 1 + x, h, l);
        TjE[jpos(x)] = h;
        if constexpr (SPLIT) TjEl[jpos(x)] = l;
    }
    for (int x = tid; x < SW_KW + RL; x += SW_NT) {
        float h, l = 0.f;
        ld(r0 + k0 - 1 + x, h, l);
        TjL[jpos(x)] = h;
        if constexpr (SPLIT) TjLl[jpos(x)] = l;
    }
    for (int x = tid; x < R; x += SW_NT) {
        const long long g = r0 + x;
        thr_r[x] = g < a.N ? static_cast<unsigned>(a.keys[g] >> 32) : 0u;
    }
    for (int x = tid; x < SW_KW + R; x += SW_NT) {
        const long long g = r0 + k0 + x;
        thr_c[x] = g < a.N ? static_cast<unsigned>(a.keys[g] >> 32) : 0u;
    }
    __syncthreads();

    const long long kt = k0 + static_cast<long long>(tid) * SW_D;  // thread's first diagonal
    const long long nd_ll = a.k_end - kt;
    const int nd = nd_ll <= 0 ? 0 : (nd_ll >= SW_D ? SW_D : static_cast<int>(nd_ll));
    const long long lim_ll = a.N - kt - r0;  // cell (u, d) valid iff u + d < lim
    const int rows = nd == 0 || lim_ll <= 0 ? 0 : (lim_ll < R ? static_cast<int>(lim_ll) : R);
    if (rows == 0) return;
    const int lim = static_cast<int>(lim_ll < (long long)R + SW_D ? lim_ll : (long long)R + SW_D);
    const int ufull = nd == SW_D ? lim - (SW_D - 1) : 0;  // rows u < ufull have all D cells
    const float p = a.p;
    const int jb = tid * SW_D;  // thread's first local diagonal

    // ---- exact anchor at u = 0 from Q block sums:  sum_l term(T[r0+l] - T[r0+k+l])
    //      T[r0 + x] = TiL[x + 1],  T[r0 + k0 + jb + d + x] = TjL[jpos(jb + d + x + 1)]
    float s[SW_D], E[SW_D];
#pragma unroll
    for (int d = 0; d < SW_D; ++d) { s[d] = 0.f; E[d] = 0.f; }
    {
        float beta[SW_D];
#pragma unroll
        for (int d = 0; d < SW_D; ++d) beta[d] = 0.f;
        for (int x = 0; x < m; ++x) {
            const float ti = TiL[x + 1];
            float til = 0.f;
            if constexpr (SPLIT) til = TiLl[x + 1];
#pragma unroll
            for (int d = 0; d < SW_D; ++d) {
                const int pj = jpos(jb + d + x + 1);
                float e = ti - TjL[pj];
                if constexpr (SPLIT) e += til - TjLl[pj];
                if constexpr (KIND == K_P2) beta[d] = fmaf(e, e, beta[d]);
                else beta[d] += term<KIND>(e, p);
            }
            if ((x + 1) % B == 0) {
                const int qb = x / B;
#pragma unroll
                for (int d = 0; d < SW_D; ++d) {
                    ring[(qb * SW_D + d) * SW_NT + tid] = beta[d];
                    s[d] += beta[d];
                    beta[d] = 0.f;
                }
            }
        }
    }

    int col[SW_D];
#pragma unroll
    for (int d = 0; d < SW_D; ++d) col[d] = 0x7fffffff;

    int ulast = 0;
    for (int ub = 0; ub < rows; ub += SW_D) {
        // j-side windows of this block: wE[x] = TjE[jpos(jb + ub + x)], wL[x] = TjL[...]
        float wE[SW_W], wL[SW_W], wEl[SW_W], wLl[SW_W];
        const int pb = jpos(jb + ub);  // jb + ub is a multiple of D
#pragma unroll
        for (int x = 0; x < SW_W; ++x) {
            wE[x] = TjE[pb + x + x / SW_D];
            wL[x] = TjL[pb + x + x / SW_D];
            if constexpr (SPLIT) {
                wEl[x] = TjEl[pb + x + x / SW_D];
                wLl[x] = TjLl[pb + x + x / SW_D];
            } else {
                wEl[x] = 0.f;
                wLl[x] = 0.f;
            }
        }
#pragma unroll
        for (int ul = 0; ul < SW_D; ++ul) {
            const int u = ub + ul;
            if (u >= rows) break;
            if (u > 0) {
                const float ti_in = TiE[u], ti_out = TiL[u];
                float til_in = 0.f, til_out = 0.f;
                if constexpr (SPLIT) { til_in = TiEl[u]; til_out = TiLl[u]; }
#pragma unroll
                for (int d = 0; d < SW_D; ++d) {
                    float e = ti_in - wE[ul + d];
                    float f = ti_out - wL[ul + d];
                    if constexpr (SPLIT) {
                        e += til_in - wEl[ul + d];
                        f += til_out - wLl[ul + d];
                    }
                    if constexpr (KIND == K_P2) {
                        s[d] = fmaf(-f, f, fmaf(e, e, s[d]));
                        E[d] = fmaf(e, e, E[d]);
                    } else {
                        const float te = term<KIND>(e, p);
                        s[d] = (s[d] + te) - term<KIND>(f, p);
                        E[d] += te;
                    }
                }
                if (u % B == 0) {  // re-anchor: swap the leaving block for the new one
                    const int slot = (u / B - 1) % Q;
#pragma unroll
                    for (int d = 0; d < SW_D; ++d) {
                        ring[(slot * SW_D + d) * SW_NT + tid] = E[d];
                        E[d] = 0.f;
                        float acc = 0.f;
                        for (int qb = 0; qb < Q; ++qb) acc += ring[(qb * SW_D + d) * SW_NT + tid];
                        s[d] = acc;
                    }
                }
            }
            // ---- keys of this row's cells
            int key[SW_D];
            if (u < ufull) {
#pragma unroll
                for (int d = 0; d < SW_D; ++d) key[d] = cell_key(s[d], d);
            } else {
#pragma unroll
                for (int d = 0; d < SW_D; ++d)
                    key[d] = (d < nd && u + d < lim) ? cell_key(s[d], d) : 0x7fffffff;
            }
            // row minimum over the D slots
            int rk = key[0];
#pragma unroll
            for (int d = 1; d < SW_D; ++d) rk = min(rk, key[d]);
            // column minima: slot (u + d) % D holds column r0 + kt + u + d
#pragma unroll
            for (int d = 0; d < SW_D; ++d) {
                const int sl = (ul + d) % SW_D;
                col[sl] = min(col[sl], key[d]);
            }
            // row candidate
            if (rk != 0x7fffffff) {
                const unsigned v = key_value(rk);
                if (v <= thr_r[u]) {
                    const unsigned wmin = __reduce_min_sync(__activemask(), v);
                    if (v == wmin) {
                        const long long k = kt + (rk & (SW_D - 1));
                        if (v <= atomicMin(&thr_r[u], v)) atomicMin(&a.keys[r0 + u], make_key(v, k, 1));
                    }
                }
            }
            // column r0 + kt + u is complete (slot ul)
            {
                const int ck = col[ul];
                col[ul] = 0x7fffffff;
                if (ck != 0x7fffffff) {
                    const unsigned v = key_value(ck);
                    const int cl = jb + u;  // local column index
                    if (v <= thr_c[cl]) {
                        const long long k = kt + (ck & (SW_D - 1));
                        if (v <= atomicMin(&thr_c[cl], v)) atomicMin(&a.keys[r0 + kt + u], make_key(v, k, 0));
                    }
                }
            }
            ulast = u;
        }
    }
    // columns still open after the last row: slot sl holds column
    // r0 + kt + ulast + ((sl - ulast) mod D)
#pragma unroll
    for (int sl = 0; sl < SW_D; ++sl) {
        const int ck = col[sl];
        if (ck == 0x7fffffff) continue;
        const int delta = ((sl - ulast) % SW_D + SW_D) % SW_D;
        const int cl = jb + ulast + delta;
        const unsigned v = key_value(ck);
        if (v <= thr_c[cl]) {
            const long long k = kt + (ck & (SW_D - 1));
            if (v <= atomicMin(&thr_c[cl], v)) atomicMin(&a.keys[r0 + kt + ulast + delta], make_key(v, k, 0));
        }
    }
}

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(SW_NT, 2) sweep_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long band, rt;
    decode_tile(a, blockIdx.x, band, rt);
    if (rt < 0 || rt >= a.C - static_cast<long long>(a.q) * band) {  // cannot happen; never touch memory
        if (threadIdx.x == 0) atomicOr(&mp_device_error, ERR_BAD_TILE);
        return;
    }
    sweep_tile<KIND, SPLIT>(a, band, rt, smem);
}

// Rows held by the leaving copies (they also serve the anchor, which needs m + 1).
inline int sweep_rows_leaving(int R, int m) {
    int rl = R > m + 1 ? R : m + 1;
    return (rl + SW_D - 1) / SW_D * SW_D + SW_D;
}

// Shared-memory bytes of one sweep CTA.
inline size_t sweep_smem_bytes(int R, int m, int Q, bool split) {
    const int RL = sweep_rows_leaving(R, m);
    const size_t series = static_cast<size_t>(R) + RL + jpos(SW_KW + R) + jpos(SW_KW + RL);
    size_t b = series * sizeof(float) * (split ? 2 : 1);
    b += (static_cast<size_t>(R) + SW_KW + R) * sizeof(unsigned);
    b += static_cast<size_t>(Q) * SW_D * SW_NT * sizeof(float);
    return b;
}

}  // namespace mpk
