// a3-a5 for the z-normalised distance (Algorithm 2): the fast FP32 sweep.
//
// The sweep carries, per diagonal, the centred covariance
//   cov_{i,j} = sum_l (t_{i+l} - mu_i)(t_{j+l} - mu_j)
// with the O(1) update cov_{i,j} = cov_{i-1,j-1} + df_{i-1} dg_{j-1} + df_{j-1} dg_{i-1}
// (Lemma 3's sums rewritten around the window means; df, dg, inv = 1/sqrt(S)
// come from the FP64 statistics kernel) and scores each cell with
//   q = 1 - rho = 1 - cov inv_i inv_j          (DZ^2 = 2 m q, Lemma 3).
// FP32 cannot hold cov to the 1e-9 relative that q ~ 0.01 needs over
// thousands of steps, so cov is a float-float pair (hi, lo): each step adds
// its two products to the low word (two chained packed FMAs; the words hold
// -cov and df is staged negated) and an error-free Fast2Sum folds the low
// word into the high word every second row: 6.5 packed f32x2 operations per
// cell pair with the score.
//
// Tiles are tall (a band of KW diagonals by up to S rows, split into two row
// streams packed in f32x2 as in the Euclidean fast path), so the anchor of
// each stream -- the covariance summed from the definition in float-float --
// is paid once per S/2 rows.  The tile is walked in chunks of RC rows per
// stream; each chunk's operands (j side: df, dg, inv of the partner windows;
// i side: df, dg, inv of the rows) and the current best values of its rows
// and columns are staged in shared memory, and the chunk's threads read them
// with conflict-free 16-byte loads.  Minima are tagged exactly as in the
// Euclidean fast path, and long series take the same block filter (the
// covariance words of a filtered block are saved in shared memory for the
// tracked replay).
//
// The same tall, chunked tiles also carry the Euclidean / p-norm sums for
// long windows (MODE = K_P2, K_P1, K_P3), where the other kernels would pay an
// O(m) anchor per 2048-row tile: the state is then the float-float sum of the
// Lemma 1 / 2 terms, the staged operands are the entering and leaving samples
// t_{w+m-1} and t_{w-1} of each window w, and a tile has S = max(8192, 8m)
// rows, so the O(m) anchor costs a fixed fraction of the tile.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"
#include "mp_sweep2.cuh"

namespace mpk {

constexpr int Z_NT = 128;             // threads per CTA
constexpr int Z_D = 8;                // diagonals per thread
constexpr int Z_KW = Z_NT * Z_D;      // diagonals per band
constexpr int Z_S = 8192;             // rows per tile of the long-window p-norm modes (at least; max(Z_S, 8m))
constexpr int Z_SZ = 65536;           // rows per tile of the z-normalised sweep (at least)
constexpr int Z_RC = 768;             // rows per stream per chunk

// Rows per tile for window length m: max(base, 8m) rounded up to 1024, with
// base Z_SZ for the z-normalised sweep (zn) and Z_S for the p-norm modes.  A
// tile pays one O(m) float-float anchor per stream and carries the state over
// S / 2 rows: the z-normalised float-float covariance drifts little (measured
// raw error 1.2e-6 at S = 8192, 2.9e-6 at S = 65536 on the C4 series) and
// taller tiles cut the anchors' share of the sweep from about a fifth to a
// few percent; the p-norm modes' sums of m terms of both signs drift more, so
// their tiles stay shorter.
__host__ __device__ inline long long z_rows_per_tile(long long m, bool zn) {
    long long S = 8 * m;
    S = (S + 1023) / 1024 * 1024;
    const long long base = zn ? Z_SZ : Z_S;
    return S < base ? base : S;
}

struct SweepZArgs {
    const float *t;                   // FP32 series (shifted like the means)
    const float *tlo;                 // low parts of a float64 series (t + tlo), or null
    const float *muh, *mul;           // window means as float-float (shifted)
    const float *df, *dg, *inv;       // operands (inv = NaN for a flat window)
    unsigned long long *keys;
    long long n, N, k_first, k_end, L, nb, tiles;
    long long S;                      // rows per tile (z_rows_per_tile(m, mode == K_Z))
    int m;
    float p;                          // exponent of the p-norm modes (unused for K_P1 / K_P2 / K_P3's own term)
};

__host__ __device__ inline long long z_prefix(long long L, long long b, long long S) {
    if (b <= 0) return 0;
    return floor_sum(b, S, Z_KW, L + S - 1 - (b - 1) * Z_KW);
}

__device__ __forceinline__ bool z_decode(const SweepZArgs &a, long long t, long long &band, long long &rt) {
    long long lo = 0, hi = a.nb - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (z_prefix(a.L, mid, a.S) <= t) lo = mid;
        else hi = mid - 1;
    }
    band = lo;
    rt = t - z_prefix(a.L, lo, a.S);
    const long long Lb = a.L - lo * Z_KW;
    return rt >= 0 && rt * a.S < Lb;
}

__host__ __device__ inline size_t sweepz_thr_bytes() {
    const size_t nc = v2_cpos(Z_KW + Z_RC + 16);  // column thresholds, per stream
    // + 3 floats in front: the row thresholds start 3 floats past a 16-byte boundary
    return ((3 + 2 * (Z_RC + 8) + 2 * nc) * sizeof(float) + 15) / 16 * 16;
}

inline size_t sweepz_smem_bytes() {
    const size_t nj = v2_jpos(Z_KW + Z_RC + 16) + 2;  // per j-side array
    const size_t ni = Z_RC + 16;                       // per i-side array
    // + the covariance words saved at the start of a filtered block (8 float4 per thread)
    return 3 * (nj + ni) * sizeof(float2) + sweepz_thr_bytes() + 8 * Z_NT * sizeof(float4);
}

__device__ __forceinline__ float2 z_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// One tile (band, rt) of one problem; every thread of the CTA calls it (the
// chunk loop synchronises the whole CTA).
// term of the p-norm modes for both streams: x^2, |x|, |x|^3
template <int MODE>
__device__ __forceinline__ float2 z_term(float2 x) {
    if constexpr (MODE == K_P1) return make_float2(fabsf(x.x), fabsf(x.y));
    else if constexpr (MODE == K_P3) {
        const float2 x2 = __fmul2_rn(x, x);
        return __fmul2_rn(make_float2(fabsf(x.x), fabsf(x.y)), x2);  // lanes round as scalar products
    } else return __fmul2_rn(x, x);
}

// FILTER: 0 no block filter; 1 the filter on each row's exact minimum
// 1 + inv_i min_d (ch + cl) inv_j; 2 (z-normalised only) the filter on the
// looser bound 1 + inv_i max_j(inv_j) min(0, min_d (ch + cl)) with the largest
// 1 / sqrt(S) of the block's 15 partner windows (one packed operation per cell
// pair instead of two; it pays where the windows' spreads vary little between
// neighbours, as for i.i.d. data, and loses on random walks).
template <int MODE, int FILTER>
__device__ __forceinline__ void sweepz_tile(const SweepZArgs &a, long long band, long long rt,
                                            unsigned char *smem) {
    constexpr bool ZN = MODE == K_Z;
    const int m = a.m;
    const int tid = threadIdx.x;
    const long long S = a.S;
    const long long k0 = a.k_first + band * Z_KW;
    const long long r0 = rt * S;
    const long long Lb = a.L - band * Z_KW;
    const int Rt = static_cast<int>(Lb - r0 < S ? Lb - r0 : S);
    const int Hs = ((Rt + 1) / 2 + Z_D - 1) & ~(Z_D - 1);  // rows per stream, a multiple of 8
    const long long rb = r0 + Hs;                           // first row of stream b

    const int njs = v2_jpos(Z_KW + Z_RC + 16) + 2;
    float2 *JF = reinterpret_cast<float2 *>(smem);
    float2 *JG = JF + njs;
    float2 *JI = JG + njs;
    float2 *IF = JI + njs;
    float2 *IG = IF + (Z_RC + 16);
    float2 *II = IG + (Z_RC + 16);
    // [2 (RC + 8)]: stream a rows, stream b rows; 3 floats past a 16-byte boundary, so
    // that the thresholds of chunk rows 8g+1 .. 8g+4 and 8g+5 .. 8g+8 are 16-byte loads
    float *thr_base = reinterpret_cast<float *>(II + (Z_RC + 16));
    float *thr_r = thr_base + 3;
    const int ncs = v2_cpos(Z_KW + Z_RC + 16);
    float *thr_ca = thr_r + 2 * (Z_RC + 8);
    float *thr_cb = thr_ca + ncs;
    float4 *zsave = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(thr_base) + sweepz_thr_bytes());

    const int jb = tid * Z_D;
    const long long kt = k0 + jb;
    const long long nd_ll = a.k_end - kt;
    const int nd = nd_ll <= 0 ? 0 : (nd_ll >= Z_D ? Z_D : static_cast<int>(nd_ll));
    const long long lim_ll = a.N - kt - r0;  // tile-local row x of slot d valid iff x + d < lim
    const bool active = nd > 0 && lim_ll > 0;
    const long long lim_cap = 2 * S + 16;
    const int lim = static_cast<int>(lim_ll <= 0 ? 0 : (lim_ll < lim_cap ? lim_ll : lim_cap));
    const int lim_b = lim - Hs;
    const int steps = lim < Hs ? lim : Hs;  // stream-local rows this thread walks
    int ufast = nd == Z_D ? lim_b - (Z_D - 1) : 0;
    ufast = ufast < 0 ? 0 : (ufast > steps ? steps : ufast);
    const float NONE = __int_as_float(0x7f800000);
    const float THR_OPEN = __int_as_float(0x7f7fffff);  // largest finite float
    const int tag_mask = ~(Z_D - 1);
    const float2 ONE = make_float2(1.f, 1.f);
    const bool r4 = ZN && m >= 64;  // fast blocks fold the low word every 4th row instead of every 2nd

    // ---- anchors in float-float, from the definition: the covariance of (row r_s,
    // diagonal kt + d) (z-norm, stored negated), or the sum of the p-norm terms
    float2 ch[Z_D], cl[Z_D];
    if (active && !ZN) {
        auto tv = [&](long long g) -> float { return (g >= 0 && g < a.n) ? __ldg(a.t + g) : 0.f; };
#pragma unroll
        for (int d = 0; d < Z_D; ++d) {
            ch[d] = make_float2(0.f, 0.f);
            cl[d] = make_float2(0.f, 0.f);
        }
        for (int l = 0; l < m; ++l) {
            const float2 ti = make_float2(tv(r0 + l), tv(rb + l));
#pragma unroll
            for (int d = 0; d < Z_D; ++d) {
                const float2 tj = make_float2(tv(r0 + kt + d + l), tv(rb + kt + d + l));
                const float2 p = z_term<MODE>(v2_sub(ti, tj));
                const float2 t = add2(ch[d], p);  // TwoSum(ch, p): exact whichever is larger
                const float2 bb = v2_sub(t, ch[d]);
                const float2 err = add2(v2_sub(ch[d], v2_sub(t, bb)), v2_sub(p, bb));
                cl[d] = add2(cl[d], err);
                ch[d] = t;
            }
        }
    }
    if (active && ZN) {
        auto tv = [&](long long g) -> float { return (g >= 0 && g < a.n) ? __ldg(a.t + g) : 0.f; };
        auto tl = [&](long long g) -> float { return (a.tlo && g >= 0 && g < a.n) ? __ldg(a.tlo + g) : 0.f; };
        auto mv = [&](const float *p, long long g) -> float { return (g >= 0 && g < a.N) ? __ldg(p + g) : 0.f; };
        const float2 mih = make_float2(mv(a.muh, r0), mv(a.muh, rb)), mil = make_float2(mv(a.mul, r0), mv(a.mul, rb));
        float2 mjh[Z_D], mjl[Z_D];
#pragma unroll
        for (int d = 0; d < Z_D; ++d) {
            mjh[d] = make_float2(mv(a.muh, r0 + kt + d), mv(a.muh, rb + kt + d));
            mjl[d] = make_float2(mv(a.mul, r0 + kt + d), mv(a.mul, rb + kt + d));
            ch[d] = make_float2(0.f, 0.f);
            cl[d] = make_float2(0.f, 0.f);
        }
        for (int l = 0; l < m; ++l) {
            const float2 ti = make_float2(tv(r0 + l), tv(rb + l));
            const float2 til = make_float2(tl(r0 + l), tl(rb + l));
            const float2 ci = add2(v2_sub(ti, mih), v2_sub(til, mil));
#pragma unroll
            for (int d = 0; d < Z_D; ++d) {
                const float2 tj = make_float2(tv(r0 + kt + d + l), tv(rb + kt + d + l));
                const float2 tjl = make_float2(tl(r0 + kt + d + l), tl(rb + kt + d + l));
                const float2 ncj = add2(v2_sub(mjh[d], tj), v2_sub(mjl[d], tjl));  // -(tj - mu_j)
                const float2 p = z_mul(ci, ncj);                   // -ci cj
                const float2 t = add2(ch[d], p);                   // Fast2Sum(ch, p)
                const float2 z = v2_sub(t, ch[d]);
                cl[d] = add2(cl[d], v2_sub(p, z));
                ch[d] = t;
            }
        }
    }

    float ca[Z_D], cb[Z_D];
    // the filter's maximum over columns 1..8 of the next fast block: its
    // columns 9..16 read with the previous block (fast blocks are contiguous;
    // thresholds only decrease, so an older read is looser)
    bool group_valid = false;
    float gca = 0.f, gcb = 0.f;
#pragma unroll
    for (int d = 0; d < Z_D; ++d) { ca[d] = NONE; cb[d] = NONE; }

    // score of the current state: q = 1 - cov inv_i inv_j (cov = -(ch + cl)), or
    // the p-norm sum ch + cl
    auto score = [&](float2 iI, float2 jI, int d) {
        if constexpr (ZN) {
            const float2 w = z_mul(iI, jI);
            return fma2(cl[d], w, fma2(ch[d], w, ONE));
        } else {
            return add2(ch[d], cl[d]);
        }
    };

    // Chunk c covers stream-local rows u0c + 1 .. u0c + RC (row 0, the anchor, is
    // done in chunk 0); blocks of 8 rows keep every window 16-byte aligned.
    const int nchunks_cta = Hs > 1 ? (Hs - 1 + Z_RC - 1) / Z_RC : 1;
    int ulast = 0;
    for (int c = 0; c < nchunks_cta; ++c) {
        const int u0c = c * Z_RC;
        __syncthreads();  // the previous chunk is done with shared memory
        {
            // j side: element x = partner index (j - 1) - y, y = r_s + u0c + k0 - 1
            const long long ya = r0 + u0c + k0 - 1, yb = ya + Hs;
            auto gv = [&](const float *p, long long g) -> float { return (g >= 0 && g < a.N) ? p[g] : 0.f; };
            const long long ia = r0 + u0c, ib = rb + u0c;
            if constexpr (ZN) {
                // df is staged negated (j side and i side), so that the covariance
                // step is two chained FMAs into the low word
                for (int x = tid; x < Z_KW + Z_RC + 16; x += Z_NT) {
                    const int px = v2_jpos(x);
                    JF[px] = make_float2(-gv(a.df, ya + x), -gv(a.df, yb + x));
                    JG[px] = make_float2(gv(a.dg, ya + x), gv(a.dg, yb + x));
                    JI[px] = make_float2(gv(a.inv, ya + x + 1), gv(a.inv, yb + x + 1));
                }
                // i side: chunk row ul uses df, dg of window i - 1 and inv of window i
                for (int ul = tid; ul < Z_RC + 16; ul += Z_NT) {
                    IF[ul] = make_float2(-gv(a.df, ia + ul - 1), -gv(a.df, ib + ul - 1));
                    IG[ul] = make_float2(gv(a.dg, ia + ul - 1), gv(a.dg, ib + ul - 1));
                    II[ul] = make_float2(gv(a.inv, ia + ul), gv(a.inv, ib + ul));
                }
            } else {
                // entering and leaving samples of window w = ya + x + 1 (j side) and
                // w = ia + ul (i side): t_{w+m-1} and t_{w-1}
                auto sv = [&](long long g) -> float { return (g >= 0 && g < a.n) ? a.t[g] : 0.f; };
                for (int x = tid; x < Z_KW + Z_RC + 16; x += Z_NT) {
                    const int px = v2_jpos(x);
                    JF[px] = make_float2(sv(ya + x + m), sv(yb + x + m));
                    JG[px] = make_float2(sv(ya + x), sv(yb + x));
                }
                for (int ul = tid; ul < Z_RC + 16; ul += Z_NT) {
                    IF[ul] = make_float2(sv(ia + ul + m - 1), sv(ib + ul + m - 1));
                    IG[ul] = make_float2(sv(ia + ul - 1), sv(ib + ul - 1));
                }
            }
            // A target without a candidate yet gets the largest finite threshold, not
            // +inf: a slot that saw only flat windows (NaN scores) holds +inf and
            // must not pass the unguarded tests of the fast blocks.
            auto thr_of = [&](long long g) -> float {
                if (g < 0 || g >= a.N) return 0.f;
                const unsigned long long key = a.keys[g];
                return key == KEY_NONE ? THR_OPEN : v2_thr_form(static_cast<unsigned>(key >> 32));
            };
            for (int ul = tid; ul < Z_RC + 8; ul += Z_NT) {
                thr_r[ul] = thr_of(ia + ul);
                thr_r[Z_RC + 8 + ul] = thr_of(ib + ul);
            }
            for (int x = tid; x < Z_KW + Z_RC + 16; x += Z_NT) {
                thr_ca[v2_cpos(x)] = thr_of(ia + k0 + x);
                thr_cb[v2_cpos(x)] = thr_of(ib + k0 + x);
            }
        }
        __syncthreads();
        if (!active || u0c >= steps) continue;

        float *trb_base = thr_r + (Z_RC + 8);
        auto col_tgt = [&](int uc, int sb) { return (sb ? rb : r0) + kt + uc; };
        auto row_tgt = [&](int u, int sb) { return (sb ? rb : r0) + u; };
        // masked processing of stream-local row u = u0c + ul (state already stepped)
        auto masked_row = [&](int u, int ul, int j) {
            float ta = NONE, tb = NONE;
#pragma unroll
            for (int d = 0; d < Z_D; ++d) {
                const float2 q = ZN ? score(II[ul], JI[v2_jpos(jb + d + ul)], d) : score(ONE, ONE, d);
                const float va = (d < nd && u + d < lim) ? v2_tag(q.x, d) : NONE;
                const float vb = (d < nd && u + d < lim_b) ? v2_tag(q.y, d) : NONE;
                ta = fminf(ta, va);
                tb = fminf(tb, vb);
                const int sl = (j + d) % Z_D;
                ca[sl] = d == Z_D - 1 ? va : fminf(ca[sl], va);
                cb[sl] = d == Z_D - 1 ? vb : fminf(cb[sl], vb);
            }
            // NONE (no valid cell) and NaN (a flat window) are never offered
            if (ta != NONE && ta <= thr_r[ul]) v2_emit(a.keys, thr_r, ul, row_tgt(u, 0), ta, kt, 1);
            if (tb != NONE && tb <= trb_base[ul]) v2_emit(a.keys, trb_base, ul, row_tgt(u, 1), tb, kt, 1);
            const int ci = v2_cpos(jb + ul);
            if (ca[j] != NONE && ca[j] <= thr_ca[ci]) v2_emit(a.keys, thr_ca, ci, col_tgt(u, 0), ca[j], kt, 0);
            if (cb[j] != NONE && cb[j] <= thr_cb[ci]) v2_emit(a.keys, thr_cb, ci, col_tgt(u, 1), cb[j], kt, 0);
            ca[j] = NONE;
            cb[j] = NONE;
        };
        // one covariance (or p-norm sum) step into chunk row ul, partner window offset o
        // The increments go into the low word only (p = 3: see below); renorm() folds it into the
        // high word with an error-free Fast2Sum after every second row (every
        // fourth for z-normalised windows of m >= 64, whose increments are small
        // against the covariance), so the low word never holds more than a few
        // increments and its rounding stays at the size of the increments' own
        // rounding.  Filter and tracked passes fold on the same rows, so a
        // block's state does not depend on which of them ran.
        auto step = [&](int ul, const float2 *WF, const float2 *WG, int o) {
            const float2 fi = IF[ul], gi = IG[ul];
#pragma unroll
            for (int d = 0; d < Z_D; ++d) {
                if constexpr (ZN) {  // cl - df_i dg_j - df_j dg_i (fi, WF hold -df)
                    cl[d] = fma2(fi, WG[o + d], fma2(WF[o + d], gi, cl[d]));
                } else {  // + term(e) - term(f), e = t_{i+m-1} - t_{j+m-1}, f = t_{i-1} - t_{j-1}
                    const float2 e = v2_sub(fi, WF[o + d]), f = v2_sub(gi, WG[o + d]);
                    if constexpr (MODE == K_P2) {
                        cl[d] = fma2(e, e, v2_sub(cl[d], z_mul(f, f)));
                    } else if constexpr (MODE == K_P3) {
                        // error-free: |x|^3 spans many orders of magnitude, and a
                        // rounded increment term(e) - term(f) would leave the FP32
                        // rounding of the largest term in the window sum long
                        // after that term left.  The leaving term comes off the
                        // high word with Fast2Sum (exact: the window holds it, so
                        // ch >= term(f) / 2), the entering one goes on with Fast2Sum
                        // after ordering the two by size (both are >= 0, so the
                        // larger value is the larger magnitude; the ordering runs on
                        // the ALU pipe, a TwoSum would take three more FMA-pipe
                        // operations), and only their rounding errors reach the low
                        // word; the sum is then the exact sum of the window's FP32
                        // terms to float-float precision.
                        const float2 xf = z_term<MODE>(f), xe = z_term<MODE>(e);
                        const float2 s1 = v2_sub(ch[d], xf);
                        const float2 e1 = v2_sub(v2_sub(ch[d], s1), xf);
                        const float2 hi = make_float2(fmaxf(s1.x, xe.x), fmaxf(s1.y, xe.y));
                        const float2 lo = make_float2(fminf(s1.x, xe.x), fminf(s1.y, xe.y));
                        const float2 s2 = add2(hi, lo);
                        const float2 e2 = v2_sub(lo, v2_sub(s2, hi));
                        ch[d] = s2;
                        cl[d] = add2(cl[d], add2(e1, e2));
                    } else {
                        cl[d] = add2(cl[d], v2_sub(z_term<MODE>(e), z_term<MODE>(f)));
                    }
                }
            }
        };
        auto renorm = [&]() {
#pragma unroll
            for (int d = 0; d < Z_D; ++d) {
                const float2 t = add2(ch[d], cl[d]);  // Fast2Sum(ch, cl)
                cl[d] = v2_sub(cl[d], v2_sub(t, ch[d]));
                ch[d] = t;
            }
        };

        // Offer the partial minima of the columns still open after stream-local
        // row ul (slot sl holds column ul + ((sl - ul) mod D)) and close them.
        auto flush_open = [&](int ul) {
#pragma unroll
            for (int sl = 0; sl < Z_D; ++sl) {
                const int delta = ((sl - ul) % Z_D + Z_D) % Z_D;
                if (delta != 0) {
                    const int uc = ul + delta;
                    const int ci = v2_cpos(jb + uc - u0c);
                    if (ca[sl] != NONE && ca[sl] <= thr_ca[ci])
                        v2_emit(a.keys, thr_ca, ci, col_tgt(uc, 0), ca[sl], kt, 0);
                    if (cb[sl] != NONE && cb[sl] <= thr_cb[ci])
                        v2_emit(a.keys, thr_cb, ci, col_tgt(uc, 1), cb[sl], kt, 0);
                }
                ca[sl] = NONE;
                cb[sl] = NONE;
            }
        };

        if (c == 0) {
            masked_row(0, 0, 0);  // the anchor row
            if (FILTER) flush_open(0);  // with the filter, column slots never cross a fast block
        }
        const float4 *JF4 = reinterpret_cast<const float4 *>(JF);
        const float4 *JG4 = reinterpret_cast<const float4 *>(JG);
        const float4 *JI4 = reinterpret_cast<const float4 *>(JI);
        for (int ulb = 0; ulb < Z_RC; ulb += Z_D) {
            const int ufirst = u0c + ulb + 1;
            if (ufirst >= steps) break;
            if (u0c + ulb + Z_D < ufast) {
                // ---- fast block: rows ufirst .. ufirst + 7, all cells valid
                float2 WF[2 * Z_D], WG[2 * Z_D], WI[2 * Z_D];
                bool track = true;
                const int qb = 5 * ((jb + ulb) >> 3);
#pragma unroll
                for (int q = 0; q < Z_D; ++q) {
                    const int o = qb + q + (q >= 4 ? 1 : 0);
                    const float4 f4 = JF4[o], g4 = JG4[o];
                    const float4 i4 = ZN ? JI4[o] : make_float4(1.f, 1.f, 1.f, 1.f);
                    WF[2 * q] = make_float2(f4.x, f4.y);
                    WF[2 * q + 1] = make_float2(f4.z, f4.w);
                    WG[2 * q] = make_float2(g4.x, g4.y);
                    WG[2 * q + 1] = make_float2(g4.z, g4.w);
                    WI[2 * q] = make_float2(i4.x, i4.y);
                    WI[2 * q + 1] = make_float2(i4.z, i4.w);
                }
                const float *tra = thr_r + ulb, *trb = trb_base + ulb;
                const float *tca = thr_ca + v2_cpos(jb + ulb), *tcb = thr_cb + v2_cpos(jb + ulb);
                if (FILTER) {
                    // ---- filter pass: the covariance steps and one running minimum of the
                    // block's scores per stream against the loosest threshold of the rows
                    // and columns they feed; the warp replays the block tracked (from the
                    // words saved in shared memory) only if some lane could pass
#pragma unroll
                    for (int p2 = 0; p2 < Z_D / 2; ++p2) {
                        zsave[p2 * Z_NT + tid] = make_float4(ch[2 * p2].x, ch[2 * p2].y, ch[2 * p2 + 1].x, ch[2 * p2 + 1].y);
                        zsave[(p2 + 4) * Z_NT + tid] =
                            make_float4(cl[2 * p2].x, cl[2 * p2].y, cl[2 * p2 + 1].x, cl[2 * p2 + 1].y);
                    }
                    float bma = NONE, bmb = NONE;
                    // FILTER == 2: the largest 1 / sqrt(S) of the block's 15 partner windows
                    float ima = 0.f, imb = 0.f;
                    if constexpr (ZN && FILTER == 2) {
                        ima = max3f(WI[1].x, WI[2].x, WI[3].x);
                        imb = max3f(WI[1].y, WI[2].y, WI[3].y);
#pragma unroll
                        for (int x = 4; x < 16; x += 2) {
                            ima = max3f(ima, WI[x].x, WI[x + 1].x);
                            imb = max3f(imb, WI[x].y, WI[x + 1].y);
                        }
                    }
#pragma unroll
                    for (int ul = 1; ul <= Z_D; ++ul) {
                        step(ulb + ul, WF, WG, ul);
                        // every 4th row the z-normalised state is folded (Fast2Sum) before its
                        // bound, which then needs the high word alone (the low word is below
                        // half an ulp of it, inside the margin); the folds fall on the same rows
                        // as in the tracked pass, so the block's end state does not change
                        constexpr bool kFold = ZN;
                        const bool fold4 = kFold && (ul & 3) == 0;
                        if (fold4) renorm();
                        if constexpr (ZN && FILTER == 2) {
                            // q = 1 + (ch + cl) inv_i inv_j >= 1 + min(0, min_d (ch + cl)) inv_i inv_max
                            // (flat partners have inv = NaN, which the maximum skips)
                            float rma = 0.f, rmb = 0.f;
#pragma unroll
                            for (int d = 0; d < Z_D; d += 2) {
                                const float2 va = fold4 ? ch[d] : add2(ch[d], cl[d]);
                                const float2 vb = fold4 ? ch[d + 1] : add2(ch[d + 1], cl[d + 1]);
                                rma = min3f(rma, va.x, vb.x);
                                rmb = min3f(rmb, va.y, vb.y);
                            }
                            const float2 iI = II[ulb + ul];
                            bma = fminf(bma, fmaf(rma * ima, iI.x, 1.f));
                            bmb = fminf(bmb, fmaf(rmb * imb, iI.y, 1.f));
                        } else if constexpr (ZN) {
                            // q = 1 + (ch + cl) inv_i inv_j and inv_i > 0 is common to the
                            // row: its minimum is 1 + inv_i min_d (ch + cl) inv_j, two packed
                            // operations per cell pair instead of three (flat windows have
                            // inv = NaN, which the minima skip)
                            float rma = NONE, rmb = NONE;
#pragma unroll
                            for (int d = 0; d < Z_D; d += 2) {
                                const float2 va = fold4 ? z_mul(ch[d], WI[ul + d])
                                                        : fma2(cl[d], WI[ul + d], z_mul(ch[d], WI[ul + d]));
                                const float2 vb = fold4 ? z_mul(ch[d + 1], WI[ul + d + 1])
                                                        : fma2(cl[d + 1], WI[ul + d + 1], z_mul(ch[d + 1], WI[ul + d + 1]));
                                rma = min3f(rma, va.x, vb.x);
                                rmb = min3f(rmb, va.y, vb.y);
                            }
                            const float2 iI = II[ulb + ul];
                            bma = fminf(bma, fmaf(rma, iI.x, 1.f));
                            bmb = fminf(bmb, fmaf(rmb, iI.y, 1.f));
                        } else {
#pragma unroll
                            for (int d = 0; d < Z_D; d += 2) {
                                const float2 qa = score(ONE, ONE, d);
                                const float2 qb = score(ONE, ONE, d + 1);
                                bma = min3f(bma, qa.x, qb.x);
                                bmb = min3f(bmb, qa.y, qb.y);
                            }
                        }
                        if (!fold4 && (ul & 1) == 0 && (!r4 || (ul & 3) == 0)) renorm();
                    }
                    if constexpr (ZN) {
                        // the row form rounds differently from the tracked pass's q
                        // (by a few units in the last place of q) and the tags move a
                        // score by up to 7 units: lower the minimum by more than both
                        // (NONE, the minimum of an all-flat block, becomes NaN and
                        // passes no test)
                        bma = bma - fmaxf(2e-5f, fabsf(bma) * 0x1p-18f);
                        bmb = bmb - fmaxf(2e-5f, fabsf(bmb) * 0x1p-18f);
                    }
                    const float4 ra0 = *reinterpret_cast<const float4 *>(tra + 1);
                    const float4 ra1 = *reinterpret_cast<const float4 *>(tra + 5);
                    const float4 rb0 = *reinterpret_cast<const float4 *>(trb + 1);
                    const float4 rb1 = *reinterpret_cast<const float4 *>(trb + 5);
                    float tma = max3f(ra0.x, ra0.y, ra0.z), tmb = max3f(rb0.x, rb0.y, rb0.z);
                    tma = max3f(tma, ra0.w, ra1.x);
                    tmb = max3f(tmb, rb0.w, rb1.x);
                    tma = max3f(tma, ra1.y, ra1.z);
                    tmb = max3f(tmb, rb1.y, rb1.z);
                    if (!group_valid) {  // columns 1..8 at padded offsets 1..7, 9
                        gca = max3f(tca[1], tca[2], tca[3]);
                        gcb = max3f(tcb[1], tcb[2], tcb[3]);
                        gca = max3f(gca, tca[4], tca[5]);
                        gcb = max3f(gcb, tcb[4], tcb[5]);
                        gca = max3f(gca, tca[6], tca[7]);
                        gcb = max3f(gcb, tcb[6], tcb[7]);
                        gca = fmaxf(gca, tca[9]);
                        gcb = fmaxf(gcb, tcb[9]);
                    }
                    // columns 9..16 at padded offsets 10..16, 18 (16 is the next block's first)
                    float uga = max3f(tca[10], tca[11], tca[12]), ugb = max3f(tcb[10], tcb[11], tcb[12]);
                    uga = max3f(uga, tca[13], tca[14]);
                    ugb = max3f(ugb, tcb[13], tcb[14]);
                    uga = max3f(uga, tca[15], tca[16]);
                    ugb = max3f(ugb, tcb[15], tcb[16]);
                    uga = fmaxf(uga, tca[18]);
                    ugb = fmaxf(ugb, tcb[18]);
                    tma = max3f(tma, ra1.w, gca);
                    tmb = max3f(tmb, rb1.w, gcb);
                    tma = fmaxf(tma, uga);
                    tmb = fmaxf(tmb, ugb);
                    gca = uga;
                    gcb = ugb;
                    group_valid = true;
                    // a tagged score is at least the score with its tag bits cleared
                    track = __any_sync(__activemask(), __int_as_float(__float_as_int(bma) & tag_mask) <= tma ||
                                                           __int_as_float(__float_as_int(bmb) & tag_mask) <= tmb);
                    if (__builtin_expect(track, 0)) {
#pragma unroll
                        for (int p2 = 0; p2 < Z_D / 2; ++p2) {
                            const float4 h = zsave[p2 * Z_NT + tid], l = zsave[(p2 + 4) * Z_NT + tid];
                            ch[2 * p2] = make_float2(h.x, h.y);
                            ch[2 * p2 + 1] = make_float2(h.z, h.w);
                            cl[2 * p2] = make_float2(l.x, l.y);
                            cl[2 * p2 + 1] = make_float2(l.z, l.w);
                        }
                    }
                }
                if (track) {
#pragma unroll
                for (int pr = 0; pr < Z_D / 2; ++pr) {
                    const int ul0 = 2 * pr + 1, ul1 = ul0 + 1;  // block-local rows
                    const int cp0 = ul0 + (ul0 >> 3), cp1 = ul1 + (ul1 >> 3);
                    float t0a[Z_D], t0b[Z_D], t1a[Z_D], t1b[Z_D];
                    float2 q[Z_D];
                    step(ulb + ul0, WF, WG, ul0);
#pragma unroll
                    for (int d = 0; d < Z_D; ++d) q[d] = score(ZN ? II[ulb + ul0] : ONE, WI[ul0 + d], d);
                    v2_tag8(t0a, q, false, tag_mask);
                    v2_tag8(t0b, q, true, tag_mask);
                    step(ulb + ul1, WF, WG, ul1);
#pragma unroll
                    for (int d = 0; d < Z_D; ++d) q[d] = score(ZN ? II[ulb + ul1] : ONE, WI[ul1 + d], d);
                    if (!r4 || (pr & 1)) renorm();
                    v2_tag8(t1a, q, false, tag_mask);
                    v2_tag8(t1b, q, true, tag_mask);
                    const float r0a = v2_min8(t0a), r0b = v2_min8(t0b), r1a = v2_min8(t1a), r1b = v2_min8(t1b);
                    const int j0 = ul0 % Z_D, j1 = ul1 % Z_D;
#pragma unroll
                    for (int jj = 0; jj < Z_D; ++jj) {
                        const int sl = (j0 + jj) % Z_D;
                        if (jj == 0) {
                            ca[sl] = fminf(ca[sl], t0a[0]);
                            cb[sl] = fminf(cb[sl], t0b[0]);
                        } else if (jj < Z_D - 1) {
                            ca[sl] = min3f(ca[sl], t0a[jj], t1a[jj - 1]);
                            cb[sl] = min3f(cb[sl], t0b[jj], t1b[jj - 1]);
                        } else {
                            ca[sl] = fminf(t0a[jj], t1a[jj - 1]);
                            cb[sl] = fminf(t0b[jj], t1b[jj - 1]);
                        }
                    }
                    const int any = v2_any_le(r0a, tra[ul0], r0b, trb[ul0], r1a, tra[ul1], r1b, trb[ul1], ca[j0],
                                              tca[cp0], cb[j0], tcb[cp0], ca[j1], tca[cp1], cb[j1], tcb[cp1]);
                    if (__builtin_expect(any != 0, 0)) {
                        const int u0 = u0c + ulb + ul0, u1 = u0 + 1;
                        const int r_0 = ulb + ul0, r_1 = r_0 + 1;  // chunk-local rows
                        if (r0a <= tra[ul0]) v2_emit(a.keys, thr_r, r_0, row_tgt(u0, 0), r0a, kt, 1);
                        if (r0b <= trb[ul0]) v2_emit(a.keys, trb_base, r_0, row_tgt(u0, 1), r0b, kt, 1);
                        if (r1a <= tra[ul1]) v2_emit(a.keys, thr_r, r_1, row_tgt(u1, 0), r1a, kt, 1);
                        if (r1b <= trb[ul1]) v2_emit(a.keys, trb_base, r_1, row_tgt(u1, 1), r1b, kt, 1);
                        const int ci0 = v2_cpos(jb + r_0), ci1 = v2_cpos(jb + r_1);
                        if (ca[j0] <= tca[cp0]) v2_emit(a.keys, thr_ca, ci0, col_tgt(u0, 0), ca[j0], kt, 0);
                        if (cb[j0] <= tcb[cp0]) v2_emit(a.keys, thr_cb, ci0, col_tgt(u0, 1), cb[j0], kt, 0);
                        if (ca[j1] <= tca[cp1]) v2_emit(a.keys, thr_ca, ci1, col_tgt(u1, 0), ca[j1], kt, 0);
                        if (cb[j1] <= tcb[cp1]) v2_emit(a.keys, thr_cb, ci1, col_tgt(u1, 1), cb[j1], kt, 0);
                    }
                    ca[j0] = t1a[Z_D - 1];
                    cb[j0] = t1b[Z_D - 1];
                    ca[j1] = NONE;
                    cb[j1] = NONE;
                }
                if (FILTER) flush_open(u0c + ulb + Z_D);
                }
                ulast = u0c + ulb + Z_D;
            } else {
                // ---- masked rows, one at a time (u % 8 stays a compile-time constant)
#pragma unroll
                for (int ui = 1; ui <= Z_D; ++ui) {
                    const int u = u0c + ulb + ui;
                    if (u >= steps) break;
                    const int ul = ulb + ui;
                    float2 WFr[Z_D], WGr[Z_D];
#pragma unroll
                    for (int d = 0; d < Z_D; ++d) {
                        const int px = v2_jpos(jb + d + ul);
                        WFr[d] = JF[px];
                        WGr[d] = JG[px];
                    }
                    step(ul, WFr, WGr, 0);
                    renorm();
                    masked_row(u, ul, ui % Z_D);
                    ulast = u;
                }
            }
        }
        if (ulast == steps - 1 && ulast >= u0c && (ulast > u0c || c == 0)) {
            // this thread's last row is in this chunk: flush the open columns
            // (slot sl holds column ulast + ((sl - ulast) mod D))
#pragma unroll
            for (int sl = 0; sl < Z_D; ++sl) {
                const int delta = ((sl - ulast) % Z_D + Z_D) % Z_D;
                if (delta == 0) continue;
                const int uc = ulast + delta;
                const int ci = v2_cpos(jb + uc - u0c);
                if (ca[sl] != NONE && ca[sl] <= thr_ca[ci]) v2_emit(a.keys, thr_ca, ci, col_tgt(uc, 0), ca[sl], kt, 0);
                if (cb[sl] != NONE && cb[sl] <= thr_cb[ci]) v2_emit(a.keys, thr_cb, ci, col_tgt(uc, 1), cb[sl], kt, 0);
            }
        }
    }
}

template <int MODE, int FILTER>
__global__ void __launch_bounds__(Z_NT, 2) sweepz_kernel(const SweepZArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long band, rt;
    if (!z_decode(a, blockIdx.x, band, rt)) {
        if (threadIdx.x == 0) atomicOr(&mp_device_error, ERR_BAD_TILE);
        return;
    }
    sweepz_tile<MODE, FILTER>(a, band, rt, smem);
}

}  // namespace mpk
