// a3-a5, fast path: the Euclidean diagonal sweep (Algorithm 1) and the
// p-norm sweep for p = 1 and 3 (Algorithm 3) for FP32 series with m a
// multiple of 32 (re-anchor interval B = m / Q: Q = 2 for p = 2, 4 for p = 1, 3).
//
// Same decomposition as the generic kernel (bands of KW diagonals, row
// tiles, D adjacent diagonals per thread), shaped for the FP32 pipes:
//
//  * Two row streams.  A tile of R = 2H rows is walked as two halves at
//    once: stream a covers rows r0 .. r0+H-1, stream b rows r0+H .. r0+2H-1.
//    Every diagonal carries one score per stream, held as a float2, so each
//    arithmetic step is one packed f32x2 instruction for two cells.
//
//  * Five packed operations per cell pair.  With e = t_{i+m-1} - t_{j+m-1}
//    (entering) and f = t_{i-1} - t_{j-1} (leaving), Lemma 1 is carried as
//        E += e^2,   F' += f^2,   s = E - F'
//    where, after each exact anchor A, E restarts at 0 and F' at -A; E is
//    also the sum of the current block of B entering terms that feeds the
//    ring of exact block sums (see the generic kernel), so the re-anchor
//    costs nothing per cell.  For p = 2 the ring holds Q = 2 blocks (one
//    re-anchor every m / 2 rows) and the other half of its space holds the
//    filter pass's saved state.
//
//  * Tagged minima.  Each score is tagged with its diagonal slot d in the low
//    log2(D) mantissa bits (one integer op per cell); tagged scores are still
//    floats ordered like the scores (to 2^-20 relative), and among equal
//    scores the smaller d, i.e. the smaller k, is smaller: the paper's
//    tie-break.  Rows are reduced with 3-input minima over the D slots;
//    columns (c = i + k) in D rotating slots, two rows at a time with 3-input
//    minima.  The winner's slot is read back from the tag, so a candidate
//    that passes its threshold costs two atomics and nothing else.
//
//  * Block filter (FILTER, for p = 2 on long series).  Each 8-row block first
//    runs the recurrence of E and F' alone and bounds the scores of each
//    group of V2_LBR rows from below by E(row before the group) - F'(last row
//    of the group), per diagonal (both sums only grow within a block); unless
//    some lane's bound could beat the loosest threshold of the rows and
//    columns its block feeds, the block is done without scores, tags or
//    slots.  Otherwise the block is replayed from the state saved in shared
//    memory at the block's start (stores on the load / store pipe instead of
//    32 register copies on the FMA pipe, and 32 registers fewer) with the
//    tracked bookkeeping above.
//
//  * Tall tiles.  A tile of R rows gives each stream Ht = R / 2 rows; on
//    long series R is several times 2 V2_H and the streams walk their rows in
//    sub-tiles of HS rows, each staged in shared memory in turn, carrying the
//    recurrence and the ring from one sub-tile to the next, so the O(m)
//    anchor from the definition is paid once per tile.
//
//  * Shared memory holds, per sub-tile, the j-side series as float2 pairs
//    (stream a, stream b) padded by 16 bytes every 64 so that each lane's
//    16-byte loads hit distinct banks, the i-side pairs, float thresholds
//    (the best tagged value known for each row / column of the sub-tile; the
//    column copy padded like the series), and, for the whole tile, the ring.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"

namespace mpk {

constexpr int V2_NT = 192;             // threads per CTA (two CTAs, 12 warps, per SM)
constexpr int V2_D = 8;                // diagonals per thread
constexpr int V2_KW = V2_NT * V2_D;    // diagonals per band
constexpr int V2_H = 1024;             // rows per stream of a one-step tile (staged at once)
constexpr int V2_R = 2 * V2_H;         // rows of a one-step tile
constexpr int V2_HT = 768;             // rows per stream of a sub-tile of a tall tile
constexpr int V2_LBR = 4;              // filter pass: rows per lower bound (divides V2_D)
constexpr int V2_QMAX = 4;             // ring space per diagonal, in blocks
// ring blocks in use: 2 for p = 2 (re-anchor every m / 2 rows; the other half
// of the ring's space holds the filter pass's saved state), 4 for p = 1, 3
__host__ __device__ constexpr int v2_ring_blocks(int kind) { return kind == K_P2 ? 2 : V2_QMAX; }
// shared memory of one CTA such that two fit on an SM (228 KB, 1 KB reserved per CTA)
constexpr size_t V2_SMEM_MAX = 113 * 1024;

struct Sweep2Args {
    const float *t;             // FP32 series, n values
    unsigned long long *keys;   // N profile keys
    long long n, N;
    long long k_first, k_end;   // diagonals [k_first, k_end)
    long long L;                // N - k_first: rows of band 0
    long long nb;               // bands
    long long tiles;
    long long R;                // rows per tile: V2_R, or a multiple of it (tall tiles: sub-tiles of V2_HT rows)
    int m, B, Q;
};

// ---- f32x2 helpers -----------------------------------------------------------------
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 ra, rb, rr;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rr;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}


// ---- tile enumeration ---------------------------------------------------------------
// Band b (diagonals k_first + b KW ...) has L_b = L - b KW rows and
// ceil(L_b / R) row tiles.  The first tile of band b is
//   prefix(b) = sum_{b' < b} floor((L - b' KW + R - 1) / R),
// a floor-sum of an arithmetic progression, evaluated in O(log) steps.
__host__ __device__ inline long long floor_sum(long long n, long long mdiv, long long a, long long b) {
    // sum_{i=0}^{n-1} floor((a i + b) / mdiv), a, b >= 0, mdiv > 0, by the standard
    // Euclid-like reduction for floor sums of a linear function (the method of the
    // AtCoder Library's floor_sum)
    long long ans = 0;
    while (true) {
        if (a >= mdiv) {
            ans += (n - 1) * n / 2 * (a / mdiv);
            a %= mdiv;
        }
        if (b >= mdiv) {
            ans += n * (b / mdiv);
            b %= mdiv;
        }
        const long long y_max = a * n + b;
        if (y_max < mdiv) break;
        n = y_max / mdiv;
        b = y_max % mdiv;
        const long long t = mdiv;
        mdiv = a;
        a = t;
    }
    return ans;
}

__host__ __device__ inline long long v2_prefix(long long L, long long b, long long R) {
    if (b <= 0) return 0;
    // i = b - 1 - b'  turns the decreasing progression into an increasing one
    return floor_sum(b, R, V2_KW, L + R - 1 - (b - 1) * V2_KW);
}

__device__ __forceinline__ bool v2_decode(const Sweep2Args &a, long long t, long long &band, long long &rt) {
    long long lo = 0, hi = a.nb - 1;  // largest b with prefix(b) <= t
    while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (v2_prefix(a.L, mid, a.R) <= t) lo = mid;
        else hi = mid - 1;
    }
    band = lo;
    rt = t - v2_prefix(a.L, lo, a.R);
    const long long Lb = a.L - lo * V2_KW;
    return rt >= 0 && rt * a.R < Lb;
}

// padded float2 index of x in the j-side array: 2 pad slots per 8
__host__ __device__ __forceinline__ int v2_jpos(int x) { return x + 2 * (x >> 3); }

// padded float index of column x in the column-threshold array: 1 pad per 8
__host__ __device__ __forceinline__ int v2_cpos(int x) { return x + (x >> 3); }

// Shared-memory layout of a tile with sub-tiles of HS rows per stream (byte
// offsets from the 16-byte-aligned base):
//   JT   nj float2          j-side pairs of KW + HS + m + 24 partner samples (padded)
//   IT   from JT + nj + 1   i-side pairs of HS + m + 24 rows (one past a 16-byte boundary)
//   thr_r, at thr_off + 12  row thresholds, nr = HS + 8 per stream (stream b after stream a)
//   thr_c, at thc_off       column thresholds (padded): cspan = KW + HS + 24 columns per
//                           stream; a tall tile keeps stream b's in a range of its own,
//                           a one-step tile (Ht <= HS) lets them overlap stream a's at Ht
//   ring, at ring_off       V2_QMAX blocks of D float2 per thread (for p = 2 the upper
//                           half holds the filter pass's saved state)
struct V2Smem {
    int nj, nr, cspan;
    int thr_off, thc_off, ring_off, bytes;
};
__host__ __device__ inline V2Smem v2_smem(int m, int HS, bool tall) {
    V2Smem L;
    L.nj = v2_jpos(V2_KW + HS + m + 24) + 2;  // even (HS, m multiples of 8)
    const int ni = HS + m + 26;                // even: thr_off stays 16-byte aligned
    L.nr = HS + 8;
    L.cspan = V2_KW + HS + 24;
    const int nc = (v2_cpos(tall ? 2 * L.cspan : L.cspan + HS) + 3) & ~3;
    L.thr_off = (L.nj + ni) * static_cast<int>(sizeof(float2));
    L.thc_off = L.thr_off + (3 + 2 * L.nr + 1) * static_cast<int>(sizeof(float));  // 2 HS + 20 floats: aligned
    L.ring_off = L.thc_off + nc * static_cast<int>(sizeof(float));
    L.bytes = L.ring_off + V2_QMAX * V2_D * V2_NT * static_cast<int>(sizeof(float2));
    return L;
}

inline int v2_sub_rows(long long R) { return R > V2_R ? V2_HT : V2_H; }

inline size_t sweep2_smem_bytes(int m, long long R) {
    return static_cast<size_t>(v2_smem(m, v2_sub_rows(R), R > V2_R).bytes);
}



// Tag a score with its slot: the low 3 bits of its FP32 pattern become d.
__device__ __forceinline__ float v2_tag(float s, int d) {
    return __int_as_float((__float_as_int(s) & ~(V2_D - 1)) | d);
}

// The same for the eight slots of one stream in a single 3-input logic op each:
// (bits & mask) | d with the mask in a register and d an immediate.
#define V2_TAG1(i)                                                                      \
    asm("lop3.b32 %0, %1, %2, " #i ", 0xEA;" : "=r"(o[i]) : "r"(__float_as_int(sb ? s[i].y : s[i].x)), "r"(mask))
__device__ __forceinline__ void v2_tag8(float *t, const float2 *s, bool sb, int mask) {
    int o[V2_D];
    V2_TAG1(0); V2_TAG1(1); V2_TAG1(2); V2_TAG1(3); V2_TAG1(4); V2_TAG1(5); V2_TAG1(6); V2_TAG1(7);
#pragma unroll
    for (int d = 0; d < V2_D; ++d) t[d] = __int_as_float(o[d]);
}
#undef V2_TAG1

// Threshold form of a value: its bits with all tag bits set, so that a tagged
// candidate with an equal (masked) value passes "<=" and the global key
// decides the tie.
__device__ __forceinline__ float v2_thr_form(unsigned value_bits) { return __uint_as_float(value_bits | (V2_D - 1)); }

// A tagged minimum that passed its threshold: tile threshold first, then the
// global key only if this candidate still matches or beats the tile's best
// (the threshold it replaced).  When all threads of a tile offer a candidate
// for the same row at once (thresholds still open early in a sweep), about
// ln(threads) of them reach the global atomic instead of every one.  Equal
// values still go out: a smaller k must win the key.
__device__ __forceinline__ void v2_emit(unsigned long long *keys, float *thr, int thr_idx, long long target,
                                        float tagged, long long kt, int right) {
    const int bits = __float_as_int(tagged);
    const unsigned v = bits < 0 ? 0u : static_cast<unsigned>(bits & ~(V2_D - 1));
    const int t = static_cast<int>(v | (V2_D - 1));
    const int old = atomicMin(reinterpret_cast<int *>(thr) + thr_idx, t);
    if (t <= old) atomicMin(&keys[target], make_key(v, kt + (bits & (V2_D - 1)), right));
}

// 1 if any of the eight tests a_i <= b_i holds: eight compares chained into
// one predicate.
__device__ __forceinline__ int v2_any_le(float a0, float b0, float a1, float b1, float a2, float b2, float a3,
                                         float b3, float a4, float b4, float a5, float b5, float a6, float b6,
                                         float a7, float b7) {
    int r;
    asm("{ .reg .pred p;\n\t"
        "setp.le.f32 p, %1, %2;\n\t"
        "setp.le.or.f32 p, %3, %4, p;\n\t"
        "setp.le.or.f32 p, %5, %6, p;\n\t"
        "setp.le.or.f32 p, %7, %8, p;\n\t"
        "setp.le.or.f32 p, %9, %10, p;\n\t"
        "setp.le.or.f32 p, %11, %12, p;\n\t"
        "setp.le.or.f32 p, %13, %14, p;\n\t"
        "setp.le.or.f32 p, %15, %16, p;\n\t"
        "selp.s32 %0, 1, 0, p; }"
        : "=r"(r)
        : "f"(a0), "f"(b0), "f"(a1), "f"(b1), "f"(a2), "f"(b2), "f"(a3), "f"(b3), "f"(a4), "f"(b4), "f"(a5),
          "f"(b5), "f"(a6), "f"(b6), "f"(a7), "f"(b7));
    return r;
}

__device__ __forceinline__ float v2_min8(const float *t) {
    return fminf(min3f(t[0], t[1], t[2]), min3f(t[3], t[4], min3f(t[5], t[6], t[7])));
}

__device__ __forceinline__ float2 v2_sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}

// acc + term(x) for both streams: x^2 (one packed FMA), |x| (one packed add, the
// absolute values taken as operand modifiers), |x|^3 = |x| x^2 (a packed multiply
// and a packed FMA).  Each lane rounds as the scalar operation would.
template <int KIND>
__device__ __forceinline__ float2 v2_acc(float2 x, float2 acc) {
    if constexpr (KIND == K_P1) {
        return __fadd2_rn(acc, make_float2(fabsf(x.x), fabsf(x.y)));
    } else if constexpr (KIND == K_P3) {
        const float2 x2 = __fmul2_rn(x, x);
        return __ffma2_rn(make_float2(fabsf(x.x), fabsf(x.y)), x2, acc);
    } else {
        return fma2(x, x, acc);
    }
}

// One tile (band, rt) of one problem.  Every thread of the CTA calls it and
// takes part in every sub-tile's staging barriers; a thread whose cells are
// done only stages after that.  TALL: a tile of a.R > V2_R rows walked in
// sub-tiles of V2_HT rows per stream; else one step of V2_H rows (a.R == V2_R).
template <int KIND, bool FILTER, bool TALL>
__device__ __forceinline__ void sweep2_tile(const Sweep2Args &a, long long band, long long rt,
                                            unsigned char *smem) {
    constexpr int HS = TALL ? V2_HT : V2_H;
    const int m = a.m, B = a.B, Q = a.Q;
    const int tid = threadIdx.x;
    const long long k0 = a.k_first + band * V2_KW;
    const long long r0 = rt * a.R;
    const long long Lb = a.L - band * V2_KW;  // rows where diagonal k0 is valid
    const int Rt = static_cast<int>(Lb - r0 < a.R ? Lb - r0 : a.R);
    // rows per stream, a multiple of 8 (stream b's extra rows lie beyond the
    // band's last row and are masked like any invalid cell)
    const int Ht = ((Rt + 1) / 2 + V2_D - 1) & ~(V2_D - 1);
    const V2Smem lay = v2_smem(m, HS, TALL);
    const int cboff = TALL ? V2_KW + HS + 24 : Ht;  // stream b's column x sits at thr_c[cpos(x + cboff)]

    // ---- shared memory, per sub-tile starting at stream-local row us
    //  JT[jpos(x)] = (t[y0 + x], t[y0 + x + Ht]),   y0 = r0 + us + k0 - 1
    //  IT[u]       = (t[r0 + us + u - 1], t[r0 + Ht + us + u - 1])
    //  thr_r[u], thr_rb[u]      threshold of row r0 + us + u (stream a), r0 + Ht + us + u (stream b)
    //  thr_c[cpos(x)]           threshold of column r0 + us + k0 + x (stream a),
    //  thr_c[cpos(x + cboff)]   of column r0 + Ht + us + k0 + x (stream b)
    float2 *JT = reinterpret_cast<float2 *>(smem);
    // IT sits one element past a 16-byte boundary, so that the pairs of rows
    // (8g+1, 8g+2), (8g+3, 8g+4), ... are 16-byte loads (m is a multiple of 32)
    float2 *IT = JT + lay.nj + 1;
    // thr_r is offset by 3 floats from a 16-byte boundary, so that the
    // thresholds of rows 8g+1 .. 8g+4 and 8g+5 .. 8g+8 are 16-byte loads
    float *thr_r = reinterpret_cast<float *>(smem + lay.thr_off) + 3;
    float *thr_rb = thr_r + (HS + 8);
    float *thr_c = reinterpret_cast<float *>(smem + lay.thc_off);
    float2 *ring = reinterpret_cast<float2 *>(smem + lay.ring_off);

    auto tv = [&](long long g) -> float { return (g >= 0 && g < a.n) ? a.t[g] : 0.f; };
    auto thr_of = [&](long long g) -> float {
        if (g < 0 || g >= a.N) return 0.f;
        const unsigned long long key = a.keys[g];
        return key == KEY_NONE ? __int_as_float(0x7f800000) : v2_thr_form(static_cast<unsigned>(key >> 32));
    };
    auto stage = [&](int us) {
        const long long y0 = r0 + us + k0 - 1, ia = r0 + us;
        for (int x = tid; x < V2_KW + HS + m + 24; x += V2_NT)
            JT[v2_jpos(x)] = make_float2(tv(y0 + x), tv(y0 + x + Ht));
        for (int u = tid; u < HS + m + 24; u += V2_NT) IT[u] = make_float2(tv(ia + u - 1), tv(ia + Ht + u - 1));
        for (int u = tid; u < HS + 8; u += V2_NT) {
            thr_r[u] = thr_of(ia + u);
            thr_rb[u] = thr_of(ia + Ht + u);
        }
        if (TALL) {
            for (int x = tid; x < lay.cspan; x += V2_NT) {
                thr_c[v2_cpos(x)] = thr_of(ia + k0 + x);
                thr_c[v2_cpos(x + cboff)] = thr_of(ia + Ht + k0 + x);
            }
        } else {
            for (int x = tid; x < lay.cspan + Ht; x += V2_NT) thr_c[v2_cpos(x)] = thr_of(ia + k0 + x);
        }
    };

    const int jb = tid * V2_D;
    const long long kt = k0 + jb;
    const long long nd_ll = a.k_end - kt;
    const int nd = nd_ll <= 0 ? 0 : (nd_ll >= V2_D ? V2_D : static_cast<int>(nd_ll));
    const long long lim_ll = a.N - kt - r0;  // stream-local row x of slot d is valid iff x + d < lim
    const long long lim_cap = 2LL * Ht + 16;
    const int lim = static_cast<int>(lim_ll <= 0 ? 0 : (lim_ll < lim_cap ? lim_ll : lim_cap));
    const int lim_b = lim - Ht;  // stream b: stream-local row u valid iff u + d < lim_b
    const int steps = lim < Ht ? lim : Ht;
    // rows u < ufast have all 16 cells (both streams, all D slots) valid
    int ufast = nd == V2_D ? lim_b - (V2_D - 1) : 0;
    ufast = ufast < 0 ? 0 : (ufast > steps ? steps : ufast);
    const float NONE = __int_as_float(0x7f800000);  // +inf: above every (finite) tagged score
    const int tag_mask = ~(V2_D - 1);

    float2 s[V2_D], E[V2_D], F[V2_D];
    int anchor_slot = 0;  // ring slot replaced at the next anchor row
    int next_anchor = B;  // anchor rows are B, 2B, ... (B is a multiple of 8)
    int us = 0;           // first stream-local row of the staged sub-tile

    // one step of the recurrence into a row (window offset o = ul + d)
    auto step = [&](bool anchor, float2 tl, float2 te, const float2 *WL, const float2 *WE, int ul) {
        if (anchor) {  // re-anchor: the block sum of entering terms just completed
#pragma unroll
            for (int d = 0; d < V2_D; ++d) {
                const float2 e = v2_sub(te, WE[ul + d]);
                E[d] = v2_acc<KIND>(e, E[d]);
                ring[(anchor_slot * V2_D + d) * V2_NT + tid] = E[d];
                float2 acc = make_float2(0.f, 0.f);
                for (int qb = 0; qb < Q; ++qb) acc = add2(acc, ring[(qb * V2_D + d) * V2_NT + tid]);
                s[d] = acc;
                E[d] = make_float2(0.f, 0.f);
                F[d] = make_float2(-acc.x, -acc.y);
            }
            anchor_slot = anchor_slot + 1 == Q ? 0 : anchor_slot + 1;
            next_anchor += B;
        } else {
#pragma unroll
            for (int d = 0; d < V2_D; ++d) {
                const float2 e = v2_sub(te, WE[ul + d]);
                const float2 f = v2_sub(tl, WL[ul + d]);
                E[d] = v2_acc<KIND>(e, E[d]);
                F[d] = v2_acc<KIND>(f, F[d]);
                s[d] = v2_sub(E[d], F[d]);
            }
        }
    };
    // targets take stream-local rows u; threshold indices are relative to the sub-tile
    auto row_tgt = [&](int u, int sb) { return r0 + (sb ? Ht : 0) + u; };
    auto col_tgt = [&](int uc, int sb) { return r0 + (sb ? Ht : 0) + kt + uc; };
    auto col_idx = [&](int uc, int sb) { return v2_cpos(jb + uc - us + (sb ? cboff : 0)); };

    // column slots (tagged), per stream; slot (u + d) % D holds column u + d
    float ca[V2_D], cb[V2_D];

    // masked processing of one row u whose scores are in s; j = u % D must be a
    // compile-time constant at every call so that the slots stay in registers
    auto masked_row = [&](int u, int j) {
        float ta = NONE, tb = NONE;
#pragma unroll
        for (int d = 0; d < V2_D; ++d) {
            const float va = (d < nd && u + d < lim) ? v2_tag(s[d].x, d) : NONE;
            const float vb = (d < nd && u + d < lim_b) ? v2_tag(s[d].y, d) : NONE;
            ta = fminf(ta, va);
            tb = fminf(tb, vb);
            const int sl = (j + d) % V2_D;
            ca[sl] = d == V2_D - 1 ? va : fminf(ca[sl], va);
            cb[sl] = d == V2_D - 1 ? vb : fminf(cb[sl], vb);
        }
        const int ul = u - us;
        if (ta != NONE && ta <= thr_r[ul]) v2_emit(a.keys, thr_r, ul, row_tgt(u, 0), ta, kt, 1);
        if (tb != NONE && tb <= thr_rb[ul]) v2_emit(a.keys, thr_rb, ul, row_tgt(u, 1), tb, kt, 1);
        if (ca[j] != NONE && ca[j] <= thr_c[col_idx(u, 0)]) v2_emit(a.keys, thr_c, col_idx(u, 0), col_tgt(u, 0), ca[j], kt, 0);
        if (cb[j] != NONE && cb[j] <= thr_c[col_idx(u, 1)]) v2_emit(a.keys, thr_c, col_idx(u, 1), col_tgt(u, 1), cb[j], kt, 0);
        ca[j] = NONE;
        cb[j] = NONE;
    };

    // Offer the partial minima of the columns still open after row ul
    // (slot sl holds column ul + ((sl - ul) mod D)) and close them: every
    // contribution is a genuine cell value, so emitting it early is exact.
    auto flush_open = [&](int ul) {
#pragma unroll
        for (int sl = 0; sl < V2_D; ++sl) {
            const int delta = ((sl - ul) % V2_D + V2_D) % V2_D;
            if (delta != 0) {
                const int uc = ul + delta;
                if (ca[sl] != NONE && ca[sl] <= thr_c[col_idx(uc, 0)])
                    v2_emit(a.keys, thr_c, col_idx(uc, 0), col_tgt(uc, 0), ca[sl], kt, 0);
                if (cb[sl] != NONE && cb[sl] <= thr_c[col_idx(uc, 1)])
                    v2_emit(a.keys, thr_c, col_idx(uc, 1), col_tgt(uc, 1), cb[sl], kt, 0);
            }
            ca[sl] = NONE;
            cb[sl] = NONE;
        }
    };

    bool done = nd == 0 || lim_ll <= 0;  // no cells left (open columns offered)
    int ub = 0;                          // rows up to ub are done
    bool group_valid = false;            // gca, gcb hold the column maxima for this block's columns 1..8
    float gca = NONE, gcb = NONE;
    constexpr bool kFilter = FILTER;
    // The rows of the staged sub-tile: row 0 (the anchors, first sub-tile only)
    // and the blocks of rows (us, us + HS] (a one-step tile: all its rows).
    auto walk = [&](bool first) {
        const float4 *JT4 = reinterpret_cast<const float4 *>(JT);
        if (first) {
            // ---- exact anchors at u = 0 from Q block sums (both streams at once)
            // T[r0 + l] = IT[l + 1], T[r0 + k + l] = JT[jb + d + l + 1]; l runs in groups of
            // 8 so that the j-side window comes in 16-byte loads (jb + l0 is a multiple of 8)
            for (int qb = 0; qb < Q; ++qb) {
                float2 beta[V2_D];
#pragma unroll
                for (int d = 0; d < V2_D; ++d) beta[d] = make_float2(0.f, 0.f);
                for (int l0 = qb * B; l0 < qb * B + B; l0 += V2_D) {  // B is a multiple of 8
                    float2 W[2 * V2_D];
                    const int qw = 5 * ((jb + l0) >> 3);
#pragma unroll
                    for (int q = 0; q < V2_D; ++q) {
                        const float4 w4 = JT4[qw + q + (q >= 4 ? 1 : 0)];
                        W[2 * q] = make_float2(w4.x, w4.y);
                        W[2 * q + 1] = make_float2(w4.z, w4.w);
                    }
#pragma unroll
                    for (int l = 0; l < V2_D; ++l) {
                        const float2 ti = IT[l0 + l + 1];
#pragma unroll
                        for (int d = 0; d < V2_D; ++d) {
                            const float2 e = v2_sub(ti, W[l + d + 1]);
                            beta[d] = v2_acc<KIND>(e, beta[d]);
                        }
                    }
                }
#pragma unroll
                for (int d = 0; d < V2_D; ++d) ring[(qb * V2_D + d) * V2_NT + tid] = beta[d];
            }
#pragma unroll
            for (int d = 0; d < V2_D; ++d) {
                float2 acc = make_float2(0.f, 0.f);
                for (int qb = 0; qb < Q; ++qb) acc = add2(acc, ring[(qb * V2_D + d) * V2_NT + tid]);
                s[d] = acc;
                E[d] = make_float2(0.f, 0.f);
                F[d] = make_float2(-acc.x, -acc.y);
            }
            // ---- row 0: the anchors themselves
#pragma unroll
            for (int d = 0; d < V2_D; ++d) { ca[d] = NONE; cb[d] = NONE; }
            masked_row(0, 0);
            if (FILTER) flush_open(0);  // with the filter, column slots never cross a block boundary
        }

        // ---- fast region: 8-row blocks (ub, ub + 8] with every cell valid --------------
        for (; ub + V2_D < ufast && (!TALL || ub < us + HS); ub += V2_D) {
            const int ubl = ub - us;  // the block's first row in the staged arrays
            // j-side samples of the block's leaving and entering windows; loaded
            // by each pass that uses them (the filter pass and, when it runs, the
            // tracked pass), so that they are not held across the filter decision
            float2 WL[2 * V2_D], WE[2 * V2_D];
            auto load_w = [&]() {
                const int qL = 5 * ((jb + ubl) >> 3), qE = 5 * ((jb + ubl + m) >> 3);
#pragma unroll
                for (int q = 0; q < V2_D; ++q) {
                    const int o = q + (q >= 4 ? 1 : 0);
                    const float4 l4 = JT4[qL + o], e4 = JT4[qE + o];
                    WL[2 * q] = make_float2(l4.x, l4.y);
                    WL[2 * q + 1] = make_float2(l4.z, l4.w);
                    WE[2 * q] = make_float2(e4.x, e4.y);
                    WE[2 * q + 1] = make_float2(e4.z, e4.w);
                }
            };
            const bool anc = ub + V2_D == next_anchor;  // B % 8 == 0: anchors fall on a block's last row
            // ---- filter pass (p = 2): the recurrence of E and F' and lower
            // bounds for the block's scores.  In the steady state no bound reaches
            // the loosest threshold of the rows and columns the block feeds, and
            // the block costs four packed operations per cell pair plus two per
            // diagonal and group.  The decision is taken for the warp's active
            // lanes together (one lane that needs the tracked pass costs the warp
            // that pass anyway).  Every block is filtered: sending the blocks after
            // a failure straight to the tracked pass measured slower on random
            // walks and on i.i.d. data alike.
            bool track = true;
            if (kFilter) {
                // the block's starting state, kept in the upper half of the ring's
                // space (p = 2 uses two of its four blocks) for a replay
                float4 *sv = reinterpret_cast<float4 *>(ring + 2 * V2_D * V2_NT) + tid;
#pragma unroll
                for (int p2 = 0; p2 < V2_D / 2; ++p2) {
                    sv[p2 * V2_NT] = make_float4(E[2 * p2].x, E[2 * p2].y, E[2 * p2 + 1].x, E[2 * p2 + 1].y);
                    sv[(p2 + V2_D / 2) * V2_NT] = make_float4(F[2 * p2].x, F[2 * p2].y, F[2 * p2 + 1].x, F[2 * p2 + 1].y);
                }
                const int slot0 = anchor_slot, next0 = next_anchor;
                // Within the block E and F' only grow (every step adds a term >= 0,
                // and rounding is monotone), so for a group of rows g+1 .. g+G,
                // E(g) - F'(g+G) is at most each of their scores s = E - F': one
                // subtraction per diagonal and group bounds G rows, and the pass
                // needs neither s nor per-cell minima.  The bound is loose by at
                // most G terms of the sums.  An anchor row (the block's last)
                // restarts E and F'; there the last group's other rows are bounded
                // with F' before the anchor and the anchor row by its exact value.
                load_w();
                float bma = NONE, bmb = NONE;
                auto fold = [&](float2 x0, float2 x1) {
                    bma = min3f(bma, x0.x, x1.x);
                    bmb = min3f(bmb, x0.y, x1.y);
                };
                {
                    const float4 *itl4 = reinterpret_cast<const float4 *>(IT + ubl + 1);
                    const float4 *ite4 = reinterpret_cast<const float4 *>(IT + ubl + m + 1);
                    float2 Eg[V2_D];  // E at the row before the current group
#pragma unroll
                    for (int d = 0; d < V2_D; ++d) Eg[d] = E[d];
#pragma unroll
                    for (int ul = 1; ul <= V2_D; ++ul) {
                        const float4 l4 = itl4[(ul - 1) >> 1], e4 = ite4[(ul - 1) >> 1];
                        const float2 tl = (ul & 1) ? make_float2(l4.x, l4.y) : make_float2(l4.z, l4.w);
                        const float2 te = (ul & 1) ? make_float2(e4.x, e4.y) : make_float2(e4.z, e4.w);
                        if (ul == V2_D && anc) {
                            if (V2_LBR > 1) {
#pragma unroll
                                for (int d = 0; d < V2_D; d += 2) fold(v2_sub(Eg[d], F[d]), v2_sub(Eg[d + 1], F[d + 1]));
                            }
                            step(true, tl, te, WL, WE, ul);
#pragma unroll
                            for (int d = 0; d < V2_D; d += 2) fold(s[d], s[d + 1]);
                        } else {
#pragma unroll
                            for (int d = 0; d < V2_D; ++d) {
                                E[d] = v2_acc<KIND>(v2_sub(te, WE[ul + d]), E[d]);
                                F[d] = v2_acc<KIND>(v2_sub(tl, WL[ul + d]), F[d]);
                            }
                            if (ul % V2_LBR == 0) {
#pragma unroll
                                for (int d = 0; d < V2_D; d += 2) fold(v2_sub(Eg[d], F[d]), v2_sub(Eg[d + 1], F[d + 1]));
                                if (ul < V2_D) {
#pragma unroll
                                    for (int d = 0; d < V2_D; ++d) Eg[d] = E[d];
                                }
                            }
                        }
                    }
                }
                // loosest thresholds of the 8 rows and 15 columns each stream's
                // scores feed; the maximum over columns 8g+1 .. 8g+8 is the one
                // read with the previous block (thresholds only decrease, so an
                // older read is looser)
                const float4 ra0 = *reinterpret_cast<const float4 *>(thr_r + ubl + 1);
                const float4 ra1 = *reinterpret_cast<const float4 *>(thr_r + ubl + 5);
                const float4 rb0 = *reinterpret_cast<const float4 *>(thr_rb + ubl + 1);
                const float4 rb1 = *reinterpret_cast<const float4 *>(thr_rb + ubl + 5);
                const float *fca = thr_c + v2_cpos(jb + ubl), *fcb = thr_c + v2_cpos(jb + cboff + ubl);
                if (!group_valid) {  // columns 1..8 of the block sit at padded offsets 1..7, 9
                    gca = max3f(fca[1], fca[2], fca[3]);
                    gcb = max3f(fcb[1], fcb[2], fcb[3]);
                    gca = max3f(gca, fca[4], fca[5]);
                    gcb = max3f(gcb, fcb[4], fcb[5]);
                    gca = max3f(gca, fca[6], fca[7]);
                    gcb = max3f(gcb, fcb[6], fcb[7]);
                    gca = fmaxf(gca, fca[9]);
                    gcb = fmaxf(gcb, fcb[9]);
                }
                // columns 9..16 at padded offsets 10..16, 18 (16 is the next block's first)
                float uga = max3f(fca[10], fca[11], fca[12]), ugb = max3f(fcb[10], fcb[11], fcb[12]);
                uga = max3f(uga, fca[13], fca[14]);
                ugb = max3f(ugb, fcb[13], fcb[14]);
                uga = max3f(uga, fca[15], fca[16]);
                ugb = max3f(ugb, fcb[15], fcb[16]);
                uga = fmaxf(uga, fca[18]);
                ugb = fmaxf(ugb, fcb[18]);
                float tma = max3f(ra0.x, ra0.y, ra0.z), tmb = max3f(rb0.x, rb0.y, rb0.z);
                tma = max3f(tma, ra0.w, ra1.x);
                tmb = max3f(tmb, rb0.w, rb1.x);
                tma = max3f(tma, ra1.y, ra1.z);
                tmb = max3f(tmb, rb1.y, rb1.z);
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
                if (__builtin_expect(track, 0)) {  // replay the block from the saved state, tracked
#pragma unroll
                    for (int p2 = 0; p2 < V2_D / 2; ++p2) {
                        const float4 e4 = sv[p2 * V2_NT], f4 = sv[(p2 + V2_D / 2) * V2_NT];
                        E[2 * p2] = make_float2(e4.x, e4.y);
                        E[2 * p2 + 1] = make_float2(e4.z, e4.w);
                        F[2 * p2] = make_float2(f4.x, f4.y);
                        F[2 * p2 + 1] = make_float2(f4.z, f4.w);
                    }
                    anchor_slot = slot0;
                    next_anchor = next0;
                }
            }
            if (track) {
                // ---- tracked pass of the block
                load_w();
                // per-block bases, so that every access below uses a constant offset
                const float *tra = thr_r + ubl, *trb = thr_rb + ubl;
                // jb + ubl and cboff are multiples of 8
                float *tca = thr_c + v2_cpos(jb + ubl), *tcb = thr_c + v2_cpos(jb + cboff + ubl);
                const float4 *itl4 = reinterpret_cast<const float4 *>(IT + ubl + 1);
                const float4 *ite4 = reinterpret_cast<const float4 *>(IT + ubl + m + 1);
#pragma unroll
                for (int pr = 0; pr < V2_D / 2; ++pr) {
                    const int ul0 = 2 * pr + 1, ul1 = ul0 + 1;  // rows u0 = ub + ul0, u1 = ub + ul1
                    const int cp0 = ul0 + (ul0 >> 3), cp1 = ul1 + (ul1 >> 3);  // padded column offsets
                    float t0a[V2_D], t0b[V2_D], t1a[V2_D], t1b[V2_D];
                    const float4 l4 = itl4[pr], e4 = ite4[pr];  // rows ul0 and ul1
                    step(false, make_float2(l4.x, l4.y), make_float2(e4.x, e4.y), WL, WE, ul0);
                    v2_tag8(t0a, s, false, tag_mask);
                    v2_tag8(t0b, s, true, tag_mask);
                    step(pr == V2_D / 2 - 1 && anc, make_float2(l4.z, l4.w), make_float2(e4.z, e4.w), WL, WE, ul1);
                    v2_tag8(t1a, s, false, tag_mask);
                    v2_tag8(t1b, s, true, tag_mask);
                    const float r0a = v2_min8(t0a), r0b = v2_min8(t0b), r1a = v2_min8(t1a), r1b = v2_min8(t1b);
                    // columns: slot j0 = u0 % D completes column u0, slot j1 completes column u1
                    const int j0 = ul0 % V2_D, j1 = ul1 % V2_D;
#pragma unroll
                    for (int jj = 0; jj < V2_D; ++jj) {
                        const int sl = (j0 + jj) % V2_D;
                        if (jj == 0) {
                            ca[sl] = fminf(ca[sl], t0a[0]);
                            cb[sl] = fminf(cb[sl], t0b[0]);
                        } else if (jj < V2_D - 1) {
                            ca[sl] = min3f(ca[sl], t0a[jj], t1a[jj - 1]);
                            cb[sl] = min3f(cb[sl], t0b[jj], t1b[jj - 1]);
                        } else {
                            ca[sl] = fminf(t0a[jj], t1a[jj - 1]);
                            cb[sl] = fminf(t0b[jj], t1b[jj - 1]);
                        }
                    }
                    // one test for the 8 candidates of this pair of rows; the rare
                    // pass re-tests each and emits it
                    const int any = v2_any_le(r0a, tra[ul0], r0b, trb[ul0], r1a, tra[ul1], r1b, trb[ul1], ca[j0],
                                              tca[cp0], cb[j0], tcb[cp0], ca[j1], tca[cp1], cb[j1], tcb[cp1]);
                    if (__builtin_expect(any != 0, 0)) {
                        const int u0 = ub + ul0, u1 = ub + ul1;
                        const int l0 = ubl + ul0, l1 = ubl + ul1;
                        if (r0a <= tra[ul0]) v2_emit(a.keys, thr_r, l0, row_tgt(u0, 0), r0a, kt, 1);
                        if (r0b <= trb[ul0]) v2_emit(a.keys, thr_rb, l0, row_tgt(u0, 1), r0b, kt, 1);
                        if (r1a <= tra[ul1]) v2_emit(a.keys, thr_r, l1, row_tgt(u1, 0), r1a, kt, 1);
                        if (r1b <= trb[ul1]) v2_emit(a.keys, thr_rb, l1, row_tgt(u1, 1), r1b, kt, 1);
                        if (ca[j0] <= tca[cp0]) v2_emit(a.keys, thr_c, col_idx(u0, 0), col_tgt(u0, 0), ca[j0], kt, 0);
                        if (cb[j0] <= tcb[cp0]) v2_emit(a.keys, thr_c, col_idx(u0, 1), col_tgt(u0, 1), cb[j0], kt, 0);
                        if (ca[j1] <= tca[cp1]) v2_emit(a.keys, thr_c, col_idx(u1, 0), col_tgt(u1, 0), ca[j1], kt, 0);
                        if (cb[j1] <= tcb[cp1]) v2_emit(a.keys, thr_c, col_idx(u1, 1), col_tgt(u1, 1), cb[j1], kt, 0);
                    }
                    ca[j0] = t1a[V2_D - 1];
                    cb[j0] = t1b[V2_D - 1];
                    ca[j1] = NONE;
                    cb[j1] = NONE;
                }
                if (kFilter) flush_open(ub + V2_D);
            }
        }

        // ---- tail: remaining rows, every cell checked (8-row groups keep u % D static)
        int ulast = ub;
        for (; ub + 1 < steps && (!TALL || ub < us + HS); ub += V2_D) {
#pragma unroll
            for (int ul = 1; ul <= V2_D; ++ul) {
                const int u = ub + ul;
                if (u >= steps) break;
                const int uo = u - us;
                float2 WLr[V2_D], WEr[V2_D];
#pragma unroll
                for (int d = 0; d < V2_D; ++d) {
                    WLr[d] = JT[v2_jpos(jb + uo + d)];
                    WEr[d] = JT[v2_jpos(jb + uo + d + m)];
                }
                step(u == next_anchor, IT[uo], IT[uo + m], WLr, WEr, 0);
                masked_row(u, ul % V2_D);
                ulast = u;
            }
        }
        if (ub + 1 >= steps) {
            // columns still open after the last row (slot sl holds column
            // ulast + ((sl - ulast) mod D)), offered while their sub-tile is staged
#pragma unroll
            for (int sl = 0; sl < V2_D; ++sl) {
                const int delta = ((sl - ulast) % V2_D + V2_D) % V2_D;
                if (delta == 0) continue;
                const int uc = ulast + delta;
                if (ca[sl] != NONE && ca[sl] <= thr_c[col_idx(uc, 0)])
                    v2_emit(a.keys, thr_c, col_idx(uc, 0), col_tgt(uc, 0), ca[sl], kt, 0);
                if (cb[sl] != NONE && cb[sl] <= thr_c[col_idx(uc, 1)])
                    v2_emit(a.keys, thr_c, col_idx(uc, 1), col_tgt(uc, 1), cb[sl], kt, 0);
            }
            done = true;
        }
    };

    if constexpr (!TALL) {  // one step: us stays 0
        stage(0);
        __syncthreads();
        if (!done) walk(true);
    } else {
        // Sub-tile sub covers the blocks of rows (sub HS, sub HS + HS]; row 0
        // belongs to sub-tile 0.  nst is the same for the whole CTA.
        const int nst = Ht > 1 ? (Ht - 2) / HS + 1 : 1;
        for (int sub = 0; sub < nst; ++sub) {
            if (sub > 0) __syncthreads();  // the previous sub-tile is done with shared memory
            us = sub * HS;
            stage(us);
            __syncthreads();
            if (!done) walk(sub == 0);
        }
    }
}

template <int KIND, bool FILTER, bool TALL>
__global__ void __launch_bounds__(V2_NT, 2) sweep2_kernel(const Sweep2Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long band, rt;
    if (!v2_decode(a, blockIdx.x, band, rt)) {
        if (threadIdx.x == 0) atomicOr(&mp_device_error, ERR_BAD_TILE);
        return;
    }
    sweep2_tile<KIND, FILTER, TALL>(a, band, rt, smem);
}

}  // namespace mpk
