// C ABI of libmp (declared in include/mp.h): argument checks, workspace
// layout and the launch sequence of the matrix-profile sweep
//   a1 convert -> [a2 stats] -> keys init -> a3-a5 sweep -> a6 finalize.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "mp.h"
#include <nvtx3/nvToolsExt.h>
#include "mp_device.cuh"
#include "mp_prep.cuh"
#include "mp_kernels.h"
#include "mp_launch.cuh"
#include "mp_batch_prep.cuh"
#include "mp_stream.cuh"

namespace {

thread_local char g_err[512] = "";
thread_local cudaEvent_t g_ev_start = nullptr, g_ev_end = nullptr;
std::atomic<unsigned long long> g_launches{0};

// Count one kernel launch of this library (reported by mp_launch_count).
inline void counted(int n = 1) { g_launches.fetch_add(static_cast<unsigned long long>(n)); }

// NVTX range over one stage of a call (seen by profilers that record NVTX;
// otherwise a no-op).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Bracket the sweep kernel with the caller's profiling events, if set.
struct SweepEvents {
    cudaStream_t st;
    explicit SweepEvents(cudaStream_t s) : st(s) {
        if (g_ev_start && g_ev_end) cudaEventRecord(g_ev_start, st);
    }
    ~SweepEvents() {
        if (g_ev_start && g_ev_end) cudaEventRecord(g_ev_end, st);
    }
};

mp_status fail(mp_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

mp_status cuda_fail(cudaError_t e, const char *what) {
    return fail(MP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t ALIGN = 256;
size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

constexpr int SUM_PARTS = 512;

// Workspace layout of one call.
struct Layout {
    size_t keys = 0, keys128 = 0, hi = 0, lo = 0, x64 = 0, part = 0, mean = 0;
    size_t mu = 0, S = 0, flat = 0, df = 0, dg = 0, inv = 0, muf = 0, mul = 0;
    size_t total = 0;
};

struct Problem {
    int dist;  // mp_dist
    int dtype;
    long long n, N;
    int m;
    long long excl;
    double p;
    mp_options opt;
    long long k_first, k_end;
};

Layout layout(const Problem &pb) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up(bytes);
        return o;
    };
    const size_t n = pb.n, N = pb.N;
    const bool f64 = pb.opt.precision == MP_PREC_FP64;
    if (f64) L.keys128 = take(N * sizeof(mpk::Key128));
    else L.keys = take(N * sizeof(unsigned long long));
    if (!f64) {
        L.hi = take(n * sizeof(float));
        if (pb.dtype == MP_F64) L.lo = take(n * sizeof(float));
    }
    L.x64 = take(n * sizeof(double));
    L.part = take(SUM_PARTS * sizeof(double));
    L.mean = take(sizeof(double));
    if (pb.dist == MP_DIST_ZNORM) {
        L.mu = take(N * sizeof(double));
        L.S = take(N * sizeof(double));
        L.flat = take(N);
        if (!f64) {
            L.df = take(N * sizeof(float));
            L.dg = take(N * sizeof(float));
            L.inv = take(N * sizeof(float));
            L.muf = take(N * sizeof(float));
            L.mul = take(N * sizeof(float));
        }
    }
    L.total = off;
    return L;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

mp_status check_problem(Problem &pb, const void *T, const double *P, const int64_t *I,
                        const mp_options *opt) {
    if (opt) {
        if (opt->struct_size != sizeof(mp_options))
            return fail(MP_ERR_INVALID_ARG, "mp_options.struct_size %u != %zu (use mp_options_default)",
                        opt->struct_size, sizeof(mp_options));
        pb.opt = *opt;
    } else {
        mp_options_default(&pb.opt);
    }
    if (pb.dtype != MP_F32 && pb.dtype != MP_F64) return fail(MP_ERR_INVALID_ARG, "dtype %d", pb.dtype);
    if (pb.n < 1) return fail(MP_ERR_INVALID_ARG, "n = %lld < 1", pb.n);
    if (pb.m < 1 || pb.m > pb.n) return fail(MP_ERR_INVALID_ARG, "m = %d outside [1, n = %lld]", pb.m, pb.n);
    if (pb.dist == MP_DIST_ZNORM && pb.m < 2) return fail(MP_ERR_INVALID_ARG, "z-normalised distance needs m >= 2");
    if (pb.excl < 0) return fail(MP_ERR_INVALID_ARG, "excl = %lld < 0", pb.excl);
    if (pb.dist == MP_DIST_PNORM && !(pb.p >= 1.0 && std::isfinite(pb.p)))
        return fail(MP_ERR_INVALID_ARG, "p = %g, need a finite p >= 1", pb.p);
    if (pb.opt.precision != MP_PREC_FP32 && pb.opt.precision != MP_PREC_FP64)
        return fail(MP_ERR_INVALID_ARG, "precision %d", pb.opt.precision);
    if (pb.opt.reanchor < 0) return fail(MP_ERR_INVALID_ARG, "reanchor %d < 0", pb.opt.reanchor);
    if (pb.opt.polish != 0 && pb.opt.polish != 1) return fail(MP_ERR_INVALID_ARG, "polish %d", pb.opt.polish);
    if (pb.opt.variant < MP_VARIANT_AUTO || pb.opt.variant > MP_VARIANT_FAST_FILTER_BOUND)
        return fail(MP_ERR_INVALID_ARG, "variant %d", pb.opt.variant);
    if (pb.opt.tile_rows < 0 || pb.opt.tile_rows % 1024 != 0 || pb.opt.tile_rows > (1 << 30))
        return fail(MP_ERR_INVALID_ARG, "tile_rows %d: 0 or a positive multiple of 1024", pb.opt.tile_rows);
    if (pb.opt.k_begin < 0) return fail(MP_ERR_INVALID_ARG, "k_begin %lld < 0", (long long)pb.opt.k_begin);
    if (!T || !P || !I) return fail(MP_ERR_INVALID_ARG, "NULL T, P or I");
    if (!aligned(T, pb.dtype == MP_F64 ? 8 : 4) || !aligned(P, 8) || !aligned(I, 8))
        return fail(MP_ERR_INVALID_ARG, "misaligned T, P or I");
    pb.N = pb.n - pb.m + 1;
    if (pb.N >= (1ll << 31) - 1) return fail(MP_ERR_UNSUPPORTED, "N = %lld >= 2^31 - 1", pb.N);
    pb.k_first = std::max<long long>(pb.excl + 1, pb.opt.k_begin);
    pb.k_end = pb.opt.k_end > 0 ? std::min<long long>(pb.N, pb.opt.k_end) : pb.N;
    return MP_OK;
}

// MP_FORCE_GENERIC=1 in the environment selects the generic FP32 kernel even
// where the fast path applies (for comparisons and tests).
bool getenv_generic() {
    const char *v = std::getenv("MP_FORCE_GENERIC");
    return v && v[0] == '1';
}

// Re-anchor interval B for the FP32 sweep: the largest divisor of m that is at
// most `target` (default min(64, m / 4): the running score must not drift over
// more than a quarter of a window) and leaves Q = m / B <= qmax ring blocks.
void choose_block(int m, int target, int qmax, int &B, int &Q) {
    if (target <= 0) target = std::max(1, std::min(64, m / 4));
    int best = 0;
    for (int b = std::min(m, target); b >= 1; --b)
        if (m % b == 0 && m / b <= qmax) { best = b; break; }
    if (best == 0)  // every divisor <= target gives too many blocks: smallest valid one
        for (int b = (m + qmax - 1) / qmax; b <= m; ++b)
            if (m % b == 0) { best = b; break; }
    B = best;
    Q = m / best;
}

int grid_for(long long work, int nt) {
    long long g = (work + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > 65535LL * 16) g = 65535LL * 16;
    return static_cast<int>(g);
}

template <typename Tin>
mp_status prep_series(const Problem &pb, const Layout &L, const void *T, char *ws, cudaStream_t st) {
    const Tin *t = static_cast<const Tin *>(T);
    double *x64 = reinterpret_cast<double *>(ws + L.x64);
    mpk::convert_f64_kernel<Tin><<<grid_for(pb.n, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(t, pb.n, pb.n, x64);
    counted();
    if (pb.opt.precision == MP_PREC_FP32) {
        const double *shift = nullptr;
        if (pb.dtype == MP_F64) {
            double *part = reinterpret_cast<double *>(ws + L.part);
            double *mean = reinterpret_cast<double *>(ws + L.mean);
            mpk::sum_partial_kernel<Tin><<<SUM_PARTS, mpk::PREP_NT, 0, st>>>(t, pb.n, part);
            mpk::sum_final_kernel<<<1, mpk::PREP_NT, 0, st>>>(part, SUM_PARTS, pb.n, mean);
            counted(2);
            shift = mean;
        }
        mpk::convert_f32_kernel<Tin><<<grid_for(pb.n, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(
            t, pb.n, pb.n, shift, reinterpret_cast<float *>(ws + L.hi),
            L.lo ? reinterpret_cast<float *>(ws + L.lo) : nullptr);
        counted();
    }
    return MP_OK;
}


// Exponent kind of a Euclidean / p-norm problem.
int kind_of(int dist, double p) {
    if (dist != MP_DIST_PNORM || p == 2.0) return mpk::K_P2;
    return p == 1.0 ? mpk::K_P1 : p == 3.0 ? mpk::K_P3 : mpk::K_PG;
}

// Fast two-stream path (f32x2 arithmetic, tagged minima): Euclidean or
// p-norm with p in {1, 2, 3}, FP32 input, m a multiple of 32 (re-anchor every
// m / 4 rows), default re-anchor interval, shared memory for two CTAs per SM.
bool fast_path_applies(const Problem &pb) {
    const bool lp = pb.dist == MP_DIST_EUCLID || (pb.dist == MP_DIST_PNORM && kind_of(pb.dist, pb.p) != mpk::K_PG);
    return lp && pb.dtype == MP_F32 && pb.m % 32 == 0 && pb.opt.reanchor == 0 &&
           mpk::sweep2_smem_bytes(pb.m, mpk::V2_R) <= mpk::V2_SMEM_MAX;
}

bool fast_path_ok(const Problem &pb) {
    if (pb.opt.variant == MP_VARIANT_GENERIC || pb.opt.variant == MP_VARIANT_TALL) return false;
    // p = 3: only on request (see p3_exact)
    if (kind_of(pb.dist, pb.p) == mpk::K_P3 && pb.opt.variant != MP_VARIANT_FAST) return false;
    return fast_path_applies(pb) && !getenv_generic();
}

// Status of a sweep launcher's result, counting the launch.
mp_status launched(cudaError_t e, const char *what) {
    if (e != cudaSuccess) return cuda_fail(e, what);
    counted();
    return MP_OK;
}

// The Euclidean sweep's block filter pays off once thresholds are tight for most
// of the sweep, i.e. on long series (each row meets many tiles); on short
// series and on the p-norm kernels (periodic data) it fails too often.
constexpr long long FILTER_MIN_N = 200000;

// Rows per tile of the two-stream sweep: the caller's tile_rows, else tall
// tiles of V2_TALL_R rows (eight one-step tiles; the O(m) anchor from the
// definition is paid once per 16,384 rows instead of once per 2,048) where
// they still leave V2_TALL_MIN_TILES tiles, else one-step tiles of V2_R rows.
// Measured on a GB300 (sweep kernel, n = 2^20): +5% for p = 2 at m = 256, +9%
// at m = 384, +2% at m = 128, +10% on i.i.d. data, +4% for p = 1, none for
// p = 3 (kept at one step), +8% at n = 2^21.  On shorter series tall tiles
// lose (-6% at n = 2^19, -13% at 2^18): the resident tiles then span many
// bands whose first blocks meet open thresholds, and each sub-tile pays its
// staging and barriers.  The choice depends on the problem only, never on the
// device, so results do not change between GPUs.
constexpr long long V2_TALL_R = 8 * mpk::V2_R;
constexpr long long V2_TALL_MIN_TILES = 16384;
constexpr long long V2_TALL_TUNE_TILES = 1216;  // the autotuner tries tall tiles from four waves of 2 x 152 CTAs
long long sweep2_rows(const Problem &pb, long long L, long long nb) {
    if (pb.opt.tile_rows > 0) return pb.opt.tile_rows;
    if (kind_of(pb.dist, pb.p) != mpk::K_P3 && mpk::v2_prefix(L, nb, V2_TALL_R) >= V2_TALL_MIN_TILES &&
        mpk::sweep2_smem_bytes(pb.m, V2_TALL_R) <= mpk::V2_SMEM_MAX)
        return V2_TALL_R;
    return mpk::V2_R;
}

mp_status run_sweep2(const Problem &pb, const Layout &L, char *ws, cudaStream_t st) {
    mpk::Sweep2Args a{};
    a.t = reinterpret_cast<const float *>(ws + L.hi);
    a.keys = reinterpret_cast<unsigned long long *>(ws + L.keys);
    a.n = pb.n;
    a.N = pb.N;
    a.k_first = pb.k_first;
    a.k_end = pb.k_end;
    a.m = pb.m;
    a.Q = mpk::v2_ring_blocks(kind_of(pb.dist, pb.p));  // B = m / Q: a multiple of 8 since m % 32 == 0
    a.B = pb.m / a.Q;
    a.L = pb.N - pb.k_first;
    a.nb = (pb.k_end - pb.k_first + mpk::V2_KW - 1) / mpk::V2_KW;
    a.R = sweep2_rows(pb, a.L, a.nb);
    a.tiles = mpk::v2_prefix(a.L, a.nb, a.R);
    if (a.tiles > 0x7fffffffLL) return fail(MP_ERR_UNSUPPORTED, "too many tiles (%lld)", a.tiles);
    if (a.tiles <= 0) return MP_OK;
    const size_t smem = mpk::sweep2_smem_bytes(a.m, a.R);
    if (smem > mpk::V2_SMEM_MAX)
        return fail(MP_ERR_UNSUPPORTED, "tile_rows %lld: the two-stream tile needs %zu bytes of shared memory",
                    a.R, smem);
    const int kind = kind_of(pb.dist, pb.p);
    SweepEvents ev(st);
    if (kind != mpk::K_P2) return launched(mpk::sweep2_p13_launch(kind, a, smem, st), "two-stream sweep launch");
    const bool filter = pb.opt.variant == MP_VARIANT_FAST_FILTER ||
                        (pb.opt.variant == MP_VARIANT_AUTO && pb.N >= FILTER_MIN_N);
    return launched(mpk::sweep2_p2_launch(filter, a, smem, st), "two-stream sweep launch");
}

// Tall-tile Euclidean / p-norm sweep (float-float sums, tiles of max(8192, 8m) rows).
mp_status run_tall(const Problem &pb, const Layout &L, char *ws, cudaStream_t st) {
    mpk::SweepZArgs a{};
    a.t = reinterpret_cast<const float *>(ws + L.hi);
    a.keys = reinterpret_cast<unsigned long long *>(ws + L.keys);
    a.n = pb.n;
    a.N = pb.N;
    a.k_first = pb.k_first;
    a.k_end = pb.k_end;
    a.m = pb.m;
    a.L = pb.N - pb.k_first;
    a.nb = (pb.k_end - pb.k_first + mpk::Z_KW - 1) / mpk::Z_KW;
    a.S = pb.opt.tile_rows > 0 ? pb.opt.tile_rows : mpk::z_rows_per_tile(pb.m, false);
    a.tiles = mpk::z_prefix(a.L, a.nb, a.S);
    if (a.tiles > 0x7fffffffLL) return fail(MP_ERR_UNSUPPORTED, "too many tiles (%lld)", a.tiles);
    if (a.tiles <= 0) return MP_OK;
    const int kind = kind_of(pb.dist, pb.p);
    SweepEvents ev(st);
    return launched(mpk::sweepz_launch(kind, kind == mpk::K_P2 && pb.N >= FILTER_MIN_N ? 1 : 0, a, mpk::sweepz_smem_bytes(), st),
                    "tall sweep launch");
}

// The generic kernel's shared memory for this problem (0 if it cannot hold m).
size_t generic_smem(const Problem &pb) {
    int B = 0, Q = 0;
    choose_block(pb.m, pb.opt.reanchor, mpk::SW_QMAX, B, Q);
    const size_t smem = mpk::sweep_smem_bytes(2048, pb.m, Q, pb.dtype == MP_F64);
    return smem > 227 * 1024 ? 0 : smem;
}

bool tall_applies(const Problem &pb) {
    return pb.dist != MP_DIST_ZNORM && kind_of(pb.dist, pb.p) != mpk::K_PG && pb.opt.precision == MP_PREC_FP32;
}

// p = 3 with float32 input goes to the tall kernel, whose p = 3 sums are
// error-free (each window sum is the float-float sum of its FP32 terms).  The
// re-anchored FP32 kernels carry the FP32 rounding of the largest sums met
// since the last anchor: |x|^3 spans many orders of magnitude, and after a
// high-amplitude stretch leaves the windows a small distance can be off by
// far more than the FP32 tolerance (measured on the sine-and-motif series,
// n = 2^18, m = 128: 306 rows off by up to 14% after the polish through the
// two-stream kernel, whose block sums are re-anchored every m / 4 rows).
bool p3_exact(const Problem &pb) {
    return kind_of(pb.dist, pb.p) == mpk::K_P3 && tall_applies(pb) && pb.dtype == MP_F32;
}

bool use_tall(const Problem &pb) {
    if (pb.opt.variant == MP_VARIANT_TALL) return true;
    if (pb.opt.variant != MP_VARIANT_AUTO || !tall_applies(pb) || getenv_generic()) return false;
    if (p3_exact(pb)) return true;
    // The tall kernel carries a whole tile without re-anchoring: the rounding of
    // each step's increment accumulates over up to S/2 rows.  An increment is
    // about 1/m of a window sum, so from m = 512 on that stays well inside the
    // FP32 tolerance; for shorter windows (where the tall kernel would be about
    // twice as fast: m = 40 .. 500, p = 1 and 2, measured) the generic kernel's
    // exact re-anchoring every B <= 64 rows keeps p = 3 and near matches exact
    // enough (the tall kernel failed the tolerance at m = 5 and 24 for p = 3).
    return generic_smem(pb) == 0 || (pb.m >= 512 && pb.dtype == MP_F32);
}

mp_status run_sweep_f32(const Problem &pb, const Layout &L, char *ws, cudaStream_t st) {
    if (fast_path_ok(pb)) return run_sweep2(pb, L, ws, st);
    if (use_tall(pb)) return run_tall(pb, L, ws, st);
    mpk::SweepArgs a{};
    a.hi = reinterpret_cast<const float *>(ws + L.hi);
    a.lo = L.lo ? reinterpret_cast<const float *>(ws + L.lo) : nullptr;
    a.keys = reinterpret_cast<unsigned long long *>(ws + L.keys);
    a.n = pb.n;
    a.N = pb.N;
    a.k_first = pb.k_first;
    a.k_end = pb.k_end;
    a.m = pb.m;
    choose_block(pb.m, pb.opt.reanchor, mpk::SW_QMAX, a.B, a.Q);
    a.R = 2048;
    a.q = mpk::SW_KW / a.R;
    a.RL = mpk::sweep_rows_leaving(a.R, a.m);
    a.L = pb.N - pb.k_first;
    a.C = (a.L + a.R - 1) / a.R;
    const long long nb = (pb.k_end - pb.k_first + mpk::SW_KW - 1) / mpk::SW_KW;
    a.nb = nb;
    a.tiles = nb * a.C - static_cast<long long>(a.q) * nb * (nb - 1) / 2;
    a.p = static_cast<float>(pb.p);
    if (a.tiles > 0x7fffffffLL) return fail(MP_ERR_UNSUPPORTED, "too many tiles (%lld)", a.tiles);
    const bool split = a.lo != nullptr;
    const size_t smem = mpk::sweep_smem_bytes(a.R, a.m, a.Q, split);
    if (smem > 227 * 1024) return fail(MP_ERR_UNSUPPORTED, "m = %d needs %zu bytes of shared memory", pb.m, smem);
    SweepEvents ev(st);
    return launched(mpk::generic_launch(kind_of(pb.dist, pb.p), split, a, smem, st), "generic sweep launch");
}

// The autotuner's cached choice for this problem class, written into opt's
// variant, reanchor and tile_rows; false if there is none (autotuning section).
bool tune_lookup(const Problem &pb, mp_options &opt);

// Every check of a one-series call that does not involve the workspace:
// check_problem, then whether the chosen kernel variant applies.  A
// MP_VARIANT_CACHED request is resolved here (to the cached choice, else AUTO).
mp_status check_call(Problem &pb, const void *T, const double *P, const int64_t *I, const mp_options *opt) {
    mp_status s = check_problem(pb, T, P, I, opt);
    if (s != MP_OK) return s;
    if (pb.opt.variant == MP_VARIANT_CACHED) {
        mp_options c = pb.opt;
        if (tune_lookup(pb, c)) {
            pb.opt.variant = c.variant;
            pb.opt.reanchor = c.reanchor;
            pb.opt.tile_rows = c.tile_rows;
        } else {
            pb.opt.variant = MP_VARIANT_AUTO;
        }
    }
    const int v = pb.opt.variant;
    // the z-normalised distance has one FP32 kernel; FAST / FAST_FILTER choose it
    // without / with its block filter
    const bool z32 = pb.dist == MP_DIST_ZNORM && pb.opt.precision == MP_PREC_FP32;
    if ((v == MP_VARIANT_FAST || v == MP_VARIANT_FAST_FILTER) && !z32 &&
        (pb.opt.precision != MP_PREC_FP32 || pb.dist == MP_DIST_ZNORM || !fast_path_applies(pb)))
        return fail(MP_ERR_UNSUPPORTED, "the two-stream kernel does not apply to this problem");
    if (v == MP_VARIANT_FAST_FILTER && !z32 && kind_of(pb.dist, pb.p) != mpk::K_P2)
        return fail(MP_ERR_UNSUPPORTED, "the block filter exists for p = 2 and for the z-normalised kernel");
    if (v == MP_VARIANT_GENERIC && (pb.opt.precision != MP_PREC_FP32 || pb.dist == MP_DIST_ZNORM))
        return fail(MP_ERR_UNSUPPORTED, "the generic kernel is the FP32 Euclidean / p-norm sweep");
    if (v == MP_VARIANT_ZRAW && pb.dist != MP_DIST_ZNORM)
        return fail(MP_ERR_UNSUPPORTED, "the raw-sum variant is Algorithm 2's, for the z-normalised distance");
    if (v == MP_VARIANT_ZF && pb.dist != MP_DIST_ZNORM)
        return fail(MP_ERR_UNSUPPORTED, "the F comparison is Sec. 4.3's, for the z-normalised distance");
    if (v == MP_VARIANT_TALL && !tall_applies(pb))
        return fail(MP_ERR_UNSUPPORTED, "the tall-tile kernel is the FP32 sweep for p in {1, 2, 3}");
    if (v == MP_VARIANT_FAST_FILTER_BOUND && !z32)
        return fail(MP_ERR_UNSUPPORTED, "the bound filter is the FP32 z-normalised kernel's");
    if (pb.opt.tile_rows != 0) {
        const bool zfast = z32 && v != MP_VARIANT_ZRAW && v != MP_VARIANT_ZF && !getenv_generic();
        const bool lp32 = !z32 && pb.dist != MP_DIST_ZNORM && pb.opt.precision == MP_PREC_FP32;
        const bool two = lp32 && fast_path_ok(pb);
        const bool tall = lp32 && !two && use_tall(pb);
        if (two && pb.opt.tile_rows % mpk::V2_R != 0)
            return fail(MP_ERR_UNSUPPORTED, "tile_rows %d: the two-stream kernel's tiles are multiples of %d rows",
                        pb.opt.tile_rows, mpk::V2_R);
        if (!zfast && !tall && !two)
            return fail(MP_ERR_UNSUPPORTED, "tile_rows applies to the two-stream and tall-tile kernels only");
    }
    return MP_OK;
}

mp_status run(Problem &pb, const void *T, double *P, int64_t *I, void *ws, size_t ws_bytes,
              const mp_options *opt, void *stream) {
    mp_status s = check_call(pb, T, P, I, opt);
    if (s != MP_OK) return s;
    const Layout L = layout(pb);
    if (!ws) return fail(MP_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", L.total);
    if (!aligned(ws, ALIGN)) return fail(MP_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (ws_bytes < L.total) return fail(MP_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(ws);
    cudaGetLastError();  // clear a stale launch error of an unrelated caller

    const bool f64 = pb.opt.precision == MP_PREC_FP64;
    Range call_range(pb.dist == MP_DIST_EUCLID ? "mp_aamp" : pb.dist == MP_DIST_PNORM ? "mp_pnorm" : "mp_acamp");
    {
        Range r("a1 convert");
        s = pb.dtype == MP_F64 ? prep_series<double>(pb, L, T, w, st) : prep_series<float>(pb, L, T, w, st);
    }
    if (s != MP_OK) return s;
    if (f64) {
        mpk::fill_u64_kernel<<<grid_for(2 * pb.N, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(
            reinterpret_cast<unsigned long long *>(w + L.keys128), 2 * pb.N, mpk::KEY_NONE);
        counted();
    } else {
        mpk::fill_u64_kernel<<<grid_for(pb.N, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(
            reinterpret_cast<unsigned long long *>(w + L.keys), pb.N, mpk::KEY_NONE);
        counted();
    }
    const double *x64 = reinterpret_cast<const double *>(w + L.x64);
    if (pb.dist == MP_DIST_ZNORM) {
        Range r("a2 window statistics");
        mpk::window_stats_kernel<<<grid_for(pb.N, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(
            x64, pb.N, pb.m, reinterpret_cast<double *>(w + L.mu), reinterpret_cast<double *>(w + L.S),
            reinterpret_cast<unsigned char *>(w + L.flat));
        counted();
        if (!f64) {
            mpk::znorm_operands_kernel<<<grid_for(pb.N, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(
                x64, pb.N, pb.m, reinterpret_cast<const double *>(w + L.mu),
                reinterpret_cast<const double *>(w + L.S), reinterpret_cast<const unsigned char *>(w + L.flat),
                reinterpret_cast<float *>(w + L.df), reinterpret_cast<float *>(w + L.dg),
                reinterpret_cast<float *>(w + L.inv), reinterpret_cast<float *>(w + L.muf),
                reinterpret_cast<float *>(w + L.mul),
                pb.dtype == MP_F64 ? reinterpret_cast<const double *>(w + L.mean) : nullptr, pb.N);
            counted();
        }
    }
    if (pb.k_first < pb.k_end) {
        Range r("a3-a5 sweep");
        if (pb.dist == MP_DIST_ZNORM || f64) {
            const mpk::TileGrid g = mpk::make_grid(pb.N, pb.k_first, pb.k_end, mpk::SM_KW, mpk::SM_KW);
            if (g.tiles > 0x7fffffffLL) return fail(MP_ERR_UNSUPPORTED, "too many tiles (%lld)", g.tiles);
            int *err = mpk::device_error_ptr();
            cudaError_t e;
            SweepEvents ev(st);
            if (g.tiles > 0) counted();
            const bool zraw = pb.opt.variant == MP_VARIANT_ZRAW;
            const bool zf = pb.opt.variant == MP_VARIANT_ZF;
            if (pb.dist == MP_DIST_ZNORM && f64 && zf) {
                mpk::VarF64ZF v{x64, reinterpret_cast<const double *>(w + L.mu),
                                reinterpret_cast<const double *>(w + L.S),
                                reinterpret_cast<const unsigned char *>(w + L.flat), pb.m,
                                reinterpret_cast<mpk::Key128 *>(w + L.keys128), err};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 256, st);
            } else if (pb.dist == MP_DIST_ZNORM && zf) {
                mpk::VarF32ZF v{reinterpret_cast<const float *>(w + L.hi), reinterpret_cast<const float *>(w + L.muf),
                                reinterpret_cast<const float *>(w + L.inv), pb.m,
                                reinterpret_cast<unsigned long long *>(w + L.keys)};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 512, st);
            } else if (pb.dist == MP_DIST_ZNORM && f64 && zraw) {
                mpk::VarF64ZRaw v{x64, reinterpret_cast<const double *>(w + L.mu),
                                  reinterpret_cast<const double *>(w + L.S),
                                  reinterpret_cast<const unsigned char *>(w + L.flat), pb.m,
                                  reinterpret_cast<mpk::Key128 *>(w + L.keys128), err};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 256, st);
            } else if (pb.dist == MP_DIST_ZNORM && f64) {
                mpk::VarF64Z v{x64, reinterpret_cast<const double *>(w + L.mu),
                               reinterpret_cast<const double *>(w + L.S),
                               reinterpret_cast<const unsigned char *>(w + L.flat), pb.m,
                               reinterpret_cast<mpk::Key128 *>(w + L.keys128), err};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 256, st);
            } else if (pb.dist == MP_DIST_ZNORM && zraw) {
                mpk::VarF32ZRaw v{reinterpret_cast<const float *>(w + L.hi), reinterpret_cast<const float *>(w + L.muf),
                                  reinterpret_cast<const float *>(w + L.inv), pb.m,
                                  reinterpret_cast<unsigned long long *>(w + L.keys)};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 512, st);
            } else if (pb.dist == MP_DIST_ZNORM && !getenv_generic()) {
                mpk::SweepZArgs za{};
                za.t = reinterpret_cast<const float *>(w + L.hi);
                za.tlo = pb.dtype == MP_F64 ? reinterpret_cast<const float *>(w + L.lo) : nullptr;
                za.muh = reinterpret_cast<const float *>(w + L.muf);
                za.mul = reinterpret_cast<const float *>(w + L.mul);
                za.df = reinterpret_cast<const float *>(w + L.df);
                za.dg = reinterpret_cast<const float *>(w + L.dg);
                za.inv = reinterpret_cast<const float *>(w + L.inv);
                za.keys = reinterpret_cast<unsigned long long *>(w + L.keys);
                za.n = pb.n;
                za.N = pb.N;
                za.k_first = pb.k_first;
                za.k_end = pb.k_end;
                za.m = pb.m;
                za.L = pb.N - pb.k_first;
                za.nb = (pb.k_end - pb.k_first + mpk::Z_KW - 1) / mpk::Z_KW;
                za.S = pb.opt.tile_rows > 0 ? pb.opt.tile_rows : mpk::z_rows_per_tile(pb.m, true);
                za.tiles = mpk::z_prefix(za.L, za.nb, za.S);
                if (za.tiles > 0x7fffffffLL) return fail(MP_ERR_UNSUPPORTED, "too many tiles (%lld)", za.tiles);
                const int filter = pb.opt.variant == MP_VARIANT_FAST_FILTER_BOUND ? 2
                                   : (pb.opt.variant == MP_VARIANT_FAST_FILTER ||
                                      (pb.opt.variant == MP_VARIANT_AUTO && pb.N >= FILTER_MIN_N)) ? 1 : 0;
                e = za.tiles > 0 ? mpk::sweepz_launch(mpk::K_Z, filter, za, mpk::sweepz_smem_bytes(), st)
                                 : cudaSuccess;
            } else if (pb.dist == MP_DIST_ZNORM) {
                mpk::VarF32Z v{reinterpret_cast<const float *>(w + L.hi), reinterpret_cast<const float *>(w + L.muf),
                               reinterpret_cast<const float *>(w + L.df), reinterpret_cast<const float *>(w + L.dg),
                               reinterpret_cast<const float *>(w + L.inv), pb.m,
                               reinterpret_cast<unsigned long long *>(w + L.keys)};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 512, st);
            } else {
                mpk::VarF64Lp v{x64, pb.m, pb.dist == MP_DIST_PNORM ? pb.p : 2.0,
                                reinterpret_cast<mpk::Key128 *>(w + L.keys128), err};
                e = mpk::launch_simple(g, v, pb.opt.reanchor > 0 ? pb.opt.reanchor : 256, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
        } else {
            s = run_sweep_f32(pb, L, w, st);
            if (s != MP_OK) return s;
        }
    }
    Range fin_range("a6 finalize");
    mpk::FinalizeArgs fa{};
    fa.keys = f64 ? nullptr : reinterpret_cast<const unsigned long long *>(w + L.keys);
    fa.keys128 = f64 ? reinterpret_cast<const mpk::Key128 *>(w + L.keys128) : nullptr;
    fa.x = x64;
    fa.mu = L.mu ? reinterpret_cast<const double *>(w + L.mu) : nullptr;
    fa.S = L.S ? reinterpret_cast<const double *>(w + L.S) : nullptr;
    fa.N = pb.N;
    fa.m = pb.m;
    fa.dist = pb.dist == MP_DIST_EUCLID ? mpk::FIN_EUCLID : pb.dist == MP_DIST_PNORM ? mpk::FIN_PNORM : mpk::FIN_ZNORM;
    fa.p = pb.dist == MP_DIST_PNORM ? pb.p : 2.0;
    fa.polish = pb.opt.polish;
    fa.fkey = pb.dist == MP_DIST_ZNORM && pb.opt.variant == MP_VARIANT_ZF;
    fa.P = P;
    fa.I = reinterpret_cast<long long *>(I);
    mpk::finalize_kernel<<<grid_for(pb.N, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(fa);
    counted();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return MP_OK;
}

}  // namespace

// ---- scratch of mp_aamp_noalloc ------------------------------------------------------
// Static device memory: loaded with the module on every device that uses the
// library, never allocated or freed by a call.  Host code must not take its
// address directly (the host symbol is only a stand-in); every call looks the
// device address up on the current device with cudaGetSymbolAddress (a host-side
// query), so no address outlives a device reset or a new primary context.
static __device__ __align__(256) unsigned char mp_noalloc_scratch[MP_NOALLOC_SCRATCH_BYTES];

namespace {
mp_status noalloc_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, mp_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    *out = p;
    return MP_OK;
}
}  // namespace

extern "C" {

void mp_options_default(mp_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->struct_size = sizeof(mp_options);
    opt->precision = MP_PREC_FP32;
    opt->reanchor = 0;
    opt->polish = 1;
    opt->k_begin = 0;
    opt->k_end = 0;
}

size_t mp_workspace_size(int dist, int dtype, int64_t n, int32_t m, const mp_options *opt) {
    Problem pb{};
    pb.dist = dist;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = 0;
    pb.p = 2.0;
    if (dist < MP_DIST_EUCLID || dist > MP_DIST_ZNORM) return 0;
    static const double dummy = 0;
    if (check_problem(pb, &dummy, reinterpret_cast<const double *>(&dummy),
                      reinterpret_cast<const int64_t *>(&dummy), opt) != MP_OK)
        return 0;
    return layout(pb).total;
}

mp_status mp_aamp(const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double *P, int64_t *I,
                  void *ws, size_t ws_bytes, const mp_options *opt, void *stream) {
    g_err[0] = 0;
    Problem pb{};
    pb.dist = MP_DIST_EUCLID;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = excl;
    pb.p = 2.0;
    return run(pb, T, P, I, ws, ws_bytes, opt, stream);
}

mp_status mp_pnorm(const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double p, double *P,
                   int64_t *I, void *ws, size_t ws_bytes, const mp_options *opt, void *stream) {
    g_err[0] = 0;
    Problem pb{};
    pb.dist = MP_DIST_PNORM;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = excl;
    pb.p = p;
    return run(pb, T, P, I, ws, ws_bytes, opt, stream);
}

mp_status mp_acamp(const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double *P, int64_t *I,
                   void *ws, size_t ws_bytes, const mp_options *opt, void *stream) {
    g_err[0] = 0;
    Problem pb{};
    pb.dist = MP_DIST_ZNORM;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = excl;
    pb.p = 2.0;
    return run(pb, T, P, I, ws, ws_bytes, opt, stream);
}

mp_status mp_aamp_noalloc(const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double *P, int64_t *I,
                          const mp_options *opt, void *stream) {
    g_err[0] = 0;
    Problem pb{};
    pb.dist = MP_DIST_EUCLID;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = excl;
    pb.p = 2.0;
    // the checks and errors of mp_aamp first, before any CUDA call
    mp_status st = check_call(pb, T, P, I, opt);
    if (st != MP_OK) return st;
    const size_t need = layout(pb).total;
    if (need > MP_NOALLOC_SCRATCH_BYTES)
        return fail(MP_ERR_UNSUPPORTED, "n = %lld needs %zu bytes of scratch; mp_aamp_noalloc has %u",
                    static_cast<long long>(n), need, MP_NOALLOC_SCRATCH_BYTES);
    void *ws = nullptr;
    st = noalloc_scratch(&ws);
    if (st != MP_OK) return st;
    Problem pr{};
    pr.dist = MP_DIST_EUCLID;
    pr.dtype = dtype;
    pr.n = n;
    pr.m = m;
    pr.excl = excl;
    pr.p = 2.0;
    return run(pr, T, P, I, ws, MP_NOALLOC_SCRATCH_BYTES, opt, stream);
}

mp_status mp_sync_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    // the error word of every translation unit that holds kernels
    int *words[] = {mpk::device_error_ptr(), mpk::sweep2_p2_error_word(), mpk::sweep2_tall_error_word(),
                    mpk::sweep2_p13_error_word(),
                    mpk::sweepz_error_word(), mpk::batch2_error_word(), mpk::generic_error_word()};
    int bits = 0;
    for (int *w : words) {
        if (!w) return fail(MP_ERR_CUDA, "device error word not found");
        int v = 0;
        e = cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
        if (v) {
            bits |= v;
            e = cudaMemset(w, 0, sizeof(int));
            if (e != cudaSuccess) return cuda_fail(e, "clearing the device error word");
        }
    }
    if (bits) return fail(MP_ERR_INTERNAL, "device-side check failed (bits 0x%x)", bits);
    return MP_OK;
}

const char *mp_last_error(void) { return g_err; }

const char *mp_status_string(mp_status s) {
    switch (s) {
        case MP_OK: return "MP_OK";
        case MP_ERR_INVALID_ARG: return "MP_ERR_INVALID_ARG";
        case MP_ERR_UNSUPPORTED: return "MP_ERR_UNSUPPORTED";
        case MP_ERR_WORKSPACE: return "MP_ERR_WORKSPACE";
        case MP_ERR_CUDA: return "MP_ERR_CUDA";
        case MP_ERR_INTERNAL: return "MP_ERR_INTERNAL";
    }
    return "MP_ERR_UNKNOWN";
}

const char *mp_version(void) { return "0.1.0"; }

uint64_t mp_launch_count(void) { return g_launches.load(); }

mp_status mp_set_sweep_events(void *ev_start, void *ev_end) {
    g_ev_start = static_cast<cudaEvent_t>(ev_start);
    g_ev_end = static_cast<cudaEvent_t>(ev_end);
    return MP_OK;
}

}  // extern "C"

// ---- a7: batches -----------------------------------------------------------------------
struct mp_batch_plan {
    enum { Q_FAST2 = 0, Q_Z = 1, Q_GEN2 = 2, Q_GENP = 3, Q_FASTP = 4, NQ = 5 };
    int device = -1;
    int S = 0;
    double p = 2.0;
    int polish = 1;
    int genp_kind = mpk::K_P2;  // exponent kind of the p-norm queues
    bool filter = false;        // the p = 2 two-stream queue runs the block filter
    long long windows = 0, zwindows = 0, samples = 0;
    std::vector<mpk::BatchSeries> series;
    std::vector<long long> w_start;
    std::vector<mpk::BatchTile> tiles[NQ];
    size_t smem[NQ] = {};
    int grid[NQ] = {};
    // device copies (owned)
    mpk::BatchSeries *d_series = nullptr;
    long long *d_wstart = nullptr;
    mpk::BatchTile *d_tiles[NQ] = {};
    // workspace layout
    size_t o_keys = 0, o_tickets = 0, o_mu = 0, o_S = 0, o_flat = 0, o_df = 0, o_dg = 0, o_inv = 0, o_muh = 0,
           o_mul = 0, ws_bytes = 0;
    // graph cache
    cudaStream_t cap = nullptr;
    // one capture stream per queue, forked from `cap` and joined before the
    // finalize, so that the queues' persistent kernels overlap in the graph
    cudaStream_t qst[NQ] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[NQ] = {};
    cudaGraphExec_t exec = nullptr;
    const void *g_T = nullptr;
    const void *g_P = nullptr;
    const void *g_I = nullptr;
    const void *g_ws = nullptr;
    int nodes = 0;
};

namespace {

void batch_free(mp_batch_plan *pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    for (int q = 0; q < mp_batch_plan::NQ; ++q) {
        if (pl->qst[q]) cudaStreamDestroy(pl->qst[q]);
        if (pl->ev_join[q]) cudaEventDestroy(pl->ev_join[q]);
    }
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->d_series) cudaFree(pl->d_series);
    if (pl->d_wstart) cudaFree(pl->d_wstart);
    for (auto *t : pl->d_tiles)
        if (t) cudaFree(t);
    delete pl;
}

// Tiles of one series for a sweep whose bands hold KW diagonals and whose
// tiles hold R rows (band b: L - b KW rows), with cost = rows x diagonals and
// the tile's rank within its series (band-major) in the spare field.
void batch_tiles(std::vector<std::pair<long long, mpk::BatchTile>> &out, int s, long long L, int KW, int R) {
    if (L <= 0) return;
    const long long nb = (L + KW - 1) / KW;
    int rank = 0;
    for (long long b = 0; b < nb; ++b) {
        const long long Lb = L - b * KW;
        const long long nd = std::min<long long>(KW, Lb);
        const long long nt = (Lb + R - 1) / R;
        for (long long rt = 0; rt < nt; ++rt) {
            const long long rows = std::min<long long>(R, Lb - rt * R);
            out.push_back({rows * nd, mpk::BatchTile{s, static_cast<int>(b), static_cast<int>(rt), rank++}});
        }
    }
}

mp_status batch_validate(const mp_batch_desc *d, const mp_options *opt, mp_options &o) {
    if (!d) return fail(MP_ERR_INVALID_ARG, "desc is NULL");
    if (d->struct_size != sizeof(mp_batch_desc))
        return fail(MP_ERR_INVALID_ARG, "mp_batch_desc.struct_size %u != %zu", d->struct_size, sizeof(mp_batch_desc));
    if (d->num_series < 1) return fail(MP_ERR_INVALID_ARG, "num_series = %d < 1", d->num_series);
    if (!d->t_offsets || !d->m || !d->dist || !d->excl) return fail(MP_ERR_INVALID_ARG, "NULL array in desc");
    if (d->dtype != MP_F32) {
        if (d->dtype == MP_F64) return fail(MP_ERR_UNSUPPORTED, "batches take float32 series only");
        return fail(MP_ERR_INVALID_ARG, "dtype %d", d->dtype);
    }
    if (opt) {
        if (opt->struct_size != sizeof(mp_options))
            return fail(MP_ERR_INVALID_ARG, "mp_options.struct_size %u != %zu", opt->struct_size, sizeof(mp_options));
        o = *opt;
    } else {
        mp_options_default(&o);
    }
    if (o.precision != MP_PREC_FP32) return fail(MP_ERR_UNSUPPORTED, "batches run the FP32 sweep only");
    if (o.reanchor != 0) return fail(MP_ERR_UNSUPPORTED, "batches use the default re-anchor interval");
    if (o.k_begin != 0 || o.k_end != 0) return fail(MP_ERR_UNSUPPORTED, "batches sweep whole diagonal ranges");
    if (o.polish != 0 && o.polish != 1) return fail(MP_ERR_INVALID_ARG, "polish %d", o.polish);
    if (o.variant != MP_VARIANT_AUTO && o.variant != MP_VARIANT_FAST && o.variant != MP_VARIANT_FAST_FILTER &&
        o.variant != MP_VARIANT_CACHED)
        return fail(MP_ERR_UNSUPPORTED, "batches take variant AUTO, FAST, FAST_FILTER or CACHED");
    if (o.tile_rows < 0 || o.tile_rows % 1024 != 0 || o.tile_rows > (1 << 30))
        return fail(MP_ERR_INVALID_ARG, "tile_rows %d: 0 or a positive multiple of 1024", o.tile_rows);
    if (d->t_offsets[0] < 0) return fail(MP_ERR_INVALID_ARG, "t_offsets[0] < 0");
    bool any_p = false;
    for (int s = 0; s < d->num_series; ++s) {
        const long long n = d->t_offsets[s + 1] - d->t_offsets[s];
        const int m = d->m[s];
        if (n < 1) return fail(MP_ERR_INVALID_ARG, "series %d: n = %lld < 1", s, n);
        if (m < 1 || m > n) return fail(MP_ERR_INVALID_ARG, "series %d: m = %d outside [1, %lld]", s, m, n);
        if (d->dist[s] > MP_DIST_ZNORM) return fail(MP_ERR_INVALID_ARG, "series %d: dist %d", s, d->dist[s]);
        if (d->dist[s] == MP_DIST_ZNORM && m < 2)
            return fail(MP_ERR_INVALID_ARG, "series %d: z-normalised distance needs m >= 2", s);
        if (d->excl[s] < 0) return fail(MP_ERR_INVALID_ARG, "series %d: excl < 0", s);
        if (n - m + 1 >= (1ll << 31) - 1) return fail(MP_ERR_UNSUPPORTED, "series %d: N >= 2^31 - 1", s);
        any_p |= d->dist[s] == MP_DIST_PNORM;
    }
    if (any_p && !(d->p >= 1.0 && std::isfinite(d->p)))
        return fail(MP_ERR_INVALID_ARG, "p = %g, need a finite p >= 1", d->p);
    return MP_OK;
}

// Persistent grid of queue qi: as many CTAs as fit on the device at once (per_sm
// from the occupancy query), at most one per tile.
void batch_grid(mp_batch_plan *pl, int q, int per_sm, int sms) {
    if (per_sm < 1) per_sm = 1;
    const long long want = static_cast<long long>(per_sm) * sms;
    pl->grid[q] = static_cast<int>(std::min<long long>(want, static_cast<long long>(pl->tiles[q].size())));
}

// Launch the sweep of queue qi on `grid` CTAs.
cudaError_t batch_queue_launch(const mp_batch_plan *pl, int qi, int grid, const mpk::BatchData &bd,
                               const mpk::BatchQueue &q, cudaStream_t st) {
    switch (qi) {
        case mp_batch_plan::Q_FAST2: return mpk::batch2_launch(mpk::K_P2, pl->filter, grid, pl->smem[qi], bd, q, st);
        case mp_batch_plan::Q_FASTP: return mpk::batch2_launch(pl->genp_kind, false, grid, pl->smem[qi], bd, q, st);
        case mp_batch_plan::Q_Z: return mpk::batchz_launch(grid, pl->smem[qi], bd, q, st);
        default:
            return mpk::batchg_launch(qi == mp_batch_plan::Q_GEN2 ? mpk::K_P2 : pl->genp_kind, grid, pl->smem[qi], bd,
                                      q, mpk::device_error_ptr(), st);
    }
}

// Record the batch on the plan's capture stream and instantiate it.
mp_status batch_build_graph(mp_batch_plan *pl, const void *T, double *P, int64_t *I, void *ws) {
    char *w = static_cast<char *>(ws);
    mpk::BatchData bd{};
    bd.series = pl->d_series;
    bd.w_start = pl->d_wstart;
    bd.S = pl->S;
    bd.windows = pl->windows;
    bd.T = static_cast<const float *>(T);
    bd.keys = reinterpret_cast<unsigned long long *>(w + pl->o_keys);
    if (pl->zwindows > 0) {
        bd.mu = reinterpret_cast<double *>(w + pl->o_mu);
        bd.Sx = reinterpret_cast<double *>(w + pl->o_S);
        bd.flat = reinterpret_cast<unsigned char *>(w + pl->o_flat);
        bd.df = reinterpret_cast<float *>(w + pl->o_df);
        bd.dg = reinterpret_cast<float *>(w + pl->o_dg);
        bd.inv = reinterpret_cast<float *>(w + pl->o_inv);
        bd.muh = reinterpret_cast<float *>(w + pl->o_muh);
        bd.mul = reinterpret_cast<float *>(w + pl->o_mul);
    }
    bd.P = P;
    bd.I = reinterpret_cast<long long *>(I);
    bd.p = pl->p;
    bd.polish = pl->polish;
    unsigned *tickets = reinterpret_cast<unsigned *>(w + pl->o_tickets);

    cudaStream_t st = pl->cap;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    int nodes = 0;
    const int gw = grid_for(pl->windows, mpk::PREP_NT);
    mpk::batch_init_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd.keys, pl->windows, tickets, mp_batch_plan::NQ);
    ++nodes;
    if (pl->zwindows > 0) {
        mpk::batch_zstats_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd);
        mpk::batch_zoperands_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd);
        nodes += 2;
    }
    // the queues' sweeps on forked streams: each starts after the statistics, the
    // finalize after all of them (CTAs of the next queue fill the SMs that the
    // tail of another leaves idle)
    cudaEventRecord(pl->ev_fork, st);
    for (int qi = 0; qi < mp_batch_plan::NQ; ++qi) {
        if (pl->tiles[qi].empty()) continue;
        const mpk::BatchQueue q{pl->d_tiles[qi], static_cast<unsigned>(pl->tiles[qi].size()), tickets + qi};
        cudaStreamWaitEvent(pl->qst[qi], pl->ev_fork, 0);
        batch_queue_launch(pl, qi, pl->grid[qi], bd, q, pl->qst[qi]);
        cudaEventRecord(pl->ev_join[qi], pl->qst[qi]);
        cudaStreamWaitEvent(st, pl->ev_join[qi], 0);
        ++nodes;
    }
    mpk::batch_finalize_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd);
    ++nodes;
    const cudaError_t le = cudaGetLastError();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le != cudaSuccess ? le : e, "recording the batch graph");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    pl->exec = exec;
    pl->nodes = nodes;
    pl->g_T = T;
    pl->g_P = P;
    pl->g_I = I;
    pl->g_ws = ws;
    return MP_OK;
}

}  // namespace

static mp_status batch_plan_build(const mp_batch_desc *desc, const mp_options *opt, unsigned long long seed,
                                  mp_batch_plan **plan, size_t *ws_bytes);

extern "C" {

mp_status mp_batch_plan_create(const mp_batch_desc *desc, const mp_options *opt, mp_batch_plan **plan,
                               size_t *ws_bytes) {
    g_err[0] = 0;
    return batch_plan_build(desc, opt, 0, plan, ws_bytes);
}

}  // extern "C"

namespace {

// splitmix64: a small counter-based generator, the same sequence on every platform
unsigned long long splitmix64(unsigned long long &x) {
    unsigned long long z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

// Build a plan; seed = 0 orders every tile queue by decreasing cost (longest
// first), another seed by a seeded random permutation (anytime runs).
static mp_status batch_plan_build(const mp_batch_desc *desc, const mp_options *opt, unsigned long long seed,
                                  mp_batch_plan **plan, size_t *ws_bytes) {
    if (!plan) return fail(MP_ERR_INVALID_ARG, "plan is NULL");
    *plan = nullptr;
    mp_options o{};
    mp_status s = batch_validate(desc, opt, o);
    if (s != MP_OK) return s;

    auto *pl = new mp_batch_plan();
    pl->S = desc->num_series;
    pl->p = desc->p;
    pl->polish = o.polish;
    pl->filter = o.variant == MP_VARIANT_FAST_FILTER;  // (CACHED: off, as AUTO, for the Euclidean queue)
    if (desc->p == 1.0) pl->genp_kind = mpk::K_P1;
    else if (desc->p == 2.0) pl->genp_kind = mpk::K_P2;
    else if (desc->p == 3.0) pl->genp_kind = mpk::K_P3;
    else pl->genp_kind = mpk::K_PG;
    std::vector<std::pair<long long, mpk::BatchTile>> q[mp_batch_plan::NQ];
    int qmax_m[mp_batch_plan::NQ] = {}, qmax_Q[mp_batch_plan::NQ] = {};
    pl->series.resize(pl->S);
    pl->w_start.resize(pl->S + 1);
    for (int si = 0; si < pl->S; ++si) {
        mpk::BatchSeries &b = pl->series[si];
        b.t_off = desc->t_offsets[si];
        b.n = desc->t_offsets[si + 1] - desc->t_offsets[si];
        b.m = desc->m[si];
        b.N = b.n - b.m + 1;
        b.k_first = desc->excl[si] + 1;
        b.w_off = pl->windows;
        pl->w_start[si] = pl->windows;
        pl->windows += b.N;
        const int dist = desc->dist[si];
        const bool p2 = dist == MP_DIST_EUCLID || (dist == MP_DIST_PNORM && desc->p == 2.0);
        b.dist = dist == MP_DIST_ZNORM ? mpk::FIN_ZNORM : dist == MP_DIST_PNORM ? mpk::FIN_PNORM : mpk::FIN_EUCLID;
        b.z_off = -1;
        choose_block(b.m, 0, mpk::SW_QMAX, b.B, b.Q);
        b.RL = mpk::sweep_rows_leaving(mpk::BATCH_GEN_R, b.m);
        const long long L = b.N - b.k_first;
        int qi;
        if (dist == MP_DIST_ZNORM) {
            b.z_off = pl->zwindows;
            pl->zwindows += b.N;
            qi = mp_batch_plan::Q_Z;
            // rows per tile: the caller's tile_rows, a cached autotuning choice for
            // this series' problem class (MP_VARIANT_CACHED), else the default
            long long zS = o.tile_rows > 0 ? o.tile_rows : mpk::z_rows_per_tile(b.m, true);
            if (o.variant == MP_VARIANT_CACHED) {
                Problem sp{};
                sp.dist = MP_DIST_ZNORM;
                sp.dtype = MP_F32;
                sp.m = b.m;
                sp.N = b.N;
                sp.p = 2.0;
                mp_options c = o;
                if (tune_lookup(sp, c) && c.tile_rows > 0) zS = c.tile_rows;
            }
            b.zS = static_cast<int>(zS);
            batch_tiles(q[qi], si, L, mpk::Z_KW, b.zS);
        } else if (b.m % 32 == 0 && mpk::sweep2_smem_bytes(b.m, mpk::V2_R) <= mpk::V2_SMEM_MAX &&
                   (p2 || pl->genp_kind == mpk::K_P1 || pl->genp_kind == mpk::K_P3)) {
            qi = p2 ? mp_batch_plan::Q_FAST2 : mp_batch_plan::Q_FASTP;
            batch_tiles(q[qi], si, L, mpk::V2_KW, mpk::V2_R);
        } else {
            qi = p2 ? mp_batch_plan::Q_GEN2 : mp_batch_plan::Q_GENP;
            batch_tiles(q[qi], si, L, mpk::SW_KW, mpk::BATCH_GEN_R);
        }
        if (L > 0) {
            qmax_m[qi] = std::max(qmax_m[qi], b.m);
            qmax_Q[qi] = std::max(qmax_Q[qi], b.Q);
        }
    }
    pl->w_start[pl->S] = pl->windows;
    pl->samples = desc->t_offsets[pl->S];
    if (pl->genp_kind == mpk::K_P2) {  // p = 2: one generic queue
        for (auto &t : q[mp_batch_plan::Q_GENP]) q[mp_batch_plan::Q_GEN2].push_back(t);
        q[mp_batch_plan::Q_GENP].clear();
        qmax_m[mp_batch_plan::Q_GEN2] = std::max(qmax_m[mp_batch_plan::Q_GEN2], qmax_m[mp_batch_plan::Q_GENP]);
        qmax_Q[mp_batch_plan::Q_GEN2] = std::max(qmax_Q[mp_batch_plan::Q_GEN2], qmax_Q[mp_batch_plan::Q_GENP]);
    }
    for (int qi = 0; qi < mp_batch_plan::NQ; ++qi) {
        if (q[qi].size() > 0xfffffffeull) {
            batch_free(pl);
            return fail(MP_ERR_UNSUPPORTED, "more than 2^32 - 2 tiles in one queue");
        }
        if (seed == 0) {
            // Round robin over the series (every series' first tile, then every
            // series' second tile, ...), longest first within a round: the tiles
            // of one series run one after another, each starting from the
            // thresholds its predecessors left, instead of all at once with
            // open thresholds; the ticket queue balances the load whatever the order.
            std::stable_sort(q[qi].begin(), q[qi].end(), [](const auto &a, const auto &b) {
                return a.second.rank < b.second.rank || (a.second.rank == b.second.rank && a.first > b.first);
            });
        } else {  // Fisher-Yates with splitmix64
            unsigned long long st = seed ^ (0x632be59bd9b4e019ull * (qi + 1));
            for (size_t t = q[qi].size(); t > 1; --t) {
                const size_t r = static_cast<size_t>(splitmix64(st) % t);
                std::swap(q[qi][t - 1], q[qi][r]);
            }
        }
        pl->tiles[qi].reserve(q[qi].size());
        for (auto &t : q[qi]) pl->tiles[qi].push_back(t.second);
        if (qi == mp_batch_plan::Q_FAST2 || qi == mp_batch_plan::Q_FASTP)
            pl->smem[qi] = mpk::sweep2_smem_bytes(std::max(qmax_m[qi], 32), mpk::V2_R);
        else if (qi == mp_batch_plan::Q_Z) pl->smem[qi] = mpk::sweepz_smem_bytes();
        else pl->smem[qi] = mpk::sweep_smem_bytes(mpk::BATCH_GEN_R, std::max(qmax_m[qi], 1), std::max(qmax_Q[qi], 1), false);
        if (!pl->tiles[qi].empty() && pl->smem[qi] > 227 * 1024) {
            batch_free(pl);
            return fail(MP_ERR_UNSUPPORTED, "m = %d needs %zu bytes of shared memory", qmax_m[qi], pl->smem[qi]);
        }
    }
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += up(bytes); return at; };
    pl->o_keys = take(static_cast<size_t>(pl->windows) * 8);
    pl->o_tickets = take(mp_batch_plan::NQ * sizeof(unsigned));
    if (pl->zwindows > 0) {
        const size_t Z = static_cast<size_t>(pl->zwindows);
        pl->o_mu = take(Z * 8);
        pl->o_S = take(Z * 8);
        pl->o_flat = take(Z);
        pl->o_df = take(Z * 4);
        pl->o_dg = take(Z * 4);
        pl->o_inv = take(Z * 4);
        pl->o_muh = take(Z * 4);
        pl->o_mul = take(Z * 4);
    }
    pl->ws_bytes = off;

    // device side
    cudaError_t e = cudaGetDevice(&pl->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_series, sizeof(mpk::BatchSeries) * pl->S);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_wstart, sizeof(long long) * (pl->S + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_series, pl->series.data(), sizeof(mpk::BatchSeries) * pl->S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(pl->d_wstart, pl->w_start.data(), sizeof(long long) * (pl->S + 1), cudaMemcpyHostToDevice);
    for (int qi = 0; qi < mp_batch_plan::NQ && e == cudaSuccess; ++qi) {
        if (pl->tiles[qi].empty()) continue;
        const size_t bytes = sizeof(mpk::BatchTile) * pl->tiles[qi].size();
        e = cudaMalloc(&pl->d_tiles[qi], bytes);
        if (e == cudaSuccess) e = cudaMemcpy(pl->d_tiles[qi], pl->tiles[qi].data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        int per_sm = 0;
        if (qi == mp_batch_plan::Q_FAST2 || qi == mp_batch_plan::Q_FASTP) {
            const int kind = qi == mp_batch_plan::Q_FAST2 ? mpk::K_P2 : pl->genp_kind;
            e = mpk::batch2_setup(kind, kind == mpk::K_P2 && pl->filter, pl->smem[qi], &per_sm);
        } else if (qi == mp_batch_plan::Q_Z) {
            e = mpk::batchz_setup(pl->smem[qi], &per_sm);
        } else {
            e = mpk::batchg_setup(qi == mp_batch_plan::Q_GEN2 ? mpk::K_P2 : pl->genp_kind, pl->smem[qi], &per_sm);
        }
        if (e == cudaSuccess) batch_grid(pl, qi, per_sm, sms);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
    for (int qi = 0; qi < mp_batch_plan::NQ && e == cudaSuccess; ++qi) {
        if (pl->tiles[qi].empty()) continue;
        e = cudaStreamCreateWithFlags(&pl->qst[qi], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_join[qi], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        batch_free(pl);
        return cuda_fail(e, "creating the batch plan");
    }
    // the tile lists stay on the host only as long as the plan (for mp_batch_tiles)
    *plan = pl;
    if (ws_bytes) *ws_bytes = pl->ws_bytes;
    return MP_OK;
}

extern "C" {

mp_status mp_batch_run(mp_batch_plan *plan, const void *T, double *P, int64_t *I, void *ws, size_t ws_bytes,
                       void *stream) {
    g_err[0] = 0;
    if (!plan) return fail(MP_ERR_INVALID_ARG, "plan is NULL");
    if (!T || !P || !I) return fail(MP_ERR_INVALID_ARG, "NULL T, P or I");
    if (!aligned(T, 4) || !aligned(P, 8) || !aligned(I, 8)) return fail(MP_ERR_INVALID_ARG, "misaligned T, P or I");
    if (!ws) return fail(MP_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", plan->ws_bytes);
    if (!aligned(ws, ALIGN)) return fail(MP_ERR_INVALID_ARG, "workspace not 256-byte aligned");
    if (ws_bytes < plan->ws_bytes)
        return fail(MP_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, plan->ws_bytes);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != plan->device) return fail(MP_ERR_INVALID_ARG, "plan made on device %d, current %d", plan->device, dev);
    cudaGetLastError();
    if (!plan->exec || plan->g_T != T || plan->g_P != P || plan->g_I != I || plan->g_ws != ws) {
        mp_status s = batch_build_graph(plan, T, P, I, ws);
        if (s != MP_OK) return s;
    }
    e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    counted(plan->nodes);
    return MP_OK;
}

int64_t mp_batch_windows(const mp_batch_plan *plan) { return plan ? plan->windows : -1; }

int64_t mp_batch_tiles(const mp_batch_plan *plan) {
    if (!plan) return -1;
    int64_t t = 0;
    for (const auto &q : plan->tiles) t += static_cast<int64_t>(q.size());
    return t;
}

mp_status mp_batch_plan_destroy(mp_batch_plan *plan) {
    batch_free(plan);
    return MP_OK;
}

}  // extern "C"

// ---- streaming append -----------------------------------------------------------------
struct mp_stream {
    int device = -1;
    int dist = MP_DIST_EUCLID;
    int m = 0;
    long long excl = 0;
    double p = 2.0;
    long long n = 0, N = 0, n_max = 0, N_max = 0;
    int reanchor = 4096;
    long long since_anchor = 0;
    double *x64 = nullptr, *state = nullptr, *R = nullptr, *P = nullptr, *mu = nullptr, *S = nullptr;
    long long *I = nullptr;
    unsigned char *flat = nullptr;
    double *part_r = nullptr;
    long long *part_k = nullptr;
    unsigned *counter = nullptr;
};

namespace {

void stream_free(mp_stream *s) {
    if (!s) return;
    void *ptrs[] = {s->x64, s->state, s->R, s->P, s->mu, s->S, s->I, s->flat, s->part_r, s->part_k, s->counter};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete s;
}

mpk::StreamArgs stream_args(const mp_stream *s) {
    mpk::StreamArgs a{};
    a.dist = s->dist == MP_DIST_EUCLID ? mpk::FIN_EUCLID : s->dist == MP_DIST_PNORM ? mpk::FIN_PNORM : mpk::FIN_ZNORM;
    a.m = s->m;
    a.excl = s->excl;
    a.p = s->dist == MP_DIST_PNORM ? s->p : 2.0;
    a.x = s->x64;
    a.state = s->state;
    a.R = s->R;
    a.P = s->P;
    a.I = reinterpret_cast<long long *>(s->I);
    a.mu = s->mu;
    a.S = s->S;
    a.flat = s->flat;
    a.part_r = s->part_r;
    a.part_k = s->part_k;
    a.counter = s->counter;
    return a;
}

template <typename Tin>
void stream_convert(const void *T, long long count, double *out, cudaStream_t st) {
    mpk::convert_f64_kernel<Tin><<<grid_for(count, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(
        static_cast<const Tin *>(T), count, count, out);
    counted();
}

}  // namespace

extern "C" {

mp_status mp_stream_create(int dist, const void *T, int dtype, int64_t n, int64_t n_max, int32_t m, int64_t excl,
                           double p, const mp_options *opt, mp_stream **out, void *stream) {
    g_err[0] = 0;
    if (!out) return fail(MP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dist < MP_DIST_EUCLID || dist > MP_DIST_ZNORM) return fail(MP_ERR_INVALID_ARG, "dist %d", dist);
    if (n_max < n) return fail(MP_ERR_INVALID_ARG, "n_max = %lld < n = %lld", (long long)n_max, (long long)n);
    if (opt && opt->struct_size == sizeof(mp_options) && (opt->k_begin != 0 || opt->k_end != 0))
        return fail(MP_ERR_UNSUPPORTED, "a streaming profile covers every diagonal");
    Problem pb{};
    pb.dist = dist;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = excl;
    pb.p = dist == MP_DIST_PNORM ? p : 2.0;
    // the full argument check of the one-shot entry points (pointers P, I are checked later)
    static const double dummy[1] = {0};
    mp_status s = check_problem(pb, T, dummy, reinterpret_cast<const int64_t *>(dummy), opt);
    if (s != MP_OK) return s;
    if (n_max - m + 1 >= (1ll << 31) - 1) return fail(MP_ERR_UNSUPPORTED, "n_max too large");
    if (pb.opt.reanchor < 0) return fail(MP_ERR_INVALID_ARG, "reanchor < 0");

    auto *sp = new mp_stream();
    sp->dist = dist;
    sp->m = m;
    sp->excl = excl;
    sp->p = pb.p;
    sp->n = n;
    sp->N = n - m + 1;
    sp->n_max = n_max;
    sp->N_max = n_max - m + 1;
    sp->reanchor = pb.opt.reanchor > 0 ? pb.opt.reanchor : 256;  // as the FP64 sweep's default
    const size_t Nm = static_cast<size_t>(sp->N_max);
    const size_t parts = (Nm + mpk::ST_NT - 1) / mpk::ST_NT + 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&sp->device);
    if (e == cudaSuccess) e = cudaMalloc(&sp->x64, sizeof(double) * n_max);
    if (e == cudaSuccess) e = cudaMalloc(&sp->state, sizeof(double) * Nm);
    if (e == cudaSuccess) e = cudaMalloc(&sp->R, sizeof(double) * Nm);
    if (e == cudaSuccess) e = cudaMalloc(&sp->P, sizeof(double) * Nm);
    if (e == cudaSuccess) e = cudaMalloc(&sp->I, sizeof(long long) * Nm);
    if (e == cudaSuccess) e = cudaMalloc(&sp->part_r, sizeof(double) * parts);
    if (e == cudaSuccess) e = cudaMalloc(&sp->part_k, sizeof(long long) * parts);
    if (e == cudaSuccess) e = cudaMalloc(&sp->counter, sizeof(unsigned));
    if (e == cudaSuccess && dist == MP_DIST_ZNORM) {
        e = cudaMalloc(&sp->mu, sizeof(double) * Nm);
        if (e == cudaSuccess) e = cudaMalloc(&sp->S, sizeof(double) * Nm);
        if (e == cudaSuccess) e = cudaMalloc(&sp->flat, Nm);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(sp->counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) {
        stream_free(sp);
        return cuda_fail(e, "allocating the streaming profile");
    }
    // the initial profile: the one-shot path (its workspace lives for this call only)
    mp_options o = pb.opt;
    o.polish = 1;
    const Layout L = layout(pb);
    void *ws = nullptr;
    e = cudaMallocAsync(&ws, L.total, st);
    if (e != cudaSuccess) {
        stream_free(sp);
        return cuda_fail(e, "allocating the initial workspace");
    }
    s = run(pb, T, sp->P, reinterpret_cast<int64_t *>(sp->I), ws, L.total, &o, stream);
    cudaFreeAsync(ws, st);
    if (s != MP_OK) {
        cudaStreamSynchronize(st);
        stream_free(sp);
        return s;
    }
    if (dtype == MP_F64) stream_convert<double>(T, n, sp->x64, st);
    else stream_convert<float>(T, n, sp->x64, st);
    const mpk::StreamArgs a = stream_args(sp);
    if (dist == MP_DIST_ZNORM) {
        mpk::window_stats_kernel<<<grid_for(sp->N, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(sp->x64, sp->N, m, sp->mu,
                                                                                        sp->S, sp->flat);
        counted();
    }
    mpk::stream_rescore_kernel<<<grid_for(sp->N, mpk::ST_NT), mpk::ST_NT, 0, st>>>(a, sp->N);
    mpk::stream_state_kernel<<<grid_for(sp->N, mpk::ST_NT), mpk::ST_NT, 0, st>>>(a, sp->N, excl + 1);
    counted(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        stream_free(sp);
        return cuda_fail(e, "initialising the streaming profile");
    }
    *out = sp;
    return MP_OK;
}

mp_status mp_stream_append(mp_stream *sp, const void *x, int dtype, int64_t count, void *stream) {
    g_err[0] = 0;
    if (!sp) return fail(MP_ERR_INVALID_ARG, "stream is NULL");
    if (count < 0) return fail(MP_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return MP_OK;
    if (!x) return fail(MP_ERR_INVALID_ARG, "x is NULL");
    if (dtype != MP_F32 && dtype != MP_F64) return fail(MP_ERR_INVALID_ARG, "dtype %d", dtype);
    if (!aligned(x, dtype == MP_F64 ? 8 : 4)) return fail(MP_ERR_INVALID_ARG, "misaligned x");
    if (sp->n + count > sp->n_max)
        return fail(MP_ERR_UNSUPPORTED, "append of %lld samples exceeds the capacity (%lld of %lld used)",
                    (long long)count, sp->n, sp->n_max);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != sp->device) return fail(MP_ERR_INVALID_ARG, "stream made on device %d, current %d", sp->device, dev);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    if (dtype == MP_F64) stream_convert<double>(x, count, sp->x64 + sp->n, st);
    else stream_convert<float>(x, count, sp->x64 + sp->n, st);
    const mpk::StreamArgs a = stream_args(sp);
    for (long long t = 0; t < count; ++t) {
        const long long j = sp->N;  // the new window
        if (sp->dist == MP_DIST_ZNORM) {
            mpk::stream_window_kernel<<<1, 32, 0, st>>>(a, j);
            counted();
        }
        const long long cand = j - sp->excl;  // diagonals excl + 1 .. j
        const unsigned blocks = static_cast<unsigned>(cand > 0 ? (cand + mpk::ST_NT - 1) / mpk::ST_NT : 1);
        mpk::stream_step_kernel<<<blocks, mpk::ST_NT, 0, st>>>(a, j);
        counted();
        sp->n += 1;
        sp->N += 1;
        if (++sp->since_anchor >= sp->reanchor) {  // the diagonals' state again from the definitions
            mpk::stream_state_kernel<<<grid_for(sp->N, mpk::ST_NT), mpk::ST_NT, 0, st>>>(a, sp->N, sp->excl + 1);
            counted();
            sp->since_anchor = 0;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "append");
    return MP_OK;
}

mp_status mp_stream_read(const mp_stream *sp, double *P, int64_t *I, void *stream) {
    g_err[0] = 0;
    if (!sp || !P || !I) return fail(MP_ERR_INVALID_ARG, "NULL stream, P or I");
    if (!aligned(P, 8) || !aligned(I, 8)) return fail(MP_ERR_INVALID_ARG, "misaligned P or I");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(P, sp->P, sizeof(double) * sp->N, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(I, sp->I, sizeof(long long) * sp->N, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "reading the streaming profile");
    return MP_OK;
}

int64_t mp_stream_windows(const mp_stream *sp) { return sp ? sp->N : -1; }

mp_status mp_stream_destroy(mp_stream *sp) {
    stream_free(sp);
    return MP_OK;
}

}  // extern "C"

// ---- anytime runs ---------------------------------------------------------------------
// One series, its tiles in a seeded random order; each run takes the next
// tiles of the queue, and the profile of the cells done so far can be read
// (and the keys checkpointed) between runs.
struct mp_anytime {
    mp_batch_plan *pl = nullptr;
    void *ws = nullptr;
    float *T = nullptr;            // the library's copy of the series
    int qi = -1;                   // the queue that holds the series' tiles
    long long cursor = 0, total = 0;
    unsigned long long seed = 0;
    bool started = false;
};

namespace {

constexpr unsigned long long ANYTIME_MAGIC = 0x4d50616e7974696dull;  // "MPanytim"

void anytime_free(mp_anytime *a) {
    if (!a) return;
    if (a->pl) batch_free(a->pl);
    if (a->ws) cudaFree(a->ws);
    if (a->T) cudaFree(a->T);
    delete a;
}

mpk::BatchData anytime_data(const mp_anytime *a, double *P, int64_t *I) {
    const mp_batch_plan *pl = a->pl;
    char *w = static_cast<char *>(a->ws);
    mpk::BatchData bd{};
    bd.series = pl->d_series;
    bd.w_start = pl->d_wstart;
    bd.S = pl->S;
    bd.windows = pl->windows;
    bd.T = a->T;
    bd.keys = reinterpret_cast<unsigned long long *>(w + pl->o_keys);
    if (pl->zwindows > 0) {
        bd.mu = reinterpret_cast<double *>(w + pl->o_mu);
        bd.Sx = reinterpret_cast<double *>(w + pl->o_S);
        bd.flat = reinterpret_cast<unsigned char *>(w + pl->o_flat);
        bd.df = reinterpret_cast<float *>(w + pl->o_df);
        bd.dg = reinterpret_cast<float *>(w + pl->o_dg);
        bd.inv = reinterpret_cast<float *>(w + pl->o_inv);
        bd.muh = reinterpret_cast<float *>(w + pl->o_muh);
        bd.mul = reinterpret_cast<float *>(w + pl->o_mul);
    }
    bd.P = P;
    bd.I = reinterpret_cast<long long *>(I);
    bd.p = pl->p;
    bd.polish = pl->polish;
    return bd;
}

// keys <- none, tickets <- 0, z statistics (once per object)
void anytime_start(mp_anytime *a, cudaStream_t st) {
    const mp_batch_plan *pl = a->pl;
    const mpk::BatchData bd = anytime_data(a, nullptr, nullptr);
    unsigned *tickets = reinterpret_cast<unsigned *>(static_cast<char *>(a->ws) + pl->o_tickets);
    const int gw = grid_for(pl->windows, mpk::PREP_NT);
    mpk::batch_init_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd.keys, pl->windows, tickets, mp_batch_plan::NQ);
    counted();
    if (pl->zwindows > 0) {
        mpk::batch_zstats_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd);
        mpk::batch_zoperands_kernel<<<gw, mpk::PREP_NT, 0, st>>>(bd);
        counted(2);
    }
    a->started = true;
}

}  // namespace

extern "C" {

mp_status mp_anytime_create(int dist, const void *T, int64_t n, int32_t m, int64_t excl, double p,
                            uint64_t seed, const mp_options *opt, mp_anytime **out, void *stream) {
    g_err[0] = 0;
    if (!out) return fail(MP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!T) return fail(MP_ERR_INVALID_ARG, "T is NULL");
    if (!aligned(T, 4)) return fail(MP_ERR_INVALID_ARG, "misaligned T");
    if (dist < MP_DIST_EUCLID || dist > MP_DIST_ZNORM) return fail(MP_ERR_INVALID_ARG, "dist %d", dist);
    const int64_t offs[2] = {0, n};
    const int32_t ms[1] = {m};
    const uint8_t ds[1] = {static_cast<uint8_t>(dist)};
    const int64_t ex[1] = {excl};
    mp_batch_desc d{};
    d.struct_size = sizeof(mp_batch_desc);
    d.num_series = 1;
    d.t_offsets = offs;
    d.m = ms;
    d.dist = ds;
    d.excl = ex;
    d.p = p;
    d.dtype = MP_F32;
    auto *a = new mp_anytime();
    a->seed = seed ? seed : 0x5eed5eed5eedull;
    size_t ws = 0;
    mp_status s = batch_plan_build(&d, opt, a->seed, &a->pl, &ws);
    if (s != MP_OK) {
        delete a;
        return s;
    }
    for (int qi = 0; qi < mp_batch_plan::NQ; ++qi)
        if (!a->pl->tiles[qi].empty()) a->qi = qi;
    a->total = a->qi < 0 ? 0 : static_cast<long long>(a->pl->tiles[a->qi].size());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&a->ws, ws);
    if (e == cudaSuccess) e = cudaMalloc(&a->T, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a->T, T, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        anytime_free(a);
        return cuda_fail(e, "allocating the anytime run");
    }
    anytime_start(a, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        anytime_free(a);
        return cuda_fail(e, "starting the anytime run");
    }
    *out = a;
    return MP_OK;
}

mp_status mp_anytime_run(mp_anytime *a, int64_t max_tiles, void *stream) {
    g_err[0] = 0;
    if (!a) return fail(MP_ERR_INVALID_ARG, "anytime run is NULL");
    if (max_tiles < 0) return fail(MP_ERR_INVALID_ARG, "max_tiles < 0");
    const long long count = std::min<long long>(max_tiles, a->total - a->cursor);
    if (count <= 0) return MP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaGetLastError();
    mp_batch_plan *pl = a->pl;
    const int qi = a->qi;
    unsigned *ticket = reinterpret_cast<unsigned *>(static_cast<char *>(a->ws) + pl->o_tickets) + qi;
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "resetting the queue ticket");
    const mpk::BatchData bd = anytime_data(a, nullptr, nullptr);
    const mpk::BatchQueue q{pl->d_tiles[qi] + a->cursor, static_cast<unsigned>(count), ticket};
    const int grid = static_cast<int>(std::min<long long>(pl->grid[qi], count));
    e = batch_queue_launch(pl, qi, grid, bd, q, st);
    counted();
    if (e != cudaSuccess) return cuda_fail(e, "anytime sweep launch");
    a->cursor += count;
    return MP_OK;
}

mp_status mp_anytime_read(const mp_anytime *a, double *P, int64_t *I, void *stream) {
    g_err[0] = 0;
    if (!a || !P || !I) return fail(MP_ERR_INVALID_ARG, "NULL anytime run, P or I");
    if (!aligned(P, 8) || !aligned(I, 8)) return fail(MP_ERR_INVALID_ARG, "misaligned P or I");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const mpk::BatchData bd = anytime_data(a, P, I);
    mpk::batch_finalize_kernel<<<grid_for(a->pl->windows, mpk::PREP_NT), mpk::PREP_NT, 0, st>>>(bd);
    counted();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "anytime finalize");
    return MP_OK;
}

int64_t mp_anytime_tiles_done(const mp_anytime *a) { return a ? a->cursor : -1; }

int64_t mp_anytime_tiles_total(const mp_anytime *a) { return a ? a->total : -1; }

size_t mp_anytime_checkpoint_size(const mp_anytime *a) {
    return a ? 4 * sizeof(unsigned long long) + sizeof(unsigned long long) * a->pl->windows : 0;
}

mp_status mp_anytime_checkpoint(const mp_anytime *a, void *host, size_t bytes, void *stream) {
    g_err[0] = 0;
    if (!a || !host) return fail(MP_ERR_INVALID_ARG, "NULL anytime run or buffer");
    if (bytes < mp_anytime_checkpoint_size(a))
        return fail(MP_ERR_INVALID_ARG, "checkpoint buffer %zu bytes < %zu", bytes, mp_anytime_checkpoint_size(a));
    unsigned long long *h = static_cast<unsigned long long *>(host);
    h[0] = ANYTIME_MAGIC;
    h[1] = a->seed;
    h[2] = static_cast<unsigned long long>(a->pl->windows);
    h[3] = static_cast<unsigned long long>(a->cursor);
    const void *keys = static_cast<const char *>(a->ws) + a->pl->o_keys;
    const cudaError_t e = cudaMemcpyAsync(h + 4, keys, sizeof(unsigned long long) * a->pl->windows,
                                          cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
    return MP_OK;
}

mp_status mp_anytime_restore(mp_anytime *a, const void *host, size_t bytes, void *stream) {
    g_err[0] = 0;
    if (!a || !host) return fail(MP_ERR_INVALID_ARG, "NULL anytime run or buffer");
    if (bytes < mp_anytime_checkpoint_size(a))
        return fail(MP_ERR_INVALID_ARG, "checkpoint buffer %zu bytes < %zu", bytes, mp_anytime_checkpoint_size(a));
    const unsigned long long *h = static_cast<const unsigned long long *>(host);
    if (h[0] != ANYTIME_MAGIC || h[1] != a->seed || h[2] != static_cast<unsigned long long>(a->pl->windows) ||
        h[3] > static_cast<unsigned long long>(a->total))
        return fail(MP_ERR_INVALID_ARG, "checkpoint does not belong to this series, seed and size");
    void *keys = static_cast<char *>(a->ws) + a->pl->o_keys;
    const cudaError_t e = cudaMemcpyAsync(keys, h + 4, sizeof(unsigned long long) * a->pl->windows,
                                          cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "restore copy");
    a->cursor = static_cast<long long>(h[3]);
    return MP_OK;
}

mp_status mp_anytime_destroy(mp_anytime *a) {
    anytime_free(a);
    return MP_OK;
}

}  // extern "C"

// ---- autotuning -------------------------------------------------------------------
namespace {

struct TuneEntry {
    int variant = 0, reanchor = 0;
    double ms = 0;
    int tile_rows = 0;
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune;

std::string tune_key(int dist, int dtype, int m, long long N, double p) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
    for (char &c : name)
        if (c == ' ' || c == '|') c = '_';
    int lg = 0;
    while ((2LL << lg) <= N) ++lg;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%d|%d|%d|%d|%.6g", name.c_str(), dist, dtype, m, lg,
             dist == MP_DIST_PNORM ? p : 2.0);
    return buf;
}

bool tune_lookup(const Problem &pb, mp_options &opt) {
    const std::string key = tune_key(pb.dist, pb.dtype, pb.m, pb.N, pb.p);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    opt.variant = it->second.variant;
    opt.reanchor = it->second.reanchor;
    opt.tile_rows = it->second.tile_rows;
    return true;
}

}  // namespace

extern "C" {

mp_status mp_autotune(int dist, const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double p,
                      double *P, int64_t *I, void *ws, size_t ws_bytes, const mp_options *opt,
                      int64_t slice_cells, int force, mp_options *best, double *times_ms,
                      int32_t max_times, int32_t *n_times, void *stream) {
    g_err[0] = 0;
    if (!best) return fail(MP_ERR_INVALID_ARG, "best is NULL");
    if (n_times) *n_times = 0;
    Problem pb{};
    pb.dist = dist;
    pb.dtype = dtype;
    pb.n = n;
    pb.m = m;
    pb.excl = excl;
    pb.p = dist == MP_DIST_PNORM ? p : 2.0;
    if (dist < MP_DIST_EUCLID || dist > MP_DIST_ZNORM) return fail(MP_ERR_INVALID_ARG, "dist %d", dist);
    mp_status s = check_problem(pb, T, P, I, opt);
    if (s != MP_OK) return s;
    *best = pb.opt;
    // candidates: (variant, reanchor, tile_rows)
    struct Cand { int variant, reanchor, tile_rows; };
    Cand cands[12];
    int nc = 0;
    if (p3_exact(pb)) {
        cands[nc++] = {MP_VARIANT_TALL, 0, 0};  // the one kernel whose p = 3 sums hold the tolerance
    } else if (pb.dist != MP_DIST_ZNORM && pb.opt.precision == MP_PREC_FP32) {
        Problem q = pb;
        q.opt.reanchor = 0;
        q.opt.tile_rows = 0;
        if (fast_path_applies(q)) {
            const int kind = kind_of(pb.dist, pb.p);
            if (kind == mpk::K_P2) cands[nc++] = {MP_VARIANT_FAST_FILTER, 0, 0};
            cands[nc++] = {MP_VARIANT_FAST, 0, 0};
            // the tile height the default does not take: one-step tiles where it
            // takes tall ones, tall ones where they still fill a few waves
            const long long L = pb.N - pb.k_first, nb = (pb.k_end - pb.k_first + mpk::V2_KW - 1) / mpk::V2_KW;
            const long long R0 = sweep2_rows(q, L, nb);
            const int variant = kind == mpk::K_P2 ? MP_VARIANT_FAST_FILTER : MP_VARIANT_FAST;
            if (R0 != mpk::V2_R) cands[nc++] = {variant, 0, static_cast<int>(mpk::V2_R)};
            else if (mpk::v2_prefix(L, nb, V2_TALL_R) >= V2_TALL_TUNE_TILES &&
                     mpk::sweep2_smem_bytes(pb.m, V2_TALL_R) <= mpk::V2_SMEM_MAX)
                cands[nc++] = {variant, 0, static_cast<int>(V2_TALL_R)};
        }
        // the generic kernel with its default interval and with 16, 32, 64 rows,
        // each effective interval (choose_block) once
        int seen[4], ns = 0;
        for (int target : {0, 16, 32, 64}) {
            int B = 0, Q = 0;
            choose_block(m, target, mpk::SW_QMAX, B, Q);
            bool dup = false;
            for (int t = 0; t < ns; ++t) dup |= seen[t] == B;
            if (dup || (target > 0 && B != target)) continue;
            seen[ns++] = B;
            Problem g = pb;
            g.opt.reanchor = target;
            if (generic_smem(g) > 0) cands[nc++] = {MP_VARIANT_GENERIC, target, 0};
        }
        // the tall kernel only where its accuracy holds (see use_tall)
        if (tall_applies(pb) && (pb.m >= 512 || generic_smem(pb) == 0)) cands[nc++] = {MP_VARIANT_TALL, 0, 0};
    } else if (pb.dist == MP_DIST_ZNORM && pb.opt.precision == MP_PREC_FP32) {
        // the z-normalised kernel with and without its filter, at the default tile
        // height and at shorter tiles (more tiles for series that do not fill the GPU)
        const long long S0 = mpk::z_rows_per_tile(pb.m, true);
        for (int t : {0, 16384, 4096}) {
            if (t > 0 && (t >= S0 || t >= pb.N)) continue;
            cands[nc++] = {MP_VARIANT_FAST_FILTER, 0, t};
            cands[nc++] = {MP_VARIANT_FAST, 0, t};
        }
        cands[nc++] = {MP_VARIANT_FAST_FILTER_BOUND, 0, 0};  // the looser, cheaper filter bound
    }
    if (nc <= 1) {  // nothing to choose
        if (nc == 1) {
            best->variant = cands[0].variant;
            best->reanchor = cands[0].reanchor;
            best->tile_rows = cands[0].tile_rows;
        }
        return MP_OK;
    }
    const std::string key = tune_key(dist, dtype, m, pb.N, pb.p);
    if (!force) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            best->variant = it->second.variant;
            best->reanchor = it->second.reanchor;
            best->tile_rows = it->second.tile_rows;
            return MP_OK;
        }
    }
    // the whole diagonal range by default: on a slice the profile's thresholds
    // stay as loose as at the start of a sweep, which misjudges the block filter
    const long long K = slice_cells > 0 ? std::max<long long>(
                                              1, std::min<long long>(pb.N - pb.k_first,
                                                                     slice_cells / std::max<long long>(pb.N, 1)))
                                        : pb.N - pb.k_first;
    if (pb.N - pb.k_first <= 0) return MP_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    cudaEvent_t user0 = g_ev_start, user1 = g_ev_end;
    double bestms = 1e300;
    int bi = -1;
    for (int c = 0; c < nc; ++c) {
        mp_options o = pb.opt;
        o.variant = cands[c].variant;
        o.reanchor = cands[c].reanchor;
        o.tile_rows = cands[c].tile_rows;
        o.polish = 0;
        o.k_begin = pb.k_first;
        o.k_end = pb.k_first + K;
        Problem q = pb;
        g_ev_start = nullptr;
        g_ev_end = nullptr;
        s = run(q, T, P, I, ws, ws_bytes, &o, stream);  // warm-up
        if (s == MP_OK) {
            q = pb;
            g_ev_start = e0;  // the sweep kernel alone
            g_ev_end = e1;
            s = run(q, T, P, I, ws, ws_bytes, &o, stream);
        }
        g_ev_start = user0;
        g_ev_end = user1;
        if (s != MP_OK) break;
        e = cudaStreamSynchronize(st);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "timing a candidate");
            break;
        }
        if (times_ms && c < max_times) times_ms[c] = ms;
        if (ms < bestms) {
            bestms = ms;
            bi = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != MP_OK) return s;
    if (n_times) *n_times = nc;
    best->variant = cands[bi].variant;
    best->reanchor = cands[bi].reanchor;
    best->tile_rows = cands[bi].tile_rows;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = TuneEntry{cands[bi].variant, cands[bi].reanchor, bestms, cands[bi].tile_rows};
    return MP_OK;
}

mp_status mp_autotune_cache_save(const char *path) {
    g_err[0] = 0;
    if (!path) return fail(MP_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "w");
    if (!f) return fail(MP_ERR_INVALID_ARG, "cannot write %s", path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    fprintf(f, "# mp autotune cache: key variant reanchor ms tile_rows\n");
    for (const auto &kv : g_tune)
        fprintf(f, "%s %d %d %.6f %d\n", kv.first.c_str(), kv.second.variant, kv.second.reanchor, kv.second.ms,
                kv.second.tile_rows);
    fclose(f);
    return MP_OK;
}

mp_status mp_autotune_cache_load(const char *path) {
    g_err[0] = 0;
    if (!path) return fail(MP_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "r");
    if (!f) return fail(MP_ERR_INVALID_ARG, "cannot read %s", path);
    std::map<std::string, TuneEntry> add;
    char line[512];
    int lineno = 0;
    while (fgets(line, sizeof line, f)) {
        ++lineno;
        if (line[0] == '#' || line[0] == '\n') continue;
        char key[300];
        TuneEntry t;
        const int got = sscanf(line, "%299s %d %d %lf %d", key, &t.variant, &t.reanchor, &t.ms, &t.tile_rows);
        if ((got != 4 && got != 5) || t.variant < MP_VARIANT_AUTO ||
            (t.variant > MP_VARIANT_TALL && t.variant != MP_VARIANT_FAST_FILTER_BOUND) || t.reanchor < 0 ||
            t.tile_rows < 0 || t.tile_rows % 1024 != 0) {
            fclose(f);
            return fail(MP_ERR_INVALID_ARG, "%s:%d: malformed entry", path, lineno);
        }
        add[key] = t;
    }
    fclose(f);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto &kv : add) g_tune[kv.first] = kv.second;
    return MP_OK;
}

int64_t mp_autotune_cache_size(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return static_cast<int64_t>(g_tune.size());
}

}  // extern "C"
