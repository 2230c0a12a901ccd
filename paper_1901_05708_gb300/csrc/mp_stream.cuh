// Streaming append: keep a matrix profile current while samples arrive.
//
// The paper notes that its incremental formulation also supports keeping the
// profile up to date when the series grows (Sec. 1), without giving the
// algorithm.  Here it is the diagonal recurrence run one row at a time at the
// end of the series: appending a sample creates one window j = N, and on
// every diagonal k = j - i the new cell (i, j) follows from the diagonal's
// previous last cell (i - 1, j - 1) in O(1) (Lemma 1, 2 or 3), except the new
// diagonal k = j (i = 0), which is computed from the definition.  Each new
// cell is offered to row i (a right neighbour) and to the new row j (a left
// neighbour), so one append costs O(N) and keeps P, I exact.
//
// State, all FP64 (an append is O(N) work, so FP64's rate is no obstacle):
//   state[k]  score of the last cell of diagonal k: the sum of squares
//             (Euclid), of |.|^p (p-norm), or the centred covariance (z-norm)
//   R[i]      score of row i's current best candidate (P[i] = finish(R[i]))
//   mu, S, flat   window statistics (z-norm)
// The state is recomputed from the definitions every `reanchor` appends, and
// a row's new best is rescored from the definition when it is found.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"
#include "mp_prep.cuh"

namespace mpk {

constexpr int ST_NT = 256;
constexpr long long ST_NO_K = 1ll << 60;  // "no candidate" (2 * ST_NO_K still fits)

struct StreamArgs {
    int dist;                 // FIN_EUCLID, FIN_PNORM, FIN_ZNORM
    int m;
    long long excl;
    double p;
    const double *x;          // series, FP64
    double *state;            // per diagonal k
    double *R;                // per window: score of the current best
    double *P;                // per window: distance of the current best
    long long *I;             // per window: index of the current best, or -1
    double *mu, *S;           // z-norm window statistics
    unsigned char *flat;
    double *part_r;           // per block: best (score, k) for the new row
    long long *part_k;
    unsigned *counter;        // blocks done (reset by the last block)
};

// score of (i, j) from the definitions
__device__ __forceinline__ double st_direct(const StreamArgs &a, long long i, long long j) {
    const double *xi = a.x + i, *xj = a.x + j;
    double acc = 0.0;
    if (a.dist == FIN_ZNORM) {
        const double mi = a.mu[i], mj = a.mu[j];
        for (int l = 0; l < a.m; ++l) acc = fma(xi[l] - mi, xj[l] - mj, acc);
    } else if (a.dist == FIN_PNORM) {
        for (int l = 0; l < a.m; ++l) acc += pow_abs(xi[l] - xj[l], a.p);
    } else {
        for (int l = 0; l < a.m; ++l) {
            const double d = xi[l] - xj[l];
            acc = fma(d, d, acc);
        }
    }
    return acc;
}

// the score the profile compares (Euclid / p-norm: the state; z-norm: 2m(1 - rho))
__device__ __forceinline__ double st_score(const StreamArgs &a, double st, long long i, long long j) {
    if (a.dist != FIN_ZNORM) return st;
    if (a.flat[i] || a.flat[j]) return __longlong_as_double(0x7ff0000000000000ll);
    const double rho = st / sqrt(a.S[i] * a.S[j]);
    return fmin(fmax(2.0 * a.m * (1.0 - rho), 0.0), 4.0 * a.m);
}

__device__ __forceinline__ double st_finish(const StreamArgs &a, double s) {
    if (s < 0) s = 0;
    if (a.dist == FIN_PNORM) {
        if (a.p == 1.0) return s;
        if (a.p == 2.0) return sqrt(s);
        return pow(s, 1.0 / a.p);
    }
    return sqrt(s);
}

// (s1, key1) < (s2, key2) with key = 2k + [right]
__device__ __forceinline__ bool st_less(double s1, long long key1, double s2, long long key2) {
    return s1 < s2 || (s1 == s2 && key1 < key2);
}

// state[k] for every diagonal k in [k0, N), from the definitions: the last
// cell (N - 1 - k, N - 1) of each diagonal.
__global__ void __launch_bounds__(ST_NT) stream_state_kernel(const StreamArgs a, long long N, long long k0) {
    for (long long k = k0 + blockIdx.x * (long long)ST_NT + threadIdx.x; k < N; k += (long long)gridDim.x * ST_NT)
        a.state[k] = st_direct(a, N - 1 - k, N - 1);
}

// R[i] = score of (i, I[i]) from the definitions (after the initial sweep).
__global__ void __launch_bounds__(ST_NT) stream_rescore_kernel(const StreamArgs a, long long N) {
    for (long long i = blockIdx.x * (long long)ST_NT + threadIdx.x; i < N; i += (long long)gridDim.x * ST_NT) {
        const long long j = a.I[i];
        a.R[i] = j < 0 ? __longlong_as_double(0x7ff0000000000000ll) : st_score(a, st_direct(a, i, j), i, j);
    }
}

// Statistics of the new window j (z-norm), one thread.
__global__ void stream_window_kernel(const StreamArgs a, long long j) {
    if (blockIdx.x == 0 && threadIdx.x == 0) window_stats_at(a.x, j, a.m, a.mu[j], a.S[j], a.flat[j]);
}

// Append window j: update every diagonal k in [excl + 1, j], offer cell
// (j - k, j) to row j - k and to row j.  Rows j - k are touched by one thread
// each; row j's best is reduced per block, then by the last block.
__global__ void __launch_bounds__(ST_NT) stream_step_kernel(const StreamArgs a, long long j) {
    __shared__ double sr[ST_NT];
    __shared__ long long sk[ST_NT];
    __shared__ bool last;
    const long long kmin = a.excl + 1;
    double best = __longlong_as_double(0x7ff0000000000000ll);
    long long bestk = ST_NO_K;
    const long long k = kmin + blockIdx.x * (long long)ST_NT + threadIdx.x;
    if (k <= j) {
        const long long i = j - k;
        double st;
        if (k == j) {
            st = st_direct(a, 0, j);  // the new diagonal
        } else if (a.dist == FIN_ZNORM) {
            // centred covariance update (Lemma 3 around the window means)
            const double *x = a.x;
            const int m = a.m;
            const double dfi = 0.5 * (x[i - 1 + m] - x[i - 1]), dfj = 0.5 * (x[j - 1 + m] - x[j - 1]);
            const double dgi = (x[i - 1 + m] - a.mu[i]) + (x[i - 1] - a.mu[i - 1]);
            const double dgj = (x[j - 1 + m] - a.mu[j]) + (x[j - 1] - a.mu[j - 1]);
            st = a.state[k] + dfi * dgj + dfj * dgi;
        } else {
            const double *x = a.x;
            const int m = a.m;
            const double e = x[i + m - 1] - x[j + m - 1], f = x[i - 1] - x[j - 1];
            st = a.state[k] + (a.dist == FIN_PNORM ? pow_abs(e, a.p) - pow_abs(f, a.p) : e * e - f * f);
        }
        a.state[k] = st;
        const double s = st_score(a, st, i, j);
        // row i: a right neighbour at distance k
        const long long Ii = a.I[i];
        const long long key_old = Ii < 0 ? 0x7fffffffffffffffll : 2 * (Ii > i ? Ii - i : i - Ii) + (Ii > i ? 1 : 0);
        const bool finite = s < __longlong_as_double(0x7ff0000000000000ll);  // false for NaN and flat windows
        if (finite && st_less(s, 2 * k + 1, a.R[i], key_old)) {
            // a new best (rare): its score again from the definition, so that P
            // carries no drift of the recurrence
            const double ex = st_score(a, st_direct(a, i, j), i, j);
            a.R[i] = ex;
            a.I[i] = j;
            a.P[i] = st_finish(a, ex);
        }
        if (finite) {
            best = s;
            bestk = k;
        }
    }
    sr[threadIdx.x] = best;
    sk[threadIdx.x] = bestk;
    __syncthreads();
    for (int w = ST_NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w && st_less(sr[threadIdx.x + w], 2 * sk[threadIdx.x + w], sr[threadIdx.x], 2 * sk[threadIdx.x])) {
            sr[threadIdx.x] = sr[threadIdx.x + w];
            sk[threadIdx.x] = sk[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.part_r[blockIdx.x] = sr[0];
        a.part_k[blockIdx.x] = sk[0];
        __threadfence();
        last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: row j from the partial minima
    __threadfence();
    best = __longlong_as_double(0x7ff0000000000000ll);
    bestk = ST_NO_K;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += ST_NT) {
        const double r = *((volatile double *)a.part_r + b);
        const long long kk = *((volatile long long *)a.part_k + b);
        if (st_less(r, 2 * kk, best, 2 * bestk)) {
            best = r;
            bestk = kk;
        }
    }
    sr[threadIdx.x] = best;
    sk[threadIdx.x] = bestk;
    __syncthreads();
    for (int w = ST_NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w && st_less(sr[threadIdx.x + w], 2 * sk[threadIdx.x + w], sr[threadIdx.x], 2 * sk[threadIdx.x])) {
            sr[threadIdx.x] = sr[threadIdx.x + w];
            sk[threadIdx.x] = sk[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool found = sk[0] != ST_NO_K && sr[0] == sr[0] &&
                           sr[0] != __longlong_as_double(0x7ff0000000000000ll);
        const double ex = found ? st_score(a, st_direct(a, j - sk[0], j), j - sk[0], j)
                                : __longlong_as_double(0x7ff0000000000000ll);
        a.R[j] = ex;
        a.I[j] = found ? j - sk[0] : -1;
        a.P[j] = found ? st_finish(a, ex) : __longlong_as_double(0x7ff0000000000000ll);
        *a.counter = 0u;
    }
}

}  // namespace mpk
