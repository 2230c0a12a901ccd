// a7: many independent matrix profiles in one graph (the batch queue).
//
// A batch is S series concatenated in one FP32 array.  Series s has n_s
// samples, window length m_s, exclusion zone excl_s and its own distance;
// its N_s = n_s - m_s + 1 profile entries sit at w_s = sum_{r<s} N_r in the
// key array and in P, I.  The per-series steps are the single-problem steps
// (window statistics, sweep, finalize) run over all series at once:
//   batch_init      keys <- none, queue tickets <- 0
//   batch_zstats    FP64 window statistics of the z-normalised series
//   batch_zoperands FP32 operands of the centred-covariance sweep
//   *_batch_kernel  persistent CTAs take tiles from a queue (one atomic
//                   ticket per tile); the queue takes the series in turn
//                   (first tiles of all series, then second tiles, ...),
//                   longest first within a turn
//   batch_finalize  keys -> P, I (FP64 polish)
// One queue per sweep kernel: the two-stream sweep (m a multiple of 32) for
// p = 2 and for the batch's p-norm exponent when it is 1 or 3, the
// float-float z-normalised sweep, and the generic FP32 sweep (other m, other
// p) for p = 2 and for the batch's exponent.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_device.cuh"
#include "mp_sweep.cuh"
#include "mp_sweep2.cuh"
#include "mp_sweep_z2.cuh"

namespace mpk {

struct BatchSeries {
    long long t_off;    // first sample in the concatenated series
    long long w_off;    // first window (keys, P, I)
    long long z_off;    // first window in the z-normalised operand arrays, or -1
    long long n, N, k_first;
    int m, dist;        // dist: FIN_EUCLID, FIN_PNORM or FIN_ZNORM (mp_prep.cuh)
    int B, Q, RL;       // generic sweep: re-anchor block, ring blocks, leaving rows
    int zS;             // z-normalised sweep: rows per tile
};

struct BatchTile {
    int series, band, rt;
    int rank;  // position among its series' tiles (queue order only)
};

struct BatchQueue {
    const BatchTile *tiles;
    unsigned count;
    unsigned *ticket;
};

struct BatchData {
    const BatchSeries *series;
    const long long *w_start;  // [S + 1]: w_off of each series, then the total
    int S;
    long long windows;         // total windows
    const float *T;
    unsigned long long *keys;
    double *mu, *Sx;           // z-normalised statistics, per z window
    unsigned char *flat;
    float *df, *dg, *inv, *muh, *mul;
    double *P;
    long long *I;
    double p;
    int polish;
};

// series that owns window g (w_start is increasing; empty series never match)
__device__ __forceinline__ int batch_series_of(const BatchData &d, long long g) {
    int lo = 0, hi = d.S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d.w_start[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Thread 0 takes the next ticket and publishes the tile; false when the queue
// is empty.  The caller synchronises before the next call (the tile body and
// the shared arguments must be done with).
__device__ __forceinline__ bool batch_next(const BatchQueue &q, const BatchData &d, BatchTile &tile,
                                           const BatchSeries *&sr, BatchTile *s_tile) {
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(q.ticket, 1u);
        *s_tile = t < q.count ? q.tiles[t] : BatchTile{-1, 0, 0, 0};
    }
    __syncthreads();
    tile = *s_tile;
    if (tile.series < 0) return false;
    sr = d.series + tile.series;
    return true;
}

template <int KIND, bool FILTER>
__global__ void __launch_bounds__(V2_NT, 2) sweep2_batch_kernel(const BatchData d, const BatchQueue q) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Sweep2Args sa;
    __shared__ BatchTile s_tile;
    for (;;) {
        BatchTile tile;
        const BatchSeries *sr;
        if (!batch_next(q, d, tile, sr, &s_tile)) break;
        if (threadIdx.x == 0) {
            sa.t = d.T + sr->t_off;
            sa.keys = d.keys + sr->w_off;
            sa.n = sr->n;
            sa.N = sr->N;
            sa.k_first = sr->k_first;
            sa.k_end = sr->N;
            sa.L = sr->N - sr->k_first;
            sa.nb = (sa.L + V2_KW - 1) / V2_KW;
            sa.tiles = 0;
            sa.m = sr->m;
            sa.Q = v2_ring_blocks(KIND);
            sa.B = sr->m / sa.Q;
            sa.R = V2_R;  // one-step tiles (the queue's tiles are V2_R rows)
        }
        __syncthreads();
        sweep2_tile<KIND, FILTER, false>(sa, tile.band, tile.rt, smem);
        __syncthreads();
    }
}

template <int MODE>
__global__ void __launch_bounds__(Z_NT, 2) sweepz_batch_kernel(const BatchData d, const BatchQueue q) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepZArgs za;
    __shared__ BatchTile s_tile;
    for (;;) {
        BatchTile tile;
        const BatchSeries *sr;
        if (!batch_next(q, d, tile, sr, &s_tile)) break;
        if (threadIdx.x == 0) {
            const long long z = sr->z_off;
            za.t = d.T + sr->t_off;
            za.tlo = nullptr;
            za.muh = d.muh + z;
            za.mul = d.mul + z;
            za.df = d.df + z;
            za.dg = d.dg + z;
            za.inv = d.inv + z;
            za.keys = d.keys + sr->w_off;
            za.n = sr->n;
            za.N = sr->N;
            za.k_first = sr->k_first;
            za.k_end = sr->N;
            za.L = sr->N - sr->k_first;
            za.nb = (za.L + Z_KW - 1) / Z_KW;
            za.tiles = 0;
            za.S = sr->zS;
            za.m = sr->m;
        }
        __syncthreads();
        sweepz_tile<MODE, 0>(za, tile.band, tile.rt, smem);
        __syncthreads();
    }
}

constexpr int BATCH_GEN_R = 2048;  // rows per tile of the generic sweep in a batch

template <int KIND>
__global__ void __launch_bounds__(SW_NT, 2) sweep_batch_kernel(const BatchData d, const BatchQueue q, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SweepArgs ga;
    __shared__ BatchTile s_tile;
    for (;;) {
        BatchTile tile;
        const BatchSeries *sr;
        if (!batch_next(q, d, tile, sr, &s_tile)) break;
        if (threadIdx.x == 0) {
            ga.hi = d.T + sr->t_off;
            ga.lo = nullptr;
            ga.keys = d.keys + sr->w_off;
            ga.err = err;
            ga.n = sr->n;
            ga.N = sr->N;
            ga.k_first = sr->k_first;
            ga.k_end = sr->N;
            ga.L = sr->N - sr->k_first;
            ga.R = BATCH_GEN_R;
            ga.q = SW_KW / BATCH_GEN_R;
            ga.C = (ga.L + ga.R - 1) / ga.R;
            ga.nb = (ga.L + SW_KW - 1) / SW_KW;
            ga.tiles = 0;
            ga.m = sr->m;
            ga.B = sr->B;
            ga.Q = sr->Q;
            ga.RL = sr->RL;
            ga.p = static_cast<float>(d.p);
        }
        __syncthreads();
        sweep_tile<KIND, false>(ga, tile.band, tile.rt, smem);
        __syncthreads();
    }
}

}  // namespace mpk
