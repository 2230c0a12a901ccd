// a7, the steps of a batch around its sweeps: keys and queue tickets, the
// z-normalised statistics and operands of every z window, and the finalize of
// every window (see mp_batch.cuh for the batch layout).  Host translation
// unit only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_batch.cuh"
#include "mp_prep.cuh"

namespace mpk {

__global__ void __launch_bounds__(PREP_NT) batch_init_kernel(unsigned long long *keys, long long windows,
                                                             unsigned *tickets, int ntickets) {
    if (blockIdx.x == 0 && threadIdx.x < ntickets) tickets[threadIdx.x] = 0u;
    for (long long x = blockIdx.x * (long long)PREP_NT + threadIdx.x; x < windows;
         x += (long long)gridDim.x * PREP_NT)
        keys[x] = KEY_NONE;
}

__global__ void __launch_bounds__(PREP_NT) batch_zstats_kernel(const BatchData d) {
    for (long long g = blockIdx.x * (long long)PREP_NT + threadIdx.x; g < d.windows;
         g += (long long)gridDim.x * PREP_NT) {
        const BatchSeries &s = d.series[batch_series_of(d, g)];
        if (s.dist != FIN_ZNORM) continue;
        const long long i = g - s.w_off, z = s.z_off;
        window_stats_at(d.T + s.t_off, i, s.m, d.mu[z + i], d.Sx[z + i], d.flat[z + i]);
    }
}

__global__ void __launch_bounds__(PREP_NT) batch_zoperands_kernel(const BatchData d) {
    for (long long g = blockIdx.x * (long long)PREP_NT + threadIdx.x; g < d.windows;
         g += (long long)gridDim.x * PREP_NT) {
        const BatchSeries &s = d.series[batch_series_of(d, g)];
        if (s.dist != FIN_ZNORM) continue;
        const long long i = g - s.w_off, z = s.z_off;
        znorm_operands_at(d.T + s.t_off, i, s.N, s.m, d.mu + z, d.Sx + z, d.flat + z, 0.0, d.df + z, d.dg + z,
                          d.inv + z, d.muh + z, d.mul + z);
    }
}

__global__ void __launch_bounds__(PREP_NT) batch_finalize_kernel(const BatchData d) {
    for (long long g = blockIdx.x * (long long)PREP_NT + threadIdx.x; g < d.windows;
         g += (long long)gridDim.x * PREP_NT) {
        const BatchSeries &s = d.series[batch_series_of(d, g)];
        FinalizeArgsT<float> a{};
        a.keys = d.keys + s.w_off;
        a.keys128 = nullptr;
        a.x = d.T + s.t_off;
        a.mu = s.dist == FIN_ZNORM ? d.mu + s.z_off : nullptr;
        a.S = s.dist == FIN_ZNORM ? d.Sx + s.z_off : nullptr;
        a.N = s.N;
        a.m = s.m;
        a.dist = s.dist;
        a.p = s.dist == FIN_PNORM ? d.p : 2.0;
        a.polish = d.polish;
        a.P = d.P + s.w_off;
        a.I = d.I + s.w_off;
        finalize_at(a, g - s.w_off);
    }
}

}  // namespace mpk
