// Launchers of the diagonal-sweep kernels (a3-a5), one group per translation
// unit so that the library's heavy kernels compile in parallel.  Each call
// sets the kernel's dynamic shared-memory limit, enqueues it on `st` and
// returns the launch status; the caller has validated every argument.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "mp_batch.cuh"
#include "mp_sweep.cuh"
#include "mp_sweep2.cuh"
#include "mp_sweep_z2.cuh"

namespace mpk {

// k_sweep2.cu: the two-stream Euclidean sweep, with or without the block
// filter, in one-step tiles (a.R == V2_R; taller tiles go to k_sweep2_tall.cu)
cudaError_t sweep2_p2_launch(bool filter, const Sweep2Args &a, size_t smem, cudaStream_t st);
int *sweep2_p2_error_word();

// k_sweep2_tall.cu: the same in tall tiles (a.R > V2_R)
cudaError_t sweep2_p2_tall_launch(bool filter, const Sweep2Args &a, size_t smem, cudaStream_t st);
int *sweep2_tall_error_word();

// k_sweep2_p13.cu: the two-stream p-norm sweep for p = 1 (kind K_P1) and p = 3
// (K_P3), one-step or tall tiles
cudaError_t sweep2_p13_launch(int kind, const Sweep2Args &a, size_t smem, cudaStream_t st);
int *sweep2_p13_error_word();

// k_sweepz.cu: tall float-float tiles (mode K_Z: z-normalised; K_P2, K_P1, K_P3:
// long Euclidean / p-norm windows) and the batch queue of z-normalised series;
// filter 0 none, 1 the exact row-minimum filter, 2 (K_Z) the partner-scale bound
cudaError_t sweepz_launch(int mode, int filter, const SweepZArgs &a, size_t smem, cudaStream_t st);
cudaError_t batchz_setup(size_t smem, int *ctas_per_sm);
cudaError_t batchz_launch(int grid, size_t smem, const BatchData &d, const BatchQueue &q, cudaStream_t st);
int *sweepz_error_word();

// k_batch2.cu: batch queues of the two-stream sweep (kind K_P2 with or without
// the filter, K_P1, K_P3)
cudaError_t batch2_setup(int kind, bool filter, size_t smem, int *ctas_per_sm);
cudaError_t batch2_launch(int kind, bool filter, int grid, size_t smem, const BatchData &d, const BatchQueue &q,
                          cudaStream_t st);
int *batch2_error_word();

// k_generic.cu: the generic FP32 sweep (any p, float64 input split hi / lo)
// and its batch queues
cudaError_t generic_launch(int kind, bool split, const SweepArgs &a, size_t smem, cudaStream_t st);
cudaError_t batchg_setup(int kind, size_t smem, int *ctas_per_sm);
cudaError_t batchg_launch(int kind, int grid, size_t smem, const BatchData &d, const BatchQueue &q, int *err,
                          cudaStream_t st);
int *generic_error_word();

}  // namespace mpk
