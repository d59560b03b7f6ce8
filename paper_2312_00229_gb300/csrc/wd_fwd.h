// Internal launch interface of the forward kernel (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wd_common.cuh"

namespace wdweno {

struct FwdArgs {
  const void* in;
  void* out;
  int in_dtype, out_dtype;
  int64_t n, m, planes;          // coarse rows, columns, channels
  int64_t in_sc, in_sh, in_sw;   // element strides
  int64_t out_sc, out_sh, out_sw;
  int64_t orows, ocols;          // output extent (2n or 2n-1, ...)
  int64_t rows_per_band;
  int out_vec;                   // unit column stride and 2-element aligned rows
  int out_vec4;                  // unit column stride and 4-element aligned rows
  int threads;                   // CTA width: 256 or 128 (one column), 128 or 64 (two)
  int cols;                      // coarse columns per thread: 1, or 2 (paired tile)
};

// CTA shape of a one-launch forward over images m columns wide: `threads`
// per CTA and `cols` coarse columns per thread (1: 256 or 128 threads, 247
// or 119 output columns per strip; 2: 128 or 64 threads, 246 or 118), the
// one that spends the fewest weighted column-steps across the width.
void fwd_shape_for(int64_t m, int* threads, int* cols);

int tile_width_fwd();
int threads_fwd();
cudaError_t launch_zoom2x_fwd(const FwdArgs& a, const MethodConsts& k, int bmode,
                              cudaStream_t stream);
// Abandoned bounded waits counted by the forward kernels of each translation
// unit (summed; optionally reset).
cudaError_t fwd_wait_timeouts(unsigned int* count, bool reset);
cudaError_t fwd_wait_timeouts_typed(unsigned int* count, bool reset);
cudaError_t fwd_wait_timeouts_batched(unsigned int* count, bool reset);

}  // namespace wdweno
