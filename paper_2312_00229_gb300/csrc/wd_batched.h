// Internal launch interface of the persistent batched forward kernel.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "wd_common.cuh"
#include "wdweno.h"

namespace wdweno {

struct BatchedArgs {
  int count;
  const weno_image* in;   // device array
  const weno_image* out;  // device array
  int in_dtype, out_dtype, out_mode;
  int64_t rows_per_band;
  int threads;            // CTA width: 256 or 128 (one column per thread), 128 or 64 (two)
  int cols;               // coarse columns per thread: 1 or 2
  void* workspace;        // >= batched_workspace_bytes(count), 16-byte aligned
};

size_t batched_workspace_bytes(int count);
cudaError_t launch_zoom2x_batched(const BatchedArgs& a, const MethodConsts& k, int bmode,
                                  cudaStream_t stream);

}  // namespace wdweno
