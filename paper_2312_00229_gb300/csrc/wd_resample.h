// Internal launch interface of the tensor-WENO resampling kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wd_common.cuh"

namespace wdweno {

struct ResampleArgs {
  const void* in;
  void* out;
  int in_dtype, out_dtype;
  int64_t n, m, planes;          // input rows, columns, channels
  int64_t n_out, m_out;          // output rows, columns
  int64_t in_sc, in_sh, in_sw;
  int64_t out_sc, out_sh, out_sw;
  int clamp_float;
  int out_vec4;                  // unit column stride, rows and planes of 4-element
                                 // multiples, 4-element aligned base
  int win_rows;                  // window rows of the tiled kernel (set by the launcher)
};

cudaError_t launch_resample(const ResampleArgs& a, float eps, float beta, int bmode,
                            cudaStream_t stream);

}  // namespace wdweno
