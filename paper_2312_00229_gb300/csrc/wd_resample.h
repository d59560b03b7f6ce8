// Internal launch interface of the tensor-WENO resampling kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wd_common.cuh"

namespace wdweno {

// Exact unsigned 32-bit division by an invariant d = n_out - 1 through a
// multiply-high (Granlund and Montgomery, "Division by Invariant Integers
// using Multiplication", PLDI 1994, Fig. 4.1): with l = ceil(log2 d) and
// mag = floor(2^32 (2^l - d) / d) + 1,
//     t1 = mulhi(mag, x),  x / d = (t1 + ((x - t1) >> sh1)) >> sh2,
// sh1 = min(l, 1), sh2 = max(l - 1, 0), for every 0 <= x < 2^32.
struct AxisDiv {
  uint32_t mag;
  int sh1, sh2;
  int fast;   // every numerator j (n - 1) of the axis is below 2^32
  float inv;  // 1 / d (for the cell offset t)
};

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
  int tile_rows;                 // output rows per tile of the tiled kernel (launcher)
  AxisDiv div_y, div_x;          // division by n_out - 1, m_out - 1 (set by the launcher)
};

cudaError_t launch_resample(const ResampleArgs& a, float eps, float beta, int bmode,
                            cudaStream_t stream);

}  // namespace wdweno
