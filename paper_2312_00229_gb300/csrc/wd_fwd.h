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
  int in_bulk;                   // input path: 0 registers, 1 or 2 bulk copies (input_bulk_ok)
};

// Which input path the forward kernel takes (fwd_tile::InputPath): bulk
// copies for 1- and 2-byte storage with unit column stride; the constant-window
// form (1) when the base, row and plane strides and the row length are
// multiples of 16 bytes, the per-row form (2) otherwise; register loads (0)
// for FP32 (measured faster) and strided columns.
__host__ __device__ inline int input_bulk_ok(const void* base, int64_t esz, int64_t m,
                                             int64_t planes, int64_t sc, int64_t sh, int64_t sw) {
  if (esz > 2 || sw != 1) return 0;
  const bool aligned = (reinterpret_cast<uintptr_t>(base) % 16) == 0 && (sh * esz) % 16 == 0 &&
                       (planes == 1 || (sc * esz) % 16 == 0) && (m * esz) % 16 == 0;
  return aligned ? 1 : 2;
}

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
