// Internal launch interface of the adjoint (backward) kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "wd_common.cuh"

namespace wdweno {

constexpr int BWD_GHOST = 2;  // extension cells per side of the workspace grid

struct BwdArgs {
  const float* x;
  const float* gout;
  float* gin;
  int64_t n, m, planes;
  int64_t x_sc, x_sh, x_sw;
  int64_t g_sc, g_sh, g_sw;
  int64_t gi_sc, gi_sh, gi_sw;
  int64_t orows, ocols;
  float* ws;  // 2 * (n + 2 BWD_GHOST) * (m + 2 BWD_GHOST) * planes floats
};

size_t bwd_workspace_bytes(int64_t n, int64_t m, int64_t planes);
cudaError_t launch_zoom2x_bwd(const BwdArgs& a, const MethodConsts& k, int bmode,
                              cudaStream_t stream);

}  // namespace wdweno
