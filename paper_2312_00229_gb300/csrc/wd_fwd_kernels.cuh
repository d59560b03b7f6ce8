// Kernel templates of the forward zoom: one launch per image (grid = strips x
// bands x planes) and the persistent batched form.  Instantiated per storage
// type pair in wd_fwd_*.cu so that the translation units compile in parallel.
#pragma once

#include "wd_batched.h"
#include "wd_fwd_tile.cuh"

#ifndef WDWENO_FWD_MIN_BLOCKS
#define WDWENO_FWD_MIN_BLOCKS 2
#endif

namespace wdweno {
namespace fwd_kernels {

using fwd_tile::Exchange;
using fwd_tile::THREADS;
using fwd_tile::TILE_W;

template <int BMODE, class IO>
__global__ void __launch_bounds__(THREADS, WDWENO_FWD_MIN_BLOCKS)
    zoom2x_fwd_kernel(FwdArgs a, MethodConsts k) {
  __shared__ Exchange ex;
  fwd_tile::zoom2x_fwd_tile<BMODE, IO>(a, k, ex, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int BMODE, class IO>
cudaError_t launch_fwd(const FwdArgs& a, const MethodConsts& k, cudaStream_t stream) {
  dim3 grid((unsigned)((a.m + TILE_W - 1) / TILE_W),
            (unsigned)((a.n + a.rows_per_band - 1) / a.rows_per_band), (unsigned)a.planes);
  zoom2x_fwd_kernel<BMODE, IO><<<grid, THREADS, 0, stream>>>(a, k);
  return cudaGetLastError();
}

}  // namespace fwd_kernels
}  // namespace wdweno
