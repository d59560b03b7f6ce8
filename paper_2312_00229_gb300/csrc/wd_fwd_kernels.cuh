// Kernel templates of the forward zoom: one launch per image (grid = strips x
// bands x planes) and the persistent batched form.  Instantiated per storage
// type pair in wd_fwd_*.cu so that the translation units compile in parallel.
#pragma once

#include "wd_batched.h"
#include "wd_fwd_tile.cuh"
#include "wd_fwd_tile2.cuh"

#ifndef WDWENO_FWD_MIN_BLOCKS
#define WDWENO_FWD_MIN_BLOCKS 2
#endif

namespace wdweno {
namespace fwd_kernels {

using fwd_tile::Exchange;
using fwd_tile::THREADS;
using fwd_tile::TILE_W;

// CTAs resident per SM that the register budget is sized for.
template <int NT>
constexpr int fwd_min_blocks() {
  return NT == THREADS ? WDWENO_FWD_MIN_BLOCKS : WDWENO_FWD_MIN_BLOCKS * THREADS / NT;
}

template <int BMODE, class IO, int NT>
__global__ void __launch_bounds__(NT, fwd_min_blocks<NT>())
    zoom2x_fwd_kernel(FwdArgs a, MethodConsts k) {
  __shared__ fwd_tile::ExchangeT<NT> ex;
  fwd_tile::zoom2x_fwd_tile<BMODE, IO, NT>(a, k, ex, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Two coarse columns per thread (wd_fwd_tile2.cuh): 2 NT columns per CTA.
template <int BMODE, class IO, int NT>
__global__ void __launch_bounds__(NT, 3 * 128 / NT)
    zoom2x_fwd_kernel2(FwdArgs a, MethodConsts k) {
  __shared__ fwd_tile::Exchange2<NT> ex;
  fwd_tile::zoom2x_fwd_tile2<BMODE, IO, NT>(a, k, ex, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int BMODE, class IO>
cudaError_t launch_fwd(const FwdArgs& a, const MethodConsts& k, cudaStream_t stream) {
  if (a.cols == 2) {
    const int nt = a.threads == 64 ? 64 : 128;
    const int64_t tw = 2 * nt - 10;
    dim3 grid((unsigned)((a.m + tw - 1) / tw),
              (unsigned)((a.n + a.rows_per_band - 1) / a.rows_per_band), (unsigned)a.planes);
    if (nt == 64)
      zoom2x_fwd_kernel2<BMODE, IO, 64><<<grid, nt, 0, stream>>>(a, k);
    else
      zoom2x_fwd_kernel2<BMODE, IO, 128><<<grid, nt, 0, stream>>>(a, k);
    return cudaGetLastError();
  }
  const int nt = a.threads == fwd_tile::THREADS_NARROW ? fwd_tile::THREADS_NARROW : THREADS;
  const int64_t tw = nt - 9;
  dim3 grid((unsigned)((a.m + tw - 1) / tw),
            (unsigned)((a.n + a.rows_per_band - 1) / a.rows_per_band), (unsigned)a.planes);
  if (nt == fwd_tile::THREADS_NARROW)
    zoom2x_fwd_kernel<BMODE, IO, fwd_tile::THREADS_NARROW><<<grid, nt, 0, stream>>>(a, k);
  else
    zoom2x_fwd_kernel<BMODE, IO, THREADS><<<grid, nt, 0, stream>>>(a, k);
  return cudaGetLastError();
}

}  // namespace fwd_kernels
}  // namespace wdweno
