// Forward 2x zoom, one launch per image (all planes): grid = strips x bands x
// planes, one CTA per tile.  The tile body is in wd_fwd_tile.cuh.
#include "wd_fwd_tile.cuh"

namespace wdweno {

namespace {

using fwd_tile::Exchange;
using fwd_tile::THREADS;
using fwd_tile::TILE_W;

template <int BMODE>
__global__ void __launch_bounds__(THREADS, 2) zoom2x_fwd_kernel(FwdArgs a, MethodConsts k) {
  __shared__ Exchange ex;
  fwd_tile::zoom2x_fwd_tile<BMODE>(a, k, ex, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace

int tile_width_fwd() { return TILE_W; }
int threads_fwd() { return THREADS; }
cudaError_t launch_zoom2x_fwd(const FwdArgs& a, const MethodConsts& k, int bmode,
                              cudaStream_t stream) {
  dim3 grid((unsigned)((a.m + TILE_W - 1) / TILE_W),
            (unsigned)((a.n + a.rows_per_band - 1) / a.rows_per_band), (unsigned)a.planes);
  switch (bmode) {
    case B2: zoom2x_fwd_kernel<B2><<<grid, THREADS, 0, stream>>>(a, k); break;
    case B0: zoom2x_fwd_kernel<B0><<<grid, THREADS, 0, stream>>>(a, k); break;
    default: zoom2x_fwd_kernel<BGEN><<<grid, THREADS, 0, stream>>>(a, k); break;
  }
  return cudaGetLastError();
}

}  // namespace wdweno
