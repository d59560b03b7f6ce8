// Forward 2x zoom, one launch per image (all planes): grid = strips x bands x
// planes, one CTA per tile.  The tile body is in wd_fwd_tile.cuh.  Storage
// types are compile-time parameters for the common pairs (wd_fwd_typed.cu);
// any other pair, and beta != 2, goes through the run-time-typed kernels here.
#include "wd_cascade.h"
#include "wd_fwd_kernels.cuh"

namespace wdweno {

cudaError_t launch_fwd_typed(const FwdArgs& a, const MethodConsts& k, int bmode,
                             cudaStream_t stream, bool* handled);

int tile_width_fwd() { return fwd_tile::TILE_W; }
int threads_fwd() { return fwd_tile::THREADS; }

int fwd_threads_for(int64_t m) {
  const int64_t tw = fwd_tile::TILE_W, tn = fwd_tile::THREADS_NARROW - 9;
  const int64_t wide = (m + tw - 1) / tw * fwd_tile::THREADS;
  const int64_t narrow = (m + tn - 1) / tn * fwd_tile::THREADS_NARROW;
  return narrow <= wide ? fwd_tile::THREADS_NARROW : fwd_tile::THREADS;
}

cudaError_t launch_zoom2x_fwd(const FwdArgs& a, const MethodConsts& k, int bmode,
                              cudaStream_t stream) {
  using fwd_tile::DynIO;
  if (bmode == B2 || bmode == B2R) {
    bool handled = false;
    cudaError_t e = launch_fwd_typed(a, k, bmode, stream, &handled);
    if (handled) return e;
    if (bmode == B2R) return fwd_kernels::launch_fwd<B2R, DynIO>(a, k, stream);
    return fwd_kernels::launch_fwd<B2, DynIO>(a, k, stream);
  }
  if (bmode == B0) return fwd_kernels::launch_fwd<B0, DynIO>(a, k, stream);
  return fwd_kernels::launch_fwd<BGEN, DynIO>(a, k, stream);
}

cudaError_t fwd_wait_timeouts(unsigned int* count, bool reset) {
  unsigned int a = 0, b = 0, c = 0, d = 0;
  cudaError_t e = fwd_tile::read_wait_timeouts(&a, reset);
  if (e == cudaSuccess) e = fwd_wait_timeouts_typed(&b, reset);
  if (e == cudaSuccess) e = fwd_wait_timeouts_batched(&c, reset);
  if (e == cudaSuccess) e = fwd_wait_timeouts_cascade(&d, reset);
  *count = a + b + c + d;
  return e;
}

}  // namespace wdweno
