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

void fwd_shape_for(int64_t m, int* threads, int* cols) {
  // Column-steps a launch spends across the width: strips x columns per
  // strip, a two-column column counted 0.9 of a one-column one (it issues
  // about 16% fewer instructions per column; measured 4-9% faster on wide
  // images).  Ties go to the earlier entry.
  struct Shape { int threads, cols; double weight; };
  const Shape shapes[4] = {{128, 2, 0.9}, {64, 2, 0.9}, {fwd_tile::THREADS, 1, 1.0},
                           {fwd_tile::THREADS_NARROW, 1, 1.0}};
  double best = 1e300;
  for (const Shape& s : shapes) {
    const int64_t span = (int64_t)s.threads * s.cols;  // columns of one CTA
    const int64_t tw = s.cols == 2 ? span - 10 : span - 9;
    const double cost = double((m + tw - 1) / tw) * double(span) * s.weight;
    if (cost < best - 1e-9) {
      best = cost;
      *threads = s.threads;
      *cols = s.cols;
    }
  }
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
