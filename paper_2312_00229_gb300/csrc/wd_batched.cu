// Batched forward 2x zoom: many images of independent sizes in one
// persistent launch fed by a device-side tile queue.
//
// Workspace (caller-owned, no initialisation needed):
//   [0]   unsigned long long  head, next tile
//   [8]   unsigned long long  total, tiles of all images
//   [16]  unsigned long long  prefix[count + 1], the exclusive prefix sum of
//                             the tiles of each image (a malformed image has
//                             none)
// The setup kernel fills it from the device-resident descriptors, so a
// stream capture of the call replays correctly with new pixel data.  The
// persistent kernel is in wd_batched_kernel.cuh; this unit instantiates it
// with one coarse column per thread, wd_batched2.cu with two.
#include "wd_batched_kernel.cuh"

namespace wdweno {

cudaError_t launch_batched_paired(const BatchedArgs& a, const MethodConsts& k, int bmode,
                                  cudaStream_t stream);

namespace {

using batched::Queue;
using batched::strip_width;

constexpr int SETUP_THREADS = 1024;

__device__ bool descriptor_ok(const weno_image& in, const weno_image& out, int out_mode) {
  if (!in.data || !out.data) return false;
  if (in.height < 1 || in.width < 1 || in.channels < 1 || in.channels >= 65536) return false;
  if (in.height >= (int64_t(1) << 31) || in.width >= (int64_t(1) << 31)) return false;
  if (in.stride_c < 1 || in.stride_h < 1 || in.stride_w < 1) return false;
  if (out.stride_c < 1 || out.stride_h < 1 || out.stride_w < 1) return false;
  const int64_t d = out_mode == WENO_OUT_2N_MINUS_1 ? 1 : 0;
  return out.height == 2 * in.height - d && out.width == 2 * in.width - d &&
         out.channels == in.channels;
}

// Tiles of one image for CTAs of `threads` x `cols` columns.
__device__ unsigned long long image_tiles(const weno_image& in, int64_t rpb, int threads,
                                          int cols) {
  const unsigned long long tw = (unsigned long long)strip_width(threads, cols);
  const unsigned long long strips = (in.width + tw - 1) / tw;
  const unsigned long long bands = (in.height + rpb - 1) / rpb;
  return strips * bands * (unsigned long long)in.channels;
}

__global__ void __launch_bounds__(SETUP_THREADS) batched_setup_kernel(BatchedArgs a) {
  Queue* q = static_cast<Queue*>(a.workspace);
  __shared__ unsigned long long part[SETUP_THREADS];
  const int t = threadIdx.x;
  const int chunk = (a.count + SETUP_THREADS - 1) / SETUP_THREADS;
  const int lo = min(a.count, t * chunk), hi = min(a.count, lo + chunk);
  unsigned long long sum = 0ULL;
  for (int i = lo; i < hi; ++i) {
    const weno_image in = a.in[i], out = a.out[i];
    if (descriptor_ok(in, out, a.out_mode))
      sum += image_tiles(in, a.rows_per_band, a.threads, a.cols);
  }
  part[t] = sum;
  __syncthreads();
  // Inclusive Hillis-Steele scan of the per-thread sums.
  for (int off = 1; off < SETUP_THREADS; off <<= 1) {
    const unsigned long long v = t >= off ? part[t - off] : 0ULL;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned long long run = part[t] - sum;  // exclusive start
  for (int i = lo; i < hi; ++i) {
    q->prefix[i] = run;
    const weno_image in = a.in[i], out = a.out[i];
    if (descriptor_ok(in, out, a.out_mode))
      run += image_tiles(in, a.rows_per_band, a.threads, a.cols);
  }
  if (t == SETUP_THREADS - 1) {
    q->prefix[a.count] = part[t];
    q->total = part[t];
    q->head = 0ULL;
  }
}

}  // namespace

size_t batched_workspace_bytes(int count) {
  size_t b = 16 + 8 * (size_t(count) + 1);
  return (b + 15) & ~size_t(15);
}

cudaError_t launch_zoom2x_batched(const BatchedArgs& a, const MethodConsts& k, int bmode,
                                  cudaStream_t stream) {
  batched_setup_kernel<<<1, SETUP_THREADS, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.cols == 2) return launch_batched_paired(a, k, bmode, stream);
  return batched::launch_typed<1>(a, k, bmode, stream);
}

cudaError_t fwd_wait_timeouts_batched(unsigned int* count, bool reset) {
  return fwd_tile::read_wait_timeouts(count, reset);
}

}  // namespace wdweno
