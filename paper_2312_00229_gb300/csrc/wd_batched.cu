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
// stream capture of the call replays correctly with new pixel data.
#include "wd_batched.h"
#include "wd_fwd_kernels.cuh"

namespace wdweno {

namespace {

using fwd_tile::THREADS;
using fwd_tile::THREADS_NARROW;

constexpr int SETUP_THREADS = 1024;

struct Queue {
  unsigned long long head;
  unsigned long long total;
  unsigned long long prefix[1];  // count + 1 entries
};


__host__ __device__ __forceinline__ int64_t dsize(int dt) {
  return dt == DT_U8 ? 1 : (dt == DT_F32 ? 4 : 2);
}

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

// Tiles of one image for CTAs `threads` wide (threads - 9 output columns).
__device__ unsigned long long image_tiles(const weno_image& in, int64_t rpb, int threads) {
  const unsigned long long tw = (unsigned long long)(threads - 9);
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
    if (descriptor_ok(in, out, a.out_mode)) sum += image_tiles(in, a.rows_per_band, a.threads);
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
    if (descriptor_ok(in, out, a.out_mode)) run += image_tiles(in, a.rows_per_band, a.threads);
  }
  if (t == SETUP_THREADS - 1) {
    q->prefix[a.count] = part[t];
    q->total = part[t];
    q->head = 0ULL;
  }
}

template <int BMODE, class IO, int NT>
__global__ void __launch_bounds__(NT, fwd_kernels::fwd_min_blocks<NT>())
    batched_fwd_kernel(BatchedArgs a, MethodConsts k) {
  __shared__ fwd_tile::ExchangeT<NT> ex;
  __shared__ unsigned long long s_tile;
  __shared__ int s_img;
  Queue* q = static_cast<Queue*>(a.workspace);
  const unsigned long long total = q->total;
  const unsigned long long* prefix = q->prefix;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long tile = atomicAdd(&q->head, 1ULL);
      int img = -1;
      if (tile < total) {
        // largest i with prefix[i] <= tile < prefix[i + 1] (images with no
        // tiles are skipped by "largest")
        int lo = 0, hi = a.count - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (prefix[mid] <= tile) lo = mid; else hi = mid - 1;
        }
        img = lo;
      }
      s_tile = tile;
      s_img = img;
    }
    __syncthreads();
    const int img = s_img;
    const unsigned long long tile = s_tile;
    __syncthreads();  // s_tile / s_img are rewritten only after everyone read them
    if (img < 0) break;
    const weno_image in = a.in[img], out = a.out[img];
    FwdArgs f;
    f.in = in.data;
    f.out = out.data;
    f.in_dtype = a.in_dtype;
    f.out_dtype = a.out_dtype;
    f.n = in.height;
    f.m = in.width;
    f.planes = in.channels;
    f.in_sc = in.stride_c; f.in_sh = in.stride_h; f.in_sw = in.stride_w;
    f.out_sc = out.stride_c; f.out_sh = out.stride_h; f.out_sw = out.stride_w;
    f.orows = out.height;
    f.ocols = out.width;
    f.rows_per_band = a.rows_per_band;
    const uintptr_t base = reinterpret_cast<uintptr_t>(out.data);
    f.out_vec = out.stride_w == 1 && out.stride_h % 2 == 0 && out.stride_c % 2 == 0 &&
                base % uintptr_t(2 * dsize(a.out_dtype)) == 0;
    const unsigned long long local = tile - prefix[img];
    constexpr unsigned long long tw = NT - 9;
    const unsigned long long strips = (f.m + tw - 1) / tw;
    const unsigned long long bands = (f.n + f.rows_per_band - 1) / f.rows_per_band;
    const unsigned long long per_plane = strips * bands;
    const int64_t plane = (int64_t)(local / per_plane);
    const unsigned long long rem = local % per_plane;
    fwd_tile::zoom2x_fwd_tile<BMODE, IO, NT>(f, k, ex, (int64_t)(rem % strips),
                                             (int64_t)(rem / strips), plane);
  }
}

int persistent_grid(const void* kernel, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
    return 0;
  return sms * (per_sm > 0 ? per_sm : 1);
}

}  // namespace

size_t batched_workspace_bytes(int count) {
  size_t b = 16 + 8 * (size_t(count) + 1);
  return (b + 15) & ~size_t(15);
}

template <int BMODE, class IO, int NT>
cudaError_t launch_width(const BatchedArgs& a, const MethodConsts& k, cudaStream_t stream) {
  const int grid = persistent_grid((const void*)batched_fwd_kernel<BMODE, IO, NT>, NT);
  if (grid <= 0) return cudaErrorInvalidValue;
  batched_fwd_kernel<BMODE, IO, NT><<<grid, NT, 0, stream>>>(a, k);
  return cudaGetLastError();
}

template <int BMODE, class IO>
cudaError_t launch_persistent(const BatchedArgs& a, const MethodConsts& k, cudaStream_t stream) {
  if (a.threads == THREADS_NARROW) return launch_width<BMODE, IO, THREADS_NARROW>(a, k, stream);
  return launch_width<BMODE, IO, THREADS>(a, k, stream);
}

cudaError_t launch_zoom2x_batched(const BatchedArgs& a, const MethodConsts& k, int bmode,
                                  cudaStream_t stream) {
  using fwd_tile::DynIO;
  using fwd_tile::TypedIO;
  batched_setup_kernel<<<1, SETUP_THREADS, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (bmode == B2R) {  // data bounded by the storage type or the caller's bound
    if (a.in_dtype == DT_U8 && a.out_dtype == DT_U8)
      return launch_persistent<B2R, TypedIO<uint8_t, uint8_t>>(a, k, stream);
    if (a.in_dtype == DT_F16 && a.out_dtype == DT_F16)
      return launch_persistent<B2R, TypedIO<__half, __half>>(a, k, stream);
    if (a.in_dtype == DT_F32 && a.out_dtype == DT_F32)
      return launch_persistent<B2R, TypedIO<float, float>>(a, k, stream);
    return launch_persistent<B2R, DynIO>(a, k, stream);
  }
  if (bmode == B2 && a.in_dtype == a.out_dtype) {
    switch (a.in_dtype) {
      case DT_U8: return launch_persistent<B2, TypedIO<uint8_t, uint8_t>>(a, k, stream);
      case DT_F16: return launch_persistent<B2, TypedIO<__half, __half>>(a, k, stream);
      case DT_BF16:
        return launch_persistent<B2, TypedIO<__nv_bfloat16, __nv_bfloat16>>(a, k, stream);
      default: return launch_persistent<B2, TypedIO<float, float>>(a, k, stream);
    }
  }
  if (bmode == B2) return launch_persistent<B2, DynIO>(a, k, stream);
  if (bmode == B0) return launch_persistent<B0, DynIO>(a, k, stream);
  return launch_persistent<BGEN, DynIO>(a, k, stream);
}

cudaError_t fwd_wait_timeouts_batched(unsigned int* count, bool reset) {
  return fwd_tile::read_wait_timeouts(count, reset);
}

}  // namespace wdweno
