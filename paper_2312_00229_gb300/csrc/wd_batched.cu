// Batched forward 2x zoom: many images of independent sizes in persistent
// launches fed by device-side tile queues.
//
// The images fall in two classes by input path: 1- and 2-byte storage with
// unit column stride takes bulk row copies (class 0), anything else register
// loads (class 1).  Each class has its own queue and persistent kernel; one
// kernel holding both paths spills.  For 1- and 2-byte storage both kernels
// are launched (class 1 is usually empty and exits at once); for FP32 only
// the register kernel.
//
// Workspace (caller-owned, no initialisation needed):
//   [0]   unsigned long long  head[2], next tile of each class
//   [16]  unsigned long long  total[2], tiles of each class
//   [32]  unsigned long long  prefix[2][count + 1], per class the exclusive
//                             prefix sum of the tiles of each image (0 for an
//                             image of the other class or a malformed one)
// The setup kernel fills it from the device-resident descriptors, so a
// stream capture of the call replays correctly with new pixel data.
#include "wd_batched.h"
#include "wd_fwd_kernels.cuh"

namespace wdweno {

namespace {

using fwd_tile::Exchange;
using fwd_tile::THREADS;
using fwd_tile::TILE_W;

constexpr int SETUP_THREADS = 1024;

struct Queue {
  unsigned long long head[2];
  unsigned long long total[2];
  unsigned long long prefix[1];  // 2 (count + 1) entries
};


__host__ __device__ __forceinline__ int64_t dsize(int dt) {
  return dt == DT_U8 ? 1 : (dt == DT_F32 ? 4 : 2);
}

// Input-path class of an image: 0 = bulk row copies, 1 = register loads.
__device__ __forceinline__ int image_class(const weno_image& in, int in_dtype) {
  return dsize(in_dtype) <= 2 && in.stride_w == 1 ? 0 : 1;
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

__device__ unsigned long long image_tiles(const weno_image& in, int64_t rpb) {
  const unsigned long long strips = (in.width + TILE_W - 1) / TILE_W;
  const unsigned long long bands = (in.height + rpb - 1) / rpb;
  return strips * bands * (unsigned long long)in.channels;
}

__global__ void __launch_bounds__(SETUP_THREADS) batched_setup_kernel(BatchedArgs a) {
  Queue* q = static_cast<Queue*>(a.workspace);
  __shared__ unsigned long long part[2][SETUP_THREADS];
  const int t = threadIdx.x;
  const int chunk = (a.count + SETUP_THREADS - 1) / SETUP_THREADS;
  const int lo = min(a.count, t * chunk), hi = min(a.count, lo + chunk);
  unsigned long long sum0 = 0ULL, sum1 = 0ULL;
  for (int i = lo; i < hi; ++i) {
    const weno_image in = a.in[i], out = a.out[i];
    if (!descriptor_ok(in, out, a.out_mode)) continue;
    const unsigned long long n = image_tiles(in, a.rows_per_band);
    if (image_class(in, a.in_dtype) == 0) sum0 += n; else sum1 += n;
  }
  part[0][t] = sum0;
  part[1][t] = sum1;
  __syncthreads();
  // Inclusive Hillis-Steele scans of the per-thread sums of both classes.
  for (int off = 1; off < SETUP_THREADS; off <<= 1) {
    const unsigned long long v0 = t >= off ? part[0][t - off] : 0ULL;
    const unsigned long long v1 = t >= off ? part[1][t - off] : 0ULL;
    __syncthreads();
    part[0][t] += v0;
    part[1][t] += v1;
    __syncthreads();
  }
  unsigned long long* pre0 = q->prefix;
  unsigned long long* pre1 = q->prefix + (a.count + 1);
  unsigned long long run0 = part[0][t] - sum0, run1 = part[1][t] - sum1;  // exclusive starts
  for (int i = lo; i < hi; ++i) {
    pre0[i] = run0;
    pre1[i] = run1;
    const weno_image in = a.in[i], out = a.out[i];
    if (!descriptor_ok(in, out, a.out_mode)) continue;
    const unsigned long long n = image_tiles(in, a.rows_per_band);
    if (image_class(in, a.in_dtype) == 0) run0 += n; else run1 += n;
  }
  if (t == SETUP_THREADS - 1) {
    pre0[a.count] = part[0][t];
    pre1[a.count] = part[1][t];
    q->total[0] = part[0][t];
    q->total[1] = part[1][t];
    q->head[0] = q->head[1] = 0ULL;
  }
}

// CLS: the image class this kernel serves (0: bulk copies, 1: registers).
template <int BMODE, class IO, int CLS>
__global__ void __launch_bounds__(THREADS, WDWENO_FWD_MIN_BLOCKS)
    batched_fwd_kernel(BatchedArgs a, MethodConsts k) {
  __shared__ Exchange ex;
  __shared__ unsigned long long s_tile;
  __shared__ int s_img;
  Queue* q = static_cast<Queue*>(a.workspace);
  const unsigned long long total = q->total[CLS];
  const unsigned long long* prefix = q->prefix + CLS * (a.count + 1);
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long tile = atomicAdd(&q->head[CLS], 1ULL);
      int img = -1;
      if (tile < total) {
        // largest i with prefix[i] <= tile < prefix[i + 1] (images of the
        // other class have no tiles here and are skipped by "largest")
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
    const unsigned long long strips = (f.m + TILE_W - 1) / TILE_W;
    const unsigned long long bands = (f.n + f.rows_per_band - 1) / f.rows_per_band;
    const unsigned long long per_plane = strips * bands;
    const int64_t plane = (int64_t)(local / per_plane);
    const unsigned long long rem = local % per_plane;
    constexpr int INB = CLS == 0 ? fwd_tile::IN_BULK_ANY : fwd_tile::IN_REG;
    f.in_bulk = INB;
    fwd_tile::zoom2x_fwd_tile<BMODE, IO, INB>(f, k, ex, (int64_t)(rem % strips),
                                              (int64_t)(rem / strips), plane);
  }
}

int persistent_grid(const void* kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, THREADS, 0) != cudaSuccess)
    return 0;
  return sms * (per_sm > 0 ? per_sm : 1);
}

}  // namespace

size_t batched_workspace_bytes(int count) {
  size_t b = 32 + 16 * (size_t(count) + 1);
  return (b + 15) & ~size_t(15);
}

template <int BMODE, class IO, int CLS>
cudaError_t launch_class(const BatchedArgs& a, const MethodConsts& k, cudaStream_t stream) {
  const int grid = persistent_grid((const void*)batched_fwd_kernel<BMODE, IO, CLS>);
  if (grid <= 0) return cudaErrorInvalidValue;
  batched_fwd_kernel<BMODE, IO, CLS><<<grid, THREADS, 0, stream>>>(a, k);
  return cudaGetLastError();
}

template <int BMODE, class IO>
cudaError_t launch_persistent(const BatchedArgs& a, const MethodConsts& k, cudaStream_t stream) {
  if (dsize(a.in_dtype) <= 2) {
    const cudaError_t e = launch_class<BMODE, IO, 0>(a, k, stream);
    if (e != cudaSuccess) return e;
  }
  return launch_class<BMODE, IO, 1>(a, k, stream);
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
