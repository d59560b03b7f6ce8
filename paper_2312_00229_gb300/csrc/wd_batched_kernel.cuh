// Kernel template of the persistent batched forward zoom, shared by the
// translation units that instantiate it (wd_batched.cu: one coarse column
// per thread; wd_batched2.cu: two), which compile in parallel.
#pragma once

#include <type_traits>

#include "wd_batched.h"
#include "wd_fwd_kernels.cuh"

namespace wdweno {
namespace batched {

using fwd_tile::THREADS;
using fwd_tile::THREADS_NARROW;

struct Queue {
  unsigned long long head;
  unsigned long long total;
  unsigned long long prefix[1];  // count + 1 entries
};

__host__ __device__ __forceinline__ int64_t dsize(int dt) {
  return dt == DT_U8 ? 1 : (dt == DT_F32 ? 4 : 2);
}

// Output columns of a strip: threads - 9 with one column per thread,
// 2 threads - 10 with two.
constexpr __host__ __device__ int strip_width(int threads, int cols) {
  return cols == 2 ? 2 * threads - 10 : threads - 9;
}

template <int NT, int COLS>
struct BatchedShape {
  using Ex = typename std::conditional<COLS == 2, fwd_tile::Exchange2<NT>,
                                       fwd_tile::ExchangeT<NT>>::type;
  static constexpr int MIN_BLOCKS = COLS == 2 ? 3 * 128 / NT : fwd_kernels::fwd_min_blocks<NT>();
};

template <int BMODE, class IO, int NT, int COLS>
__global__ void __launch_bounds__(NT, (BatchedShape<NT, COLS>::MIN_BLOCKS))
    batched_fwd_kernel(BatchedArgs a, MethodConsts k) {
  __shared__ typename BatchedShape<NT, COLS>::Ex ex;
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
    f.out_vec4 = out.stride_w == 1 && out.stride_h % 4 == 0 && out.stride_c % 4 == 0 &&
                 base % uintptr_t(4 * dsize(a.out_dtype)) == 0;
    const unsigned long long local = tile - prefix[img];
    constexpr unsigned long long tw = strip_width(NT, COLS);
    const unsigned long long strips = (f.m + tw - 1) / tw;
    const unsigned long long bands = (f.n + f.rows_per_band - 1) / f.rows_per_band;
    const unsigned long long per_plane = strips * bands;
    const int64_t plane = (int64_t)(local / per_plane);
    const unsigned long long rem = local % per_plane;
    if constexpr (COLS == 2)
      fwd_tile::zoom2x_fwd_tile2<BMODE, IO, NT>(f, k, ex, (int64_t)(rem % strips),
                                                (int64_t)(rem / strips), plane);
    else
      fwd_tile::zoom2x_fwd_tile<BMODE, IO, NT>(f, k, ex, (int64_t)(rem % strips),
                                               (int64_t)(rem / strips), plane);
  }
}

inline int persistent_grid(const void* kernel, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
    return 0;
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <int BMODE, class IO, int NT, int COLS>
cudaError_t launch_width(const BatchedArgs& a, const MethodConsts& k, cudaStream_t stream) {
  const int grid = persistent_grid((const void*)batched_fwd_kernel<BMODE, IO, NT, COLS>, NT);
  if (grid <= 0) return cudaErrorInvalidValue;
  batched_fwd_kernel<BMODE, IO, NT, COLS><<<grid, NT, 0, stream>>>(a, k);
  return cudaGetLastError();
}

// The persistent launch for the storage types and weight form of `a`, with
// CTAs of COLS coarse columns per thread.
template <int COLS>
cudaError_t launch_typed(const BatchedArgs& a, const MethodConsts& k, int bmode,
                         cudaStream_t stream) {
  using fwd_tile::DynIO;
  using fwd_tile::TypedIO;
  auto go = [&](auto bm, auto io) -> cudaError_t {
    constexpr int BM = decltype(bm)::value;
    using IO = decltype(io);
    if constexpr (COLS == 2) {
      if (a.threads == 64) return launch_width<BM, IO, 64, 2>(a, k, stream);
      return launch_width<BM, IO, 128, 2>(a, k, stream);
    } else {
      if (a.threads == THREADS_NARROW)
        return launch_width<BM, IO, THREADS_NARROW, 1>(a, k, stream);
      return launch_width<BM, IO, THREADS, 1>(a, k, stream);
    }
  };
  using C2R = std::integral_constant<int, B2R>;
  using C2 = std::integral_constant<int, B2>;
  using C0 = std::integral_constant<int, B0>;
  using CG = std::integral_constant<int, BGEN>;
  if (bmode == B2R) {  // data bounded by the storage type or the caller's bound
    if (a.in_dtype == DT_U8 && a.out_dtype == DT_U8) return go(C2R(), TypedIO<uint8_t, uint8_t>());
    if (a.in_dtype == DT_F16 && a.out_dtype == DT_F16) return go(C2R(), TypedIO<__half, __half>());
    if (a.in_dtype == DT_F32 && a.out_dtype == DT_F32) return go(C2R(), TypedIO<float, float>());
    return go(C2R(), DynIO());
  }
  if (bmode == B2 && a.in_dtype == a.out_dtype) {
    switch (a.in_dtype) {
      case DT_U8: return go(C2(), TypedIO<uint8_t, uint8_t>());
      case DT_F16: return go(C2(), TypedIO<__half, __half>());
      case DT_BF16: return go(C2(), TypedIO<__nv_bfloat16, __nv_bfloat16>());
      default: return go(C2(), TypedIO<float, float>());
    }
  }
  if (bmode == B2) return go(C2(), DynIO());
  if (bmode == B0) return go(C0(), DynIO());
  return go(CG(), DynIO());
}

}  // namespace batched
}  // namespace wdweno
