// Fused 2^k zoom (arXiv 2312.00229, Sec. 3.3, Eq. zoomfactor): every level of
// a cascade of 2x zooms in one persistent launch.
//
// The tiles of all levels form one queue, level after level.  A CTA takes the
// next tile; a tile of level L >= 1 first waits until the bands of level L-1
// that hold its input rows (with the sweep's 4-before / 5-after halo) are
// finished in every strip, then runs the forward tile body of the one-level
// kernel.  Tiles are taken in queue order, so every tile a CTA waits for was
// taken earlier by a CTA that is running, and that tile waits only for tiles
// taken before it: the launch always progresses, whatever the number of CTAs
// resident.  Each wait is bounded (one second of %globaltimer); one that gives
// up is counted in weno_wait_timeouts and the tile runs on.
//
// Level L's input is the FP32 image level L-1 wrote in this launch; it is read
// through L2 (ld.global.cg): the read-only cache could hold a stale line with
// the edge of a band that was finished after this SM read its neighbour.
// Finished tiles are published with a fence by every thread, a barrier and a
// release increment by thread 0; waits use acquire loads.
#include <type_traits>

#include "wd_cascade.h"
#include "wd_fwd_kernels.cuh"

namespace wdweno {

namespace {

constexpr int THREADS = CASCADE_THREADS;
using Exchange = fwd_tile::ExchangeT<THREADS>;

constexpr unsigned long long WAIT_NS = 1000000000ull;
constexpr int SETUP_THREADS = 256;

// Storage access of one cascade level, types fixed at compile time: FP32
// input (written earlier in this launch) is read through L2, the caller's
// input of other types through the read-only path.
template <class TIn, class TOut>
struct CascadeIO {
  __device__ __forceinline__ static uint32_t load_bits(const void* base, int64_t idx, int) {
    if constexpr (std::is_same<TIn, float>::value)
      return __float_as_uint(__ldcg(static_cast<const float*>(base) + idx));
    else
      return load_elem_bits(base, idx, DTypeOf<TIn>::value);
  }
  __device__ __forceinline__ static float value(uint32_t b, int) {
    return elem_bits_value(b, DTypeOf<TIn>::value);
  }
  __device__ __forceinline__ static void store1(void* out, int64_t idx, float v, int, int clampf) {
    store_typed<TOut>(out, idx, v, clampf);
  }
  __device__ __forceinline__ static void store2(void* out, int64_t idx, float v0, float v1, int,
                                                int clampf) {
    store2_typed<TOut>(out, idx, v0, v1, clampf);
  }
};

// Any storage pair, types chosen at run time.
struct CascadeDynIO {
  __device__ __forceinline__ static uint32_t load_bits(const void* base, int64_t idx, int dt) {
    if (dt == DT_F32) return __float_as_uint(__ldcg(static_cast<const float*>(base) + idx));
    return load_elem_bits(base, idx, dt);
  }
  __device__ __forceinline__ static float value(uint32_t b, int dt) {
    return elem_bits_value(b, dt);
  }
  __device__ __forceinline__ static void store1(void* out, int64_t idx, float v, int dt,
                                                int clampf) {
    store_elem(out, idx, v, dt, clampf);
  }
  __device__ __forceinline__ static void store2(void* out, int64_t idx, float v0, float v1, int dt,
                                                int clampf) {
    store2_vec(out, idx, v0, v1, dt, clampf);
  }
};

// One tile of a level, compiled as a function of its own so that its
// registers are allocated apart from the persistent loop and the other
// levels' bodies.
template <int BMODE, class IO>
__device__ __noinline__ void level_tile(const FwdArgs& f, const MethodConsts& k, Exchange& ex,
                                        int64_t strip, int64_t band, int64_t plane) {
  fwd_tile::zoom2x_fwd_tile<BMODE, IO, THREADS>(f, k, ex, strip, band, plane);
}

// The tile body of level L with the storage types of its position in the
// chain: TIn -> FP32 first, FP32 -> FP32 between, FP32 -> TOut last
// (TIn -> TOut for a single level).  One body per position measured faster
// than one body with run-time storage branches (234 against 247 us for the
// 8x cascade), although it spills more registers.
template <int BMODE, class TIn, class TOut>
struct LevelTypes {
  __device__ __forceinline__ static void run(const CascadeArgs& c, int L, Exchange& ex,
                                             int64_t strip, int64_t band, int64_t plane) {
    const FwdArgs& f = c.f[L];
    const bool first = L == 0, last = L == c.levels - 1;
    if (first && last)
      level_tile<BMODE, CascadeIO<TIn, TOut>>(f, c.k[L], ex, strip, band, plane);
    else if (first)
      level_tile<BMODE, CascadeIO<TIn, float>>(f, c.k[L], ex, strip, band, plane);
    else if (last)
      level_tile<BMODE, CascadeIO<float, TOut>>(f, c.k[L], ex, strip, band, plane);
    else
      level_tile<BMODE, CascadeIO<float, float>>(f, c.k[L], ex, strip, band, plane);
  }
};

template <int BMODE>
struct LevelDyn {
  __device__ __forceinline__ static void run(const CascadeArgs& c, int L, Exchange& ex,
                                             int64_t strip, int64_t band, int64_t plane) {
    fwd_tile::zoom2x_fwd_tile<BMODE, CascadeDynIO, THREADS>(c.f[L], c.k[L], ex, strip, band,
                                                            plane);
  }
};

__device__ __forceinline__ unsigned int load_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void add_release(unsigned int* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

// Waits (bounded) until *p >= need.
__device__ void wait_count(const unsigned int* p, unsigned int need) {
  if (load_acquire(p) >= need) return;
  const uint64_t t0 = fwd_tile::global_ns();
  for (;;) {
    __nanosleep(256);
    if (load_acquire(p) >= need) return;
    if (fwd_tile::global_ns() - t0 > WAIT_NS) {
      atomicAdd(&fwd_tile::g_wait_timeouts, 1u);
      return;
    }
  }
}

__global__ void __launch_bounds__(SETUP_THREADS)
    cascade_setup_kernel(unsigned long long* head, unsigned int* done, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * SETUP_THREADS + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * SETUP_THREADS)
    done[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *head = 0ULL;
}

template <class LEVEL>
__global__ void __launch_bounds__(THREADS, fwd_kernels::fwd_min_blocks<THREADS>())
    cascade_fwd_kernel(const __grid_constant__ CascadeArgs c) {
  __shared__ Exchange ex;
  __shared__ long long s_item;
  const long long total = c.first[c.levels];
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(c.head, 1ULL);
    __syncthreads();
    const long long item = s_item;
    __syncthreads();  // s_item is rewritten only after everyone read it
    if (item >= total) break;
    int L = 0;
    while (L + 1 < c.levels && item >= c.first[L + 1]) ++L;
    const FwdArgs& f = c.f[L];
    // 32-bit decode: a level has far fewer than 2^31 tiles (its bands are
    // limited to 65535 and its planes to 65535 on the host)
    const int strips = (int)c.strips[L], planes = (int)f.planes;
    const int local = (int)(item - c.first[L]);
    const int strip = local % strips;
    const int bp = local / strips;
    const int plane = bp % planes, band = bp / planes;
    if (L > 0 && threadIdx.x == 0) {
      // input rows of the band's sweep (clamped), and the level L-1 bands
      // whose output rows they are (a band of Hp coarse rows writes 2 Hp rows)
      const int64_t H = f.rows_per_band, a0 = (int64_t)band * H;
      const int64_t lo = a0 - 4 > 0 ? a0 - 4 : 0;
      const int64_t hi = a0 + H + 5 < f.n - 1 ? a0 + H + 5 : f.n - 1;
      const int64_t hp2 = 2 * c.f[L - 1].rows_per_band;
      const unsigned int need = (unsigned int)c.strips[L - 1];
      for (int64_t b = lo / hp2; b <= hi / hp2; ++b)
        wait_count(c.done + c.done_off[L - 1] + b * planes + plane, need);
    }
    __syncthreads();
    LEVEL::run(c, L, ex, strip, band, plane);
    __threadfence();  // this thread's outputs before the tile is published
    __syncthreads();
    if (threadIdx.x == 0) add_release(c.done + c.done_off[L] + (int64_t)band * planes + plane);
  }
}

int cascade_grid(const void* kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, THREADS, 0) != cudaSuccess)
    return 0;
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <class LEVEL>
cudaError_t launch_levels(const CascadeArgs& c, cudaStream_t stream) {
  const int blocks = (int)((c.done_count + SETUP_THREADS - 1) / SETUP_THREADS);
  cascade_setup_kernel<<<blocks < 1 ? 1 : (blocks > 64 ? 64 : blocks), SETUP_THREADS, 0,
                         stream>>>(c.head, c.done, c.done_count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int grid = cascade_grid((const void*)cascade_fwd_kernel<LEVEL>);
  if (grid <= 0) return cudaErrorInvalidValue;
  cascade_fwd_kernel<LEVEL><<<grid, THREADS, 0, stream>>>(c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_zoom2x_cascade(const CascadeArgs& c, int bmode, int in_t, int out_t,
                                  cudaStream_t stream) {
  if (bmode == B2R || bmode == B2) {
    const bool r = bmode == B2R;
    if (in_t == DT_U8 && out_t == DT_U8)
      return r ? launch_levels<LevelTypes<B2R, uint8_t, uint8_t>>(c, stream)
               : launch_levels<LevelTypes<B2, uint8_t, uint8_t>>(c, stream);
    if (in_t == DT_F32 && out_t == DT_F32)
      return r ? launch_levels<LevelTypes<B2R, float, float>>(c, stream)
               : launch_levels<LevelTypes<B2, float, float>>(c, stream);
    if (in_t == DT_F16 && out_t == DT_F16)
      return r ? launch_levels<LevelTypes<B2R, __half, __half>>(c, stream)
               : launch_levels<LevelTypes<B2, __half, __half>>(c, stream);
    return r ? launch_levels<LevelDyn<B2R>>(c, stream) : launch_levels<LevelDyn<B2>>(c, stream);
  }
  if (bmode == B0) return launch_levels<LevelDyn<B0>>(c, stream);
  return launch_levels<LevelDyn<BGEN>>(c, stream);
}

cudaError_t fwd_wait_timeouts_cascade(unsigned int* count, bool reset) {
  return fwd_tile::read_wait_timeouts(count, reset);
}

}  // namespace wdweno
