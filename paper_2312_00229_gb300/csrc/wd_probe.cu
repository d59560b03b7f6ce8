// FP32-pipe calibration kernel: the measured counterpart of the nominal
// FP32 issue peak (SMs x 128 lanes x clock) that the forward pass's
// roofline divides by.  Each thread runs 16 independent chains of FP32
// fused multiply-adds, enough independent work per warp to cover the
// pipe's latency, and stores the chains' sum so that nothing is removed.
#include <cuda_runtime.h>

#include "wdweno.h"

namespace wdweno {
namespace {

constexpr int CHAINS = 16;

__global__ void __launch_bounds__(256) k_fp32_probe(int iters, float a, float b, float* out) {
  float x[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) x[j] = (float)threadIdx.x * 1e-3f + (float)j;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) x[j] = fmaf(x[j], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += x[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace wdweno

// Largest accepted blocks and iters (the operation count stays below 2^63).
constexpr int kProbeMax = 1 << 23;

extern "C" int weno_fp32_probe(int blocks, int iters, float* out, void* stream) {
  if (blocks < 1 || iters < 1 || blocks > kProbeMax || iters > kProbeMax || !out)
    return WENO_EINVAL;
  wdweno::k_fp32_probe<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      iters, 0.999999f, 1e-6f, out);
  return cudaGetLastError() == cudaSuccess ? WENO_OK : WENO_ECUDA;
}

extern "C" long long weno_fp32_probe_ops(int blocks, int iters) {
  if (blocks < 1 || iters < 1 || blocks > kProbeMax || iters > kProbeMax) return -1;
  return (long long)blocks * 256 * iters * 8 * wdweno::CHAINS;
}
