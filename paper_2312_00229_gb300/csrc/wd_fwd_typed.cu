// Forward kernels with the storage types fixed at compile time (beta = 2):
// the same-type pairs and the uint8 <-> FP32 pairs of a cascade, and the
// direct 1/D^2 weights (B2R) for the common pairs, used when the data are
// bounded (by the input type or by the caller's weno_params::data_bound).
#include "wd_fwd_kernels.cuh"

namespace wdweno {

// The direct 1/D^2 weights (B2R) are in wd_fwd_typed_b2r.cu (compiled in
// parallel).
cudaError_t launch_fwd_typed_b2r(const FwdArgs& a, const MethodConsts& k, cudaStream_t stream,
                                 bool* handled);

cudaError_t launch_fwd_typed(const FwdArgs& a, const MethodConsts& k, int bmode,
                             cudaStream_t stream, bool* handled) {
  using fwd_kernels::launch_fwd;
  using fwd_tile::TypedIO;
  *handled = true;
  const int i = a.in_dtype, o = a.out_dtype;
  if (bmode == B2R) return launch_fwd_typed_b2r(a, k, stream, handled);
  if (i == DT_U8 && o == DT_U8) return launch_fwd<B2, TypedIO<uint8_t, uint8_t>>(a, k, stream);
  if (i == DT_F16 && o == DT_F16) return launch_fwd<B2, TypedIO<__half, __half>>(a, k, stream);
  if (i == DT_BF16 && o == DT_BF16)
    return launch_fwd<B2, TypedIO<__nv_bfloat16, __nv_bfloat16>>(a, k, stream);
  if (i == DT_F32 && o == DT_F32) return launch_fwd<B2, TypedIO<float, float>>(a, k, stream);
  if (i == DT_U8 && o == DT_F32) return launch_fwd<B2, TypedIO<uint8_t, float>>(a, k, stream);
  if (i == DT_F32 && o == DT_U8) return launch_fwd<B2, TypedIO<float, uint8_t>>(a, k, stream);
  *handled = false;
  return cudaSuccess;
}

cudaError_t fwd_wait_timeouts_typed(unsigned int* count, bool reset) {
  return fwd_tile::read_wait_timeouts(count, reset);
}

}  // namespace wdweno
