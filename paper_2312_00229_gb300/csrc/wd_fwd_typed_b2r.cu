// Forward kernels with the storage types fixed at compile time and the
// direct 1/D^2 weights of Eq. (alpha) at beta = 2 (B2R), used when the data
// are bounded (by the input type or by the caller's weno_params::data_bound):
// the common storage pairs.  Split from wd_fwd_typed.cu so that the two
// translation units compile in parallel.
#include "wd_fwd_kernels.cuh"

namespace wdweno {

cudaError_t launch_fwd_typed_b2r(const FwdArgs& a, const MethodConsts& k, cudaStream_t stream,
                                 bool* handled) {
  using fwd_kernels::launch_fwd;
  using fwd_tile::TypedIO;
  *handled = true;
  const int i = a.in_dtype, o = a.out_dtype;
  if (i == DT_U8 && o == DT_U8) return launch_fwd<B2R, TypedIO<uint8_t, uint8_t>>(a, k, stream);
  if (i == DT_F16 && o == DT_F16) return launch_fwd<B2R, TypedIO<__half, __half>>(a, k, stream);
  if (i == DT_U8 && o == DT_F32) return launch_fwd<B2R, TypedIO<uint8_t, float>>(a, k, stream);
  if (i == DT_F32 && o == DT_F32) return launch_fwd<B2R, TypedIO<float, float>>(a, k, stream);
  if (i == DT_F32 && o == DT_U8) return launch_fwd<B2R, TypedIO<float, uint8_t>>(a, k, stream);
  if (i == DT_BF16 && o == DT_BF16)
    return launch_fwd<B2R, TypedIO<__nv_bfloat16, __nv_bfloat16>>(a, k, stream);
  *handled = false;
  return cudaSuccess;
}

}  // namespace wdweno
