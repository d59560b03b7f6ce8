// The persistent batched forward zoom with two coarse columns per thread
// (wd_batched_kernel.cuh), in a translation unit of its own so that it
// compiles in parallel with the one-column form (wd_batched.cu).
#include "wd_batched_kernel.cuh"

namespace wdweno {

cudaError_t launch_batched_paired(const BatchedArgs& a, const MethodConsts& k, int bmode,
                                  cudaStream_t stream) {
  return batched::launch_typed<2>(a, k, bmode, stream);
}

}  // namespace wdweno
