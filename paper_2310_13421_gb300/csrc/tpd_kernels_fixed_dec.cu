// complex128 block-fixed-point decomposition pass kernels (a translation unit
// of their own so that the library's kernels compile in parallel).
#include "tpd_kernels_impl.cuh"

namespace tpd {

cudaError_t launch_pass_fixed_dec(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s) {
  return launch_pass_t<FixedArith, true>(pd, args, ntiles_total, s);
}

cudaError_t launch_pass_pipe_fixed_dec(const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s) {
  return launch_pass_pipe_t<true>(pd, args, nsm, s);
}

}  // namespace tpd
