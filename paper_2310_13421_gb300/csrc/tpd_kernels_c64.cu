// complex64 kernels: IEEE fp32, TwoSum-compensated fp32 and int64 block fixed
// point (whole small matrices of the fixed-point form use the compensated
// kernel).
#include "tpd_kernels_impl.cuh"

namespace tpd {

cudaError_t launch_pass_c64(int arith, bool dec, const PassDesc& pd, const PassArgs& args,
                            long long ntiles_total, cudaStream_t s) {
  if (arith == kArithF32C)
    return dec ? launch_pass_t<F32CArith, true>(pd, args, ntiles_total, s)
               : launch_pass_t<F32CArith, false>(pd, args, ntiles_total, s);
  if (arith == kArithF32Fixed)
    return dec ? launch_pass_t<Fixed32Arith, true>(pd, args, ntiles_total, s)
               : launch_pass_t<Fixed32Arith, false>(pd, args, ntiles_total, s);
  return dec ? launch_pass_t<F32Arith, true>(pd, args, ntiles_total, s)
             : launch_pass_t<F32Arith, false>(pd, args, ntiles_total, s);
}

cudaError_t launch_small_c64(int arith, bool dec, const SmallArgs& args, int blocks, int n_max, cudaStream_t s) {
  if (arith == kArithF32C || arith == kArithF32Fixed)
    return dec ? launch_small_t<F32CArith, true>(args, blocks, n_max, s)
               : launch_small_t<F32CArith, false>(args, blocks, n_max, s);
  return dec ? launch_small_t<F32Arith, true>(args, blocks, n_max, s)
             : launch_small_t<F32Arith, false>(args, blocks, n_max, s);
}

}  // namespace tpd
