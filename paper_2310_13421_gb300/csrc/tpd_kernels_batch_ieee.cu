// Persistent batched kernels for the IEEE arithmetics (fp64, fp32, fp32
// compensated) and the arithmetic dispatch of launch_batch.
#include "tpd_batch.cuh"

namespace tpd {

cudaError_t launch_batch_fixed(bool dec, const BatchParams& bp, int* grid_out, cudaStream_t s);

cudaError_t launch_batch(int arith, bool dec, const BatchParams& bp, int* grid_out, cudaStream_t s) {
  switch (arith) {
    case kArithFixed: return launch_batch_fixed(dec, bp, grid_out, s);
    case kArithF64:
      return dec ? launch_batch_t<F64Arith, true>(bp, grid_out, s) : launch_batch_t<F64Arith, false>(bp, grid_out, s);
    case kArithF32:
      return dec ? launch_batch_t<F32Arith, true>(bp, grid_out, s) : launch_batch_t<F32Arith, false>(bp, grid_out, s);
    case kArithF32Fixed:
      return dec ? launch_batch_t<Fixed32Arith, true>(bp, grid_out, s)
                 : launch_batch_t<Fixed32Arith, false>(bp, grid_out, s);
    default:
      return dec ? launch_batch_t<F32CArith, true>(bp, grid_out, s)
                 : launch_batch_t<F32CArith, false>(bp, grid_out, s);
  }
}

}  // namespace tpd
