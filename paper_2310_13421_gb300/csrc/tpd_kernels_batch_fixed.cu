// Persistent batched kernels, complex128 block fixed point (a translation
// unit of its own so that the library's kernels compile in parallel).
#include "tpd_batch.cuh"

namespace tpd {

cudaError_t launch_batch_fixed(bool dec, const BatchParams& bp, int* grid_out, cudaStream_t s) {
  return dec ? launch_batch_t<FixedArith, true>(bp, grid_out, s) : launch_batch_t<FixedArith, false>(bp, grid_out, s);
}

}  // namespace tpd
