// complex64 block-fixed-point pass kernels compiled for the common pass
// layouts (tpd_shape.h), at the CTAs per SM the planner gives each layout.
#include "tpd_kernels_impl.cuh"

namespace tpd {

PassKernel shape_kernel_fx32(int shape, int min_blocks) {
  using A = Fixed32Arith;
  constexpr int kT = kStdThreads;
  if (min_blocks == kOccHigh) {
    switch (shape) {
      case kShapeFirst6: return k_pass<A, true, kT, kOccHigh, 0, kShapeFirst6>;
      case kShapeFirst5: return k_pass<A, true, kT, kOccHigh, 0, kShapeFirst5>;
      case kShapeFirst4: return k_pass<A, true, kT, kOccHigh, 0, kShapeFirst4>;
      case kShapeMid4: return k_pass<A, true, kT, kOccHigh, 0, kShapeMid4>;
      default: return nullptr;
    }
  }
  if (min_blocks == kOccLow && shape == kShapeMid4D11) return k_pass<A, true, kT, kOccLow, 0, kShapeMid4D11>;
  if (min_blocks == 1 && shape == kShapeMid5D13) return k_pass<A, true, kBigThreads, 1, 0, kShapeMid5D13>;
  return nullptr;
}

}  // namespace tpd
