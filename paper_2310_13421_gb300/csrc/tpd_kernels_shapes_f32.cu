// complex64 plain fp32 pass kernels compiled for the common pass layouts
// (tpd_shape.h), one instantiation per (layout, CTAs per SM).
#include "tpd_kernels_impl.cuh"

namespace tpd {

namespace {
template <int kMin>
PassKernel f32_table(int shape) {
  switch (shape) {
    case kShapeFirst6: return k_pass<F32Arith, true, kStdThreads, kMin, 0, kShapeFirst6>;
    case kShapeFirst5: return k_pass<F32Arith, true, kStdThreads, kMin, 0, kShapeFirst5>;
    case kShapeFirst4: return k_pass<F32Arith, true, kStdThreads, kMin, 0, kShapeFirst4>;
    case kShapeMid4: return k_pass<F32Arith, true, kStdThreads, kMin, 0, kShapeMid4>;
    case kShapeMid4D11: return k_pass<F32Arith, true, kStdThreads, kMin, 0, kShapeMid4D11>;
    case kShapeMid3: return k_pass<F32Arith, true, kStdThreads, kMin, 0, kShapeMid3>;
    default: return nullptr;
  }
}
}  // namespace

PassKernel shape_kernel_f32(int shape, int min_blocks) {
  if (shape == kShapeMid5D13)
    return min_blocks == 1 ? k_pass<F32Arith, true, kBigThreads, 1, 0, kShapeMid5D13> : nullptr;
  return min_blocks == kOccHigh ? f32_table<kOccHigh>(shape) : f32_table<kOccLow>(shape);
}

}  // namespace tpd
