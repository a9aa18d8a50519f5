// complex64 pass kernels (fp32, compensated fp32, block fixed point) compiled
// for the common pass layouts (tpd_shape.h), one instantiation per (layout,
// CTAs per SM) the planner's default plans use.
#include "tpd_kernels_impl.cuh"

namespace tpd {

namespace {
template <class A, int kMin, int kShape>
PassKernel c64_k() {
  return k_pass<A, true, kStdThreads, kMin, 0, kShape>;
}
}  // namespace

PassKernel shape_kernel_c64(int arith, bool dec, int shape, int min_blocks) {
  if (!dec) return nullptr;
  const int key = shape * 4 + min_blocks;
  if (arith == kArithF32C) {
    switch (key) {
      case kShapeFirst6 * 4 + kOccHigh: return c64_k<F32CArith, kOccHigh, kShapeFirst6>();
      case kShapeFirst4 * 4 + kOccHigh: return c64_k<F32CArith, kOccHigh, kShapeFirst4>();
      case kShapeMid4 * 4 + kOccLow: return c64_k<F32CArith, kOccLow, kShapeMid4>();
      case kShapeMid3 * 4 + kOccHigh: return c64_k<F32CArith, kOccHigh, kShapeMid3>();
      default: return nullptr;
    }
  }
  if (arith == kArithF32) {
    switch (key) {
      case kShapeFirst6 * 4 + kOccLow: return c64_k<F32Arith, kOccLow, kShapeFirst6>();
      case kShapeFirst5 * 4 + kOccLow: return c64_k<F32Arith, kOccLow, kShapeFirst5>();
      case kShapeFirst4 * 4 + kOccLow: return c64_k<F32Arith, kOccLow, kShapeFirst4>();
      case kShapeMid4 * 4 + kOccLow: return c64_k<F32Arith, kOccLow, kShapeMid4>();
      case kShapeMid4D11 * 4 + kOccLow: return c64_k<F32Arith, kOccLow, kShapeMid4D11>();
      default: return nullptr;
    }
  }
  return nullptr;
}

}  // namespace tpd
