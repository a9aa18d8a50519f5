// complex64 pass kernels compiled for the common pass layouts (tpd_shape.h),
// one instantiation per (layout, CTAs per SM): compensated fp32 here, plain
// fp32 in tpd_kernels_shapes_f32.cu (translation units compile in parallel).
#include "tpd_kernels_impl.cuh"

namespace tpd {

namespace {
template <class A, int kMin, int kShape>
PassKernel c64_k() {
  return k_pass<A, true, kStdThreads, kMin, 0, kShape>;
}

template <class A, int kMin>
PassKernel c64_table(int shape) {
  switch (shape) {
    case kShapeFirst6: return c64_k<A, kMin, kShapeFirst6>();
    case kShapeFirst5: return c64_k<A, kMin, kShapeFirst5>();
    case kShapeFirst4: return c64_k<A, kMin, kShapeFirst4>();
    case kShapeMid4: return c64_k<A, kMin, kShapeMid4>();
    case kShapeMid4D11: return c64_k<A, kMin, kShapeMid4D11>();
    case kShapeMid3: return c64_k<A, kMin, kShapeMid3>();
    default: return nullptr;
  }
}
}  // namespace

PassKernel shape_kernel_f32(int shape, int min_blocks);
PassKernel shape_kernel_fx32(int shape, int min_blocks);

PassKernel shape_kernel_c64(int arith, bool dec, int shape, int min_blocks) {
  if (!dec) return nullptr;
  if (arith == kArithF32C) {
    if (shape == kShapeMid5D13) return nullptr;
    return min_blocks == kOccHigh ? c64_table<F32CArith, kOccHigh>(shape) : c64_table<F32CArith, kOccLow>(shape);
  }
  if (arith == kArithF32) return shape_kernel_f32(shape, min_blocks);
  if (arith == kArithF32Fixed) return shape_kernel_fx32(shape, min_blocks);
  return nullptr;
}

}  // namespace tpd
