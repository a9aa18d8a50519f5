// complex128 block-fixed-point pass kernels compiled for the common pass
// layouts (tpd_shape.h), one instantiation per (layout, role) the planner's
// default plans use.
#include "tpd_kernels_impl.cuh"

namespace tpd {

namespace {
template <bool kDec, int kRole, int kShape>
PassKernel fixed_k() {
  return k_pass<FixedArith, kDec, kStdThreads, kOccLow, kRole, kShape>;
}
}  // namespace

PassKernel shape_kernel_fixed(bool dec, int shape, int role, int min_blocks) {
  if (!dec || min_blocks != kOccLow) return nullptr;
  constexpr int kIn = kRoleIntIn, kOut = kRoleIntOut, kInOut = kRoleIntIn | kRoleIntOut;
  switch (shape * 4 + role) {
    case kShapeFirst6 * 4 + kOut: return fixed_k<true, kOut, kShapeFirst6>();
    case kShapeFirst5 * 4 + kOut: return fixed_k<true, kOut, kShapeFirst5>();
    case kShapeFirst4 * 4 + kOut: return fixed_k<true, kOut, kShapeFirst4>();
    case kShapeMid4 * 4 + kInOut: return fixed_k<true, kInOut, kShapeMid4>();
    case kShapeMid4 * 4 + kIn: return fixed_k<true, kIn, kShapeMid4>();
    case kShapeMid4D11 * 4 + kIn: return fixed_k<true, kIn, kShapeMid4D11>();
    default: return nullptr;
  }
}

}  // namespace tpd
