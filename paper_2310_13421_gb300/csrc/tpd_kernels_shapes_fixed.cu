// complex128 block-fixed-point pass kernels compiled for the common pass
// layouts (tpd_shape.h), one instantiation per (layout, role) the planner's
// default plans use, for the decomposition and the composition.
#include "tpd_kernels_impl.cuh"

namespace tpd {

namespace {
template <bool kDec, int kMin, int kRole, int kShape>
PassKernel fixed_k() {
  return k_pass<FixedArith, kDec, kStdThreads, kMin, kRole, kShape>;
}

template <bool kDec, int kMin>
PassKernel fixed_table(int shape, int role) {
  constexpr int kIn = kRoleIntIn, kOut = kRoleIntOut, kInOut = kRoleIntIn | kRoleIntOut;
  switch (shape * 4 + role) {
    case kShapeFirst6 * 4 + kOut: return fixed_k<kDec, kMin, kOut, kShapeFirst6>();
    case kShapeFirst5 * 4 + kOut: return fixed_k<kDec, kMin, kOut, kShapeFirst5>();
    case kShapeFirst4 * 4 + kOut: return fixed_k<kDec, kMin, kOut, kShapeFirst4>();
    case kShapeMid4 * 4 + kInOut: return fixed_k<kDec, kMin, kInOut, kShapeMid4>();
    case kShapeMid4 * 4 + kIn: return fixed_k<kDec, kMin, kIn, kShapeMid4>();
    case kShapeMid4D11 * 4 + kIn: return fixed_k<kDec, kMin, kIn, kShapeMid4D11>();
    case kShapeMid4D11 * 4 + kInOut: return fixed_k<kDec, kMin, kInOut, kShapeMid4D11>();
    default: return nullptr;
  }
}
}  // namespace

PassKernel shape_kernel_fixed(bool dec, int shape, int role, int min_blocks) {
  if (min_blocks == kOccLow) return dec ? fixed_table<true, kOccLow>(shape, role) : fixed_table<false, kOccLow>(shape, role);
  return nullptr;
}

// The persistent prefetching form (k_pass_pf) of the decomposition for a
// compiled layout and role where it was measured faster on GB300, or nullptr:
// the first passes (double -> int64; n = 14 first pass 1.864 -> 1.754 ms,
// n = 15 7.50 -> 6.97 ms) and the last pass of n = 15 on 2^11-element tiles
// (7.72 -> 7.12 ms); the later passes on 2^12-element tiles ran as fast or
// slower (n = 14 last pass 1.703 -> 1.870 ms).
PassKernel shape_kernel_fixed_pf(int shape, int role) {
  constexpr int kIn = kRoleIntIn, kOut = kRoleIntOut;
  switch (shape * 4 + role) {
    case kShapeFirst6 * 4 + kOut: return k_pass_pf<true, kOut, kShapeFirst6>;
    case kShapeFirst5 * 4 + kOut: return k_pass_pf<true, kOut, kShapeFirst5>;
    case kShapeFirst4 * 4 + kOut: return k_pass_pf<true, kOut, kShapeFirst4>;
    case kShapeMid4D11 * 4 + kIn: return k_pass_pf<true, kIn, kShapeMid4D11>;
    default: return nullptr;
  }
}

// 2^13-element tiles as two-CTA clusters (the 5-level passes of n = 11 and 15)
PassKernel shape_kernel_fixed_cl(bool dec, int shape, int role) {
  if (shape != kShapeMid5D13) return nullptr;
  constexpr int kIn = kRoleIntIn, kInOut = kRoleIntIn | kRoleIntOut;
  if (role == kInOut) return dec ? k_pass_cl<FixedArith, true, kInOut, kShapeMid5D13>
                                 : k_pass_cl<FixedArith, false, kInOut, kShapeMid5D13>;
  if (role == kIn) return dec ? k_pass_cl<FixedArith, true, kIn, kShapeMid5D13>
                              : k_pass_cl<FixedArith, false, kIn, kShapeMid5D13>;
  return nullptr;
}

}  // namespace tpd
