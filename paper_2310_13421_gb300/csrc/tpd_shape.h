// Pass shapes compiled into the pass kernels.
//
// A pass's in-tile layout -- its tile bits D, levels K, the stages' register,
// lane and warp maps and its class bits -- depends only on how the pass's
// levels sit among its tile bits, not on n or on where the tiles lie in the
// matrix, so the planner's default plans for every matrix size share a
// handful of layouts.  For those the pass kernels are also compiled with the
// layout as a compile-time constant (GeoCT in tpd_pass.cuh): the per-tile
// work a run-time PassDesc costs -- constant-bank loads of the stage maps,
// the loop over stages, the choice between in-register and shuffle levels,
// index arithmetic from run-time bit positions -- folds away.  Any other plan
// runs the same kernel code with the run-time descriptor; both forms apply the
// same operations to the same elements in the same order, so their results are
// identical bit for bit.
#pragma once

#include <stdint.h>

#include "tpd_plan.h"

namespace tpd {

constexpr int kShapeMaxStages = 3;

struct ShapeDesc {
  int D, K, nstage;
  int8_t reg[kShapeMaxStages][4];
  int8_t lane[kShapeMaxStages][5];
  int8_t warp[kShapeMaxStages][4];
  int8_t npair[kShapeMaxStages];
  int8_t nshfl[kShapeMaxStages];
  int8_t shfl_lane[kShapeMaxStages][4];
  int8_t cls_bit[kMaxTileBits];   // PassDesc::cls_w[i] = 1 << cls_bit[i]
};

// The layouts of the planner's default passes that carry most of the work
// (tile bits in ascending global order; "first": the pass starting at level 0,
// whose column bits are the matrix's lowest bits; "middle": a later pass, its
// passengers -- the lowest column bits -- below its level bits).
enum ShapeId {
  kShapeFirst6 = 0,   // 6 levels on 2^12 elements (n = 14, 15 and others)
  kShapeFirst5,       // 5 levels on 2^12 (n = 13 and others)
  kShapeMid4,         // 4 levels + 4 passengers on 2^12 (most later passes)
  kShapeFirst4,       // 4 levels on 2^12, complex64 compensated first pass (128-byte runs)
  kShapeMid4D11,      // 4 levels + 3 passengers on 2^11 (complex128 middle passes, n = 15 last pass)
  kShapeMid3,         // 3 levels + 6 passengers on 2^12 (compensated complex64 last passes)
  kShapeMid5D13,      // 5 levels + 3 passengers on 2^13, one 512-thread CTA (complex64 n = 11, 15)
  kNumShapes
};

constexpr ShapeDesc kShapes[kNumShapes] = {
    // kShapeFirst6: levels 0-5, no passengers
    {12, 6, 2,
     {{6, 7, 8, 9}, {4, 10, 5, 11}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 1, 2, 3, 6}, {0, 0, 0, 0, 0}},
     {{5, 10, 11, 0}, {7, 8, 9, 0}, {0, 0, 0, 0}},
     {0, 2, 0},
     {4, 0, 0},
     {{0, 1, 2, 3}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 0, 1, 2, 3, 4, 5, 0}},
    // kShapeFirst5: levels 0-4 + 2 passengers
    {12, 5, 2,
     {{7, 8, 9, 11}, {3, 10, 4, 11}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 1, 2, 5, 6}, {0, 0, 0, 0, 0}},
     {{5, 6, 10, 0}, {7, 8, 9, 0}, {0, 0, 0, 0}},
     {0, 2, 0},
     {3, 0, 0},
     {{0, 1, 2, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 6, 0, 1, 2, 3, 4, 0}},
    // kShapeMid4: 4 passengers, levels' column bits 4-7, row bits 8-11
    {12, 4, 2,
     {{5, 9, 6, 10}, {4, 8, 7, 11}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 1, 2, 3, 5}, {0, 0, 0, 0, 0}},
     {{7, 8, 11, 0}, {6, 9, 10, 0}, {0, 0, 0, 0}},
     {2, 2, 0},
     {0, 0, 0},
     {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 6, 7, 4, 5, 6, 7, 0}},
    // kShapeFirst4: levels 0-3 + 4 passengers, one stage of four shuffle levels
    {12, 4, 1,
     {{8, 9, 10, 11}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}},
     {{5, 6, 7, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 0, 0},
     {4, 0, 0},
     {{0, 1, 2, 3}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 6, 7, 0, 1, 2, 3, 0}},
    // kShapeMid4D11: 3 passengers, levels' column bits 3-6, row bits 7-10
    {11, 4, 2,
     {{5, 9, 6, 10}, {3, 7, 4, 8}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 1, 2, 5, 6}, {0, 0, 0, 0, 0}},
     {{7, 8, 0, 0}, {9, 10, 0, 0}, {0, 0, 0, 0}},
     {2, 2, 0},
     {0, 0, 0},
     {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 6, 3, 4, 5, 6, 0, 0}},
    // kShapeMid3: 6 passengers, levels' column bits 6-8, row bits 9-11
    {12, 3, 2,
     {{6, 9, 11, 10}, {7, 10, 8, 11}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 1, 2, 3, 4}, {0, 0, 0, 0, 0}},
     {{5, 7, 8, 0}, {5, 6, 9, 0}, {0, 0, 0, 0}},
     {1, 2, 0},
     {0, 0, 0},
     {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 6, 7, 8, 6, 7, 8, 0}},
    // kShapeMid5D13: 3 passengers, levels' column bits 3-7, row bits 8-12
    {13, 5, 2,
     {{5, 10, 8, 9}, {6, 11, 7, 12}, {0, 0, 0, 0}},
     {{0, 1, 2, 3, 4}, {0, 1, 2, 3, 4}, {0, 0, 0, 0, 0}},
     {{6, 7, 11, 12}, {5, 8, 9, 10}, {0, 0, 0, 0}},
     {1, 2, 0},
     {2, 0, 0},
     {{3, 4, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}},
     {0, 1, 2, 3, 4, 5, 6, 7, 3, 4, 5, 6, 7}},
};

// Packed forms (4 bits per tile-bit number, 3 per shuffle lane) from which
// the kernels read the layout with shifts of constants.
constexpr uint64_t shape_pack_reg(const ShapeDesc& s) {
  uint64_t v = 0;
  for (int t = 0; t < s.nstage; ++t)
    for (int i = 0; i < 4; ++i) v |= (uint64_t)(s.reg[t][i] & 15) << (16 * t + 4 * i);
  return v;
}
constexpr uint64_t shape_pack_lane(const ShapeDesc& s) {
  uint64_t v = 0;
  for (int t = 0; t < s.nstage; ++t)
    for (int i = 0; i < 5; ++i) v |= (uint64_t)(s.lane[t][i] & 15) << (20 * t + 4 * i);
  return v;
}
constexpr uint64_t shape_pack_warp(const ShapeDesc& s) {
  uint64_t v = 0;
  for (int t = 0; t < s.nstage; ++t)
    for (int i = 0; i < 4; ++i) v |= (uint64_t)(s.warp[t][i] & 15) << (16 * t + 4 * i);
  return v;
}
constexpr uint64_t shape_pack_stage(const ShapeDesc& s) {
  uint64_t v = 0;
  for (int t = 0; t < s.nstage; ++t) v |= (uint64_t)((s.npair[t] & 3) | (s.nshfl[t] & 7) << 2) << (8 * t);
  return v;
}
constexpr uint64_t shape_pack_shfl(const ShapeDesc& s) {
  uint64_t v = 0;
  for (int t = 0; t < s.nstage; ++t)
    for (int j = 0; j < 4; ++j) v |= (uint64_t)(s.shfl_lane[t][j] & 7) << (12 * t + 3 * j);
  return v;
}
constexpr uint64_t shape_pack_cls(const ShapeDesc& s) {
  uint64_t v = 0;
  for (int i = 0; i < s.D; ++i) v |= (uint64_t)(s.cls_bit[i] & 15) << (4 * i);
  return v;
}

template <int kId>
struct ShapeT {
  static constexpr int kD = kShapes[kId].D;
  static constexpr int kK = kShapes[kId].K;
  static constexpr int kNStage = kShapes[kId].nstage;
  static constexpr uint64_t kReg = shape_pack_reg(kShapes[kId]);
  static constexpr uint64_t kLane = shape_pack_lane(kShapes[kId]);
  static constexpr uint64_t kWarp = shape_pack_warp(kShapes[kId]);
  static constexpr uint64_t kStg = shape_pack_stage(kShapes[kId]);
  static constexpr uint64_t kShfl = shape_pack_shfl(kShapes[kId]);
  static constexpr uint64_t kCls = shape_pack_cls(kShapes[kId]);
};

// The compiled shape a pass's layout equals, or -1.
inline int match_shape(const PassDesc& pd) {
  for (int id = 0; id < kNumShapes; ++id) {
    const ShapeDesc& s = kShapes[id];
    if (pd.D != s.D || pd.K != s.K || pd.nstage != s.nstage) continue;
    bool ok = true;
    for (int i = 0; i < pd.D && ok; ++i) ok = pd.cls_w[i] == (1 << s.cls_bit[i]);
    for (int t = 0; t < pd.nstage && ok; ++t) {
      const Stage& st = pd.st[t];
      ok = st.npair == s.npair[t] && st.nshfl == s.nshfl[t];
      for (int i = 0; i < kRegBits && ok; ++i) ok = st.reg[i] == s.reg[t][i];
      for (int i = 0; i < kLaneBits && ok; ++i) ok = st.lane[i] == s.lane[t][i];
      for (int i = 0; i < pd.D - kMinTileBits && ok; ++i) ok = st.warp[i] == s.warp[t][i];
      for (int j = 0; j < st.nshfl && ok; ++j) ok = st.shfl_lane[j] == s.shfl_lane[t][j];
    }
    if (ok) return id;
  }
  return -1;
}

}  // namespace tpd
