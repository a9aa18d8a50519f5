// Pass plans for the in-place Pauli decomposition butterfly.
//
// The element at flat index r*N + c of an N x N matrix (N = 2^n) has 2n index
// bits: column bits c_0..c_{n-1} are global bits 0..n-1, row bits r_0..r_{n-1}
// are global bits n..2n-1.  One qubit level beta applies Eq. 4 to every 2x2
// quad over (r_beta, c_beta), i.e. it couples global bits beta and n+beta.
// Eq. 5 makes the levels commute, so a pass may apply any group of levels.
//
// A pass applies the levels [b, b+K).  Its work unit, a *tile*, is the set of
// 2^D elements that agree on all global bits outside a D-bit tile mask; the
// mask holds the 2K bits of the levels plus D-2K "passenger" bits, the lowest
// column bits, so that every thread's memory runs are at least 128 bytes.
// Tile bit i is the i-th lowest global bit of the mask.
//
// Inside a CTA of 2^(D-4) threads each thread holds E = 16 elements in
// registers.  A *stage* fixes which tile bits are register bits, lane bits and
// warp bits.  A level is applied in a stage either in registers (its column
// and row bit are both register bits) or across lanes with shuffles (column
// bit a lane bit, row bit a register bit).  Consecutive stages exchange the
// tile through shared memory.  Lanes always cover tile bits 0..2 (0..3 for
// the compensated complex64 form), so accesses of 16-byte elements to shared
// memory are conflict-free, and global accesses cover runs of 8 elements
// (128 bytes in complex128, 64 in complex64; 16 elements for the compensated
// form).
#pragma once

#include <stdint.h>

namespace tpd {

constexpr int kRegBits = 4;                 // E = 2^kRegBits elements per thread
constexpr int kElems = 1 << kRegBits;
constexpr int kRegSlots = 4;                // register-bit entries of a stage (those >= kRegBits unused, 0)
constexpr int kLaneBits = 5;
constexpr int kMinTileBits = kRegBits + kLaneBits;   // one warp
constexpr int kMaxTileBits = 13;
constexpr int kMaxWarpBits = kMaxTileBits - kMinTileBits;
constexpr int kStdTileBits = 12;                      // the default tile
constexpr int kStdThreads = 1 << (kStdTileBits - kRegBits);   // threads of a default tile's CTA
constexpr int kBigThreads = 1 << (kMaxTileBits - kRegBits);   // threads of a 2^13-element tile
constexpr int kClThreads = kBigThreads / 2;                    // per CTA of a two-CTA cluster
constexpr int kClWarpBit = kMaxWarpBits - 1;          // the warp bit that is the cluster rank
// CTAs per SM the pass kernels are compiled for, a tile of up to 2^12
// elements: kOccHigh (fewer registers per thread) or kOccLow
constexpr int kOccHigh = kRegBits >= 4 ? 3 : 2;
constexpr int kOccLow = kOccHigh - 1;
// Reduction slots of a CTA: one per warp of the largest tile for each of the
// three tile-wide reductions, and as many spare.  Kept small: three
// 2^12-element complex64 CTAs (64 KB each) must fit the 196 KB shared-memory
// carve-out, which leaves the L1 room for their spilled registers (at 512
// bytes they needed the 228 KB one: n = 15 compensated 20.55 -> 22.27 ms).
constexpr int kRedStride = 1 << kMaxWarpBits;
constexpr int kRedInts = 4 * kRedStride;
constexpr int kRedBytes = kRedInts * 4;
constexpr int kMaxStages = 4;
constexpr int kMaxQubits = 16;
constexpr int kMaxRuns = 2 * kMaxQubits;
constexpr int kMaxLevels = 6;

struct Stage {
  int8_t reg[kRegSlots];     // tile bit of register-index bit i (i < kRegBits)
  int8_t lane[kLaneBits];    // tile bit of lane bit i
  int8_t warp[kMaxWarpBits]; // tile bit of warp bit i (D-9 of them)
  int8_t npair;              // in-register levels: reg bits (2p, 2p+1) = (column, row)
  int8_t nshfl;              // shuffle levels: reg bit 2*npair+s is the row bit ...
  int8_t shfl_lane[4];       // ... and lane bit shfl_lane[s] the column bit
};

struct PassDesc {
  int32_t n;                 // qubits of the matrix
  int32_t D;                 // tile bits
  int32_t K;                 // levels applied by this pass
  int32_t b;                 // first level
  int32_t nstage;
  int32_t nrest;             // tile-id bits = 2n - D
  int64_t ntiles;            // 2^(2n - D)
  Stage st[kMaxStages];
  int8_t gbit[kMaxTileBits];            // global bit of tile bit i
  int8_t rest_gbit[2 * kMaxQubits];     // global bit of tile-id bit j (ascending)
  // Zero-skip bookkeeping.  The tile id, in the NEXT pass, of an element is
  // linear in the element's global bits: next_w[i] per tile bit i and
  // next_rest_w[j] per tile-id bit j (0 where the bit lies inside the next
  // pass's tile).
  int32_t has_next;
  int32_t next_w[kMaxTileBits];
  int64_t next_rest_w[2 * kMaxQubits];
  int32_t min_blocks;        // CTAs per SM the pass kernel is compiled for (2 or 3); D = 13: 1 = one
                             // CTA of 512 threads, 2 = a two-CTA cluster of 256 (complex128)
  int32_t rt_layout;         // 1: run the kernel that reads the layout from this descriptor even
                             // where a compiled shape (tpd_shape.h) matches it
  // Block fixed point: the *class* of a tile position.  A pass only ever adds
  // elements that agree on every passenger bit and on x_j = r_j xor c_j of
  // each of its levels j (Eq. 4 adds a00 to a11 and a01 to a10, and both
  // outputs keep the quad's x), so each class -- 2^K elements -- is summed
  // on its own binary point.  The class index is linear (XOR) in the tile
  // bits: cls_w[i] is the class bit of tile bit i, a level's column and row
  // bit sharing one; the column-type bits take class bits in ascending tile
  // order, so the lowest tile bits (stage 0's lanes) get the lowest class
  // bits.  2^(D-K) classes per tile.
  int32_t cls_w[kMaxTileBits];
  // Block fixed point between passes: a pass that does not end the plan
  // stores its int64 sums in place and one binary point per class, at index
  // (tile id << (D - K)) | class in its binary-point array.  The index, in the
  // PREVIOUS pass's array, of the class an element of this pass came from is
  // linear (XOR) in the element's global bits: src_w[i] per tile bit i and
  // src_rest_w[j] per tile-id bit j (below 2^31: 2n - K bits).
  int32_t has_prev;
  uint32_t src_w[kMaxTileBits];
  uint32_t src_rest_w[2 * kMaxQubits];
};

// A whole-matrix plan: one pass per group of levels.
struct Plan {
  int32_t n;
  int32_t npass;
  int32_t elem_bytes;        // 16 (c128, compensated c64 in registers) or 8
  PassDesc pass[kMaxQubits];  // one level per pass at worst
};

}  // namespace tpd
