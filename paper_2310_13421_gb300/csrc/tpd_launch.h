// Host-visible launch interface of the Pauli butterfly kernels.  The kernels
// themselves live in tpd_kernels_c128.cu (fixed point and fp64) and
// tpd_kernels_c64.cu (fp32 plain and compensated).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tpd_plan.h"

namespace tpd {

enum Arith { kArithFixed = 0, kArithF64 = 1, kArithF32 = 2, kArithF32C = 3 };

struct PassArgs {
  // batched launches: tile t of the grid belongs to matrix ptrs[items[t / tiles_per_mat]]
  void* const* ptrs;          // nullptr: single matrix `mat`
  const int* items;
  long long tiles_per_mat;
  void* mat;                  // matrix base (A::Store*), device
  const uint8_t* flags_in;    // per tile of this pass: 0 = all zero, skip; nullptr = no skipping
  uint8_t* flags_out;         // per tile of the next pass: set to 1 when it gets a nonzero; nullptr = none
  int skip_zero;              // test loaded tiles for all-zero and leave them untouched
  int out_pow2;               // fixed point: output multiplied by 2^out_pow2 (exact)
  double out_mul;             // IEEE paths: output multiplier (exact power of two or user scale);
                              // fixed point: non-power-of-two residual factor (1.0 normally)
  // Fixed point between passes.  A pass that does not end the plan stores its
  // int64 sums in place and its tile's binary point q (value = v * 2^q) in
  // q_out[tile]; the next pass reads q_in[previous tile] per element.
  // Markers: kQZero (tile never written: its elements are zero) and kQIeee
  // (tile holds IEEE doubles: it met an Inf or NaN).
  const int* q_in;            // nullptr: input is IEEE doubles
  int* q_out;                 // nullptr: output is IEEE doubles
  long long q_in_stride;      // batched: q entries per matrix (previous pass's tile count)
  long long q_out_stride;     // batched: q entries per matrix (this pass's tile count)
};

// q values above kQValidMin are binary points; kQIeee marks an IEEE tile; any
// other value (e.g. the 0xC0 byte fill of a cleared array) a zero tile.
constexpr int kQValidMin = -0x20000000;
constexpr int kQIeee = -0x30000000;
constexpr unsigned char kQFillByte = 0xC0;

struct SmallArgs {
  void* const* ptrs;          // batched: device array of matrix pointers (nullptr: use `mat`)
  const int* ns;              // batched: device array of n_i
  const int* items;           // batched: matrix index per CTA (nullptr: CTA i = matrix i)
  void* mat;                  // single matrix
  int n;                      // single matrix qubits
  int skip_zero;
  int scale_mode;             // compose: 0 scale 1, 1 scale 2^-n; decompose ignores
};

// Bytes per element in registers / shared memory for an arithmetic.
inline int arith_vbytes(int arith) { return arith == kArithF32 ? 8 : 16; }

cudaError_t launch_pass_c128(int arith, bool dec, const PassDesc& pd, const PassArgs& args, long long ntiles_total,
                             cudaStream_t s);
cudaError_t launch_small_c128(int arith, bool dec, const SmallArgs& args, int blocks, int n_max, cudaStream_t s);
cudaError_t launch_pass_c64(int arith, bool dec, const PassDesc& pd, const PassArgs& args, long long ntiles_total,
                            cudaStream_t s);
cudaError_t launch_small_c64(int arith, bool dec, const SmallArgs& args, int blocks, int n_max, cudaStream_t s);

// Persistent double-buffered fixed-point pass (D <= 12, single matrix, no
// zero skipping): one CTA per SM, nsm = SM count.
cudaError_t launch_pass_pipe_c128(bool dec, const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s);

// Bucket matrices by qubit count: for each n in [0, 32), out_offsets[n] is the
// start of its list in out_items (matrix indices, any order within a list).
// scratch: 64 ints.
cudaError_t launch_bucket(const int* ns_dev, int count, int* out_items, int* out_offsets, int* scratch,
                          cudaStream_t s);

inline cudaError_t launch_pass(int arith, bool dec, const PassDesc& pd, const PassArgs& args,
                               long long ntiles_total, cudaStream_t s) {
  return (arith == kArithFixed || arith == kArithF64) ? launch_pass_c128(arith, dec, pd, args, ntiles_total, s)
                                                      : launch_pass_c64(arith, dec, pd, args, ntiles_total, s);
}
inline cudaError_t launch_small(int arith, bool dec, const SmallArgs& args, int blocks, int n_max,
                                cudaStream_t s) {
  return (arith == kArithFixed || arith == kArithF64) ? launch_small_c128(arith, dec, args, blocks, n_max, s)
                                                      : launch_small_c64(arith, dec, args, blocks, n_max, s);
}

}  // namespace tpd
