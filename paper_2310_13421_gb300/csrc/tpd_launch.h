// Host-visible launch interface of the Pauli butterfly kernels.  The kernels
// themselves live in tpd_kernels_c128.cu (fixed point and fp64) and
// tpd_kernels_c64.cu (fp32 plain and compensated).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tpd_plan.h"

namespace tpd {

enum Arith { kArithFixed = 0, kArithF64 = 1, kArithF32 = 2, kArithF32C = 3, kArithF32Fixed = 4 };

struct PassArgs {
  // batched launches: tile t of the grid belongs to matrix ptrs[items[t / tiles_per_mat]]
  void* const* ptrs;          // nullptr: single matrix `mat`
  const int* items;
  long long tiles_per_mat;
  void* mat;                  // matrix base (A::Store*), device
  const uint8_t* flags_in;    // per tile of this pass: 0 = all zero, skip; nullptr = no skipping
  const uint8_t* need;        // per tile of this pass: 0 = feeds no requested weight (partial
                              // decomposition), skip; nullptr = every tile
  uint8_t* flags_out;         // per tile of the next pass: set to 1 when it gets a nonzero; nullptr = none
  int skip_zero;              // test loaded tiles for all-zero and leave them untouched
  int out_pow2;               // fixed point: output multiplied by 2^out_pow2 (exact)
  double out_mul;             // IEEE paths: output multiplier (exact power of two or user scale);
                              // fixed point: non-power-of-two residual factor (1.0 normally)
  // Block fixed point between passes.  A pass that does not end the plan
  // stores its int64 sums in place and each class's binary point q (value =
  // v * 2^q) in q_out[(tile << (D - K)) | class]; the next pass reads, per
  // element, the binary point of the class it came from (PassDesc::src_w).
  // Markers: kQIeee (the class holds IEEE doubles: its tile met an Inf or
  // NaN); any other value at or below kQValidMin (e.g. the 0x80 byte fill of
  // a cleared array) a class whose elements are all zero.
  const int16_t* q_in;        // nullptr: input is IEEE numbers
  int16_t* q_out;             // nullptr: output is IEEE numbers
  long long q_in_stride;      // batched: q entries per matrix (previous pass's classes)
  long long q_out_stride;     // batched: q entries per matrix (this pass's classes)
  // L2 chunk of a single matrix: CTA b runs tile chunk_or | (bit k of b) << chunk_free[k]
  int chunked;
  int nfree;
  unsigned long long chunk_or;
  int8_t chunk_free[2 * kMaxQubits];
};

// Role of a block-fixed-point pass: input IEEE numbers (0) or int64 sums of a
// previous pass (kRoleIntIn); output IEEE numbers (0) or int64 sums for a
// next pass (kRoleIntOut).
constexpr int kRoleIntIn = 1;
constexpr int kRoleIntOut = 2;

// binary points are in [-1100, 1100]; kQIeee marks an IEEE class; any other
// value at or below kQValidMin a zero class
constexpr int kQValidMin = -4096;
constexpr int kQIeee = -30000;
constexpr unsigned char kQFillByte = 0x80;

struct SmallArgs {
  void* const* ptrs;          // batched: device array of matrix pointers (nullptr: use `mat`)
  const int* ns;              // batched: device array of n_i
  const int* items;           // batched: matrix index per CTA (nullptr: CTA i = matrix i)
  void* mat;                  // single matrix
  int n;                      // single matrix qubits
  int skip_zero;
  int scale_mode;             // compose: 0 scale 1, 1 scale 2^-n; decompose ignores
};

// ---------------------------------------------------------------- batched, one launch
//
// The persistent batched kernel walks one global list of work items, claimed
// in order from a device counter: item 0 buckets the matrices by qubit count;
// then one *segment* per qubit count n.  For n >= 7 a segment holds every
// pass of every matrix of that n, software-pipelined: round r = (pass 0 of
// matrix r, pass 1 of matrix r - lag, pass 2 of matrix r - 2 lag, ...), each
// pass as tiles / tpi items (tile-major), out-of-range (pass, matrix) slots empty.
// A matrix's later passes thus run `lag` rounds after its earlier ones, while
// its data (16 * 4^n bytes) is still in L2, so for matrices up to a few MB a
// pass after the first reads, and the passes overwrite, lines that have not
// gone back to HBM.  A tile of pass p > 0 waits (bounded) until all tiles of
// pass p-1 of ITS matrix are done, counted per (pass, matrix) in `done`.  For
// n <= 6 a segment holds one item per whole matrix.  An item of a pipelined
// segment is up to kBatchTilesPerItem consecutive tiles of one pass of one
// matrix.  A CTA claims its next item as it starts the current one (two claims
// per CTA in flight).
constexpr int kBatchMaxDescs = 16;
constexpr int kBatchMaxSegs = 12;
constexpr int kBatchMaxN = 12;
constexpr int kSegMaxPasses = 3;
constexpr long long kBatchTilesPerItem = 32;
constexpr int kSegSmall = 0;
constexpr int kSegPipe = 1;

struct BatchSeg {
  PassArgs args[kSegMaxPasses];  // per pass (q arrays: pass-level bases, matrix j at + j * stride)
  int32_t kind;               // kSegSmall / kSegPipe
  int32_t n;                  // qubits of the segment's matrices
  int32_t npass;              // kSegPipe: passes per matrix (1..kSegMaxPasses)
  int32_t desc;               // kSegPipe: pass p uses BatchParams::desc[desc + p]
  int32_t item_start;         // first bucket position of the segment's matrices
  int32_t nmat;               // matrices in the segment
  int32_t lag;                // kSegPipe: rounds between consecutive passes of a matrix
  int32_t done;               // kSegPipe: counter of (pass p, matrix j) at ctrl[kCtrlDone + done + p * nmat + j]
  int32_t wait_extra;         // test hook: added to every wait's target
  int8_t shape[4];            // kSegPipe, block fixed point: compiled layout of pass p (tpd_shape.h), or -1
  int64_t first;              // first work index of the segment
  int64_t tiles;              // tiles per pass (1 for kSegSmall)
  int64_t tpi;                // kSegPipe: consecutive tiles of one pass per work item (divides tiles)
};

struct BatchParams {
  PassDesc desc[kBatchMaxDescs];
  BatchSeg seg[kBatchMaxSegs];
  int32_t nseg;
  int32_t count;              // matrices
  int32_t hist[kBatchMaxN + 1];  // host's count per qubit number (checked by the bucket item)
  int32_t scale_mode;         // compose: 0 scale 1, 1 scale 2^-n (small matrices)
  int64_t total;              // work items
  void* const* ptrs;          // device array of matrix pointers
  const int* ns;              // device array of n_i
  int* items;                 // bucketed matrix indices (written by item 0)
  unsigned long long* bptrs;  // bucketed matrix pointers, ptrs[items[k]] (written by item 0)
  unsigned* ctrl;             // [0] next work item, [1] status, [2] bucket done, [3] -, then done counters
};

// status codes the kernel writes to ctrl[kCtrlStatus] (tpd_status values)
constexpr unsigned kBatchStatusBadSizes = 1;    // TPD_ERR_INVALID_ARG: ns_dev disagrees with ns
constexpr unsigned kBatchStatusTimeout = 6;     // TPD_ERR_TIMEOUT: a bounded wait gave up

// control words (unsigned) at the head of BatchParams::ctrl; cleared before each launch
constexpr int kCtrlWork = 0;
constexpr int kCtrlStatus = 1;
constexpr int kCtrlBucket = 2;
constexpr int kCtrlDone = 4;

// Persistent batched kernel for an arithmetic: `grid` CTAs of 256 threads.
cudaError_t launch_batch(int arith, bool dec, const BatchParams& bp, int* grid_out, cudaStream_t s);

// Nonzero weights in string order (|re| > tol or |im| > tol; NaN kept): the
// first `capacity` go to strings / weights, the number of all to *total.
size_t nonzero_workspace_bytes(int n);
cudaError_t launch_nonzero(const void* W, int n, int elem_bytes, double tol, unsigned long long* strings,
                           void* weights, unsigned long long capacity, unsigned long long* total, void* ws,
                           cudaStream_t s);

// Sparse (COO, complex128) decomposition into the list of nonzero weights,
// sorted by string index; max_entries bounds the live entries of a level
// (*status = 4 if exceeded).
size_t sparse_workspace_bytes(unsigned long long max_entries);
cudaError_t launch_sparse(const int* rows, const int* cols, const void* vals, unsigned long long m, int n,
                          unsigned long long max_entries, unsigned long long* strings, void* weights,
                          unsigned long long capacity, unsigned long long* count, void* ws, unsigned* status,
                          cudaStream_t s);

// out[i] = mat[pos[i]] for i < count (elements of elem_bytes).
cudaError_t launch_gather(const void* mat, const unsigned long long* pos, unsigned long long count, int elem_bytes,
                          void* out, cudaStream_t s);

// Layout conversion RC <-> STRING (out of place) and the fp64 sum of squared
// magnitudes (deterministic; workspace of sumsq_workspace_bytes()).
cudaError_t launch_layout(const void* src, void* dst, int n, int elem_bytes, int to_string, cudaStream_t s);
size_t sumsq_workspace_bytes();
cudaError_t launch_sumsq(const void* x, unsigned long long count, int elem_bytes, double* out, void* ws,
                         cudaStream_t s);

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

// Bucket matrices by qubit count: out_items lists the matrix indices of each
// n in turn (ascending n).  The device counts are checked against the host's
// histogram hist[0..12]; on a mismatch (ns_dev disagreeing with the host's ns)
// the kernel sets *status to kBatchStatusBadSizes and fills out_items with -1,
// which every batched kernel treats as "no matrix" (nothing is touched).
struct BucketHist { int h[13]; };
cudaError_t launch_bucket(const int* ns_dev, int count, const BucketHist& hist, int* out_items, unsigned* status,
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
