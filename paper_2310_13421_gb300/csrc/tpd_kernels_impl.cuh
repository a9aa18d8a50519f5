// Launch helpers shared by the per-storage-type kernel translation units.
#pragma once

#include <type_traits>

#include "tpd_launch.h"
#include "tpd_pass.cuh"

namespace tpd {

using PassKernel = void (*)(const PassDesc, const PassArgs);

// Raise kernel fn's dynamic shared-memory limit to `bytes`, the largest
// launch it can ever get, once per device (tpd_kernels_c128.cu).  The limit is
// never set to one launch's own size: a kernel node captured in a CUDA graph
// keeps the shared-memory size of its capture, and relaunching it (a graph
// replay on some drivers, or a profiler replaying graph nodes one by one) after
// a smaller launch of the same kernel had lowered the limit would fail to
// launch.
cudaError_t ensure_smem_limit(const void* fn, size_t bytes);

// Class slots of the block fixed point: 2^(D-K) ints, at most 2^(D-1) (K >= 1).
template <class A>
constexpr bool kBlockFixed = A::kFixed || A::kFixed32;
inline size_t class_slot_bytes(const PassDesc& pd) { return sizeof(int) << (pd.D - pd.K); }

// The instantiation compiled for a pass's layout (tpd_shape.h), role and
// occupancy, or nullptr: tpd_kernels_shapes_fixed.cu (complex128 block fixed
// point), tpd_kernels_shapes_c64.cu (complex64).
// min_blocks: the pass's CTAs per SM (1: one CTA of 512 threads on a 2^13-element tile).
PassKernel shape_kernel_fixed(bool dec, int shape, int role, int min_blocks);
PassKernel shape_kernel_fixed_cl(bool dec, int shape, int role);   // two-CTA clusters
PassKernel shape_kernel_fixed_pf(int shape, int role);              // persistent, prefetching
int device_sm_count();                                              // of the current device (cached)
PassKernel shape_kernel_c64(int arith, bool dec, int shape, int min_blocks);

template <class A>
constexpr int arith_code() {
  if constexpr (std::is_same<A, FixedArith>::value) return kArithFixed;
  else if constexpr (std::is_same<A, F64Arith>::value) return kArithF64;
  else if constexpr (std::is_same<A, F32Arith>::value) return kArithF32;
  else if constexpr (std::is_same<A, F32CArith>::value) return kArithF32C;
  else return kArithF32Fixed;
}

// the instantiation for a pass's CTA size, occupancy and (block fixed point) role
template <class A, bool kDec, int kRole>
PassKernel pick_pass_kernel(const PassDesc& pd, int threads) {
  if (threads > kStdThreads) return k_pass<A, kDec, kBigThreads, 1, kRole>;
  return pd.min_blocks >= kOccHigh ? k_pass<A, kDec, kStdThreads, kOccHigh, kRole>
                                   : k_pass<A, kDec, kStdThreads, kOccLow, kRole>;
}

// the role of a complex128 block-fixed-point pass from its binary-point arrays
inline int fixed_role(const PassArgs& args) {
  return (args.q_in ? kRoleIntIn : 0) | (args.q_out ? kRoleIntOut : 0);
}

// complex128 tiles of 2^13 elements planned as two-CTA clusters (min_blocks 2)
template <class A>
constexpr bool kClusterArith = std::is_same<A, FixedArith>::value || std::is_same<A, F64Arith>::value;

template <class A, bool kDec>
cudaError_t launch_pass_cl_t(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s) {
  const size_t smem = ((size_t)16 << (pd.D - 1)) + kRedBytes + (kBlockFixed<A> ? class_slot_bytes(pd) : 0);
  const size_t smem_max = ((size_t)16 << (kMaxTileBits - 1)) + kRedBytes +
                          (kBlockFixed<A> ? sizeof(int) << (kMaxTileBits - 1) : 0);
  PassKernel kfn = k_pass_cl<A, kDec, 0>;
  if constexpr (A::kFixed) {
    switch (fixed_role(args)) {
      case kRoleIntIn: kfn = k_pass_cl<A, kDec, kRoleIntIn>; break;
      case kRoleIntOut: kfn = k_pass_cl<A, kDec, kRoleIntOut>; break;
      case kRoleIntIn | kRoleIntOut: kfn = k_pass_cl<A, kDec, kRoleIntIn | kRoleIntOut>; break;
      default: break;
    }
    if (!pd.rt_layout) {
      const int shape = match_shape(pd);
      PassKernel sk = shape >= 0 ? shape_kernel_fixed_cl(kDec, shape, fixed_role(args)) : nullptr;
      if (sk != nullptr) kfn = sk;
    }
  }
  cudaError_t e = ensure_smem_limit((const void*)kfn, smem_max);
  if (e != cudaSuccess) return e;
  if (ntiles_total <= 0) return cudaSuccess;
  if (2 * ntiles_total > 0x7fffffffll) return cudaErrorInvalidValue;
  kfn<<<(unsigned)(2 * ntiles_total), kClThreads, smem, s>>>(pd, args);
  return cudaGetLastError();
}

template <class A, bool kDec>
cudaError_t launch_pass_t(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s) {
  const int threads = 1 << (pd.D - kRegBits);
  if constexpr (kClusterArith<A>) {
    if (pd.D == kMaxTileBits && pd.min_blocks == 2) return launch_pass_cl_t<A, kDec>(pd, args, ntiles_total, s);
  }
  const size_t vbytes = kBlockFixed<A> ? 16 : sizeof(typename A::V);
  // exchange area, reduction slots, class slots (block fixed point)
  const size_t smem = ((size_t)1 << pd.D) * vbytes + kRedBytes + (kBlockFixed<A> ? class_slot_bytes(pd) : 0);
  const int dmax = threads > kStdThreads ? kMaxTileBits : kStdTileBits;
  const size_t smem_max = ((size_t)1 << dmax) * vbytes + kRedBytes + (kBlockFixed<A> ? sizeof(int) << (dmax - 1) : 0);
  PassKernel kfn = nullptr;
  if (!pd.rt_layout) {
    const int shape = match_shape(pd);
    if constexpr (A::kFixed && kDec) {
      // one matrix, every tile: the persistent form that prefetches each
      // CTA's next tile while it finishes the current one
      const bool plain = args.ptrs == nullptr && !args.skip_zero && args.flags_in == nullptr &&
                         args.flags_out == nullptr && args.need == nullptr && !args.chunked;
      PassKernel pk = (plain && shape >= 0 && pd.min_blocks == kOccLow && threads <= kStdThreads)
                          ? shape_kernel_fixed_pf(shape, fixed_role(args)) : nullptr;
      if (pk != nullptr) {
        const size_t smem_pf = ((size_t)16 << pd.D) + kRedBytes + class_slot_bytes(pd);
        const size_t smem_pf_max = ((size_t)16 << kStdTileBits) + kRedBytes + (sizeof(int) << (kStdTileBits - 1));
        cudaError_t e = ensure_smem_limit((const void*)pk, smem_pf_max);
        if (e != cudaSuccess) return e;
        if (ntiles_total <= 0) return cudaSuccess;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pk, threads, smem_pf);
        if (e != cudaSuccess) return e;
        long long grid = (long long)device_sm_count() * (per_sm > 0 ? per_sm : 1);
        if (grid > ntiles_total) grid = ntiles_total;
        pk<<<(unsigned)grid, threads, smem_pf, s>>>(pd, args);
        return cudaGetLastError();
      }
    }
    if (shape >= 0) {
      if constexpr (A::kFixed) kfn = shape_kernel_fixed(kDec, shape, fixed_role(args), pd.min_blocks);
      else if constexpr (arith_code<A>() != kArithF64) kfn = shape_kernel_c64(arith_code<A>(), kDec, shape, pd.min_blocks);
    }
  }
  if (kfn == nullptr) {
    kfn = pick_pass_kernel<A, kDec, 0>(pd, threads);
    if constexpr (A::kFixed) {
      switch (fixed_role(args)) {
        case kRoleIntIn: kfn = pick_pass_kernel<A, kDec, kRoleIntIn>(pd, threads); break;
        case kRoleIntOut: kfn = pick_pass_kernel<A, kDec, kRoleIntOut>(pd, threads); break;
        case kRoleIntIn | kRoleIntOut: kfn = pick_pass_kernel<A, kDec, kRoleIntIn | kRoleIntOut>(pd, threads); break;
        default: break;
      }
    }
  }
  cudaError_t e = ensure_smem_limit((const void*)kfn, smem_max);
  if (e != cudaSuccess) return e;
  if (ntiles_total <= 0) return cudaSuccess;
  if (ntiles_total > 0x7fffffffll) return cudaErrorInvalidValue;
  kfn<<<(unsigned)ntiles_total, threads, smem, s>>>(pd, args);
  return cudaGetLastError();
}

// whole matrices of n <= 6 qubits: 4^n elements (16 bytes in registers for
// every arithmetic but plain fp32) and, block fixed point, 2^n class slots
template <class A, bool kDec>
cudaError_t launch_small_t(const SmallArgs& args, int blocks, int n_max, cudaStream_t s) {
  const size_t vbytes = A::kFixed ? 16 : sizeof(typename A::V);
  const size_t cls = A::kFixed ? sizeof(int) << n_max : 0;
  size_t smem = ((size_t)1 << (2 * n_max)) * vbytes + cls;
  if (smem < 256) smem = 256;
  const size_t smem_max = ((size_t)1 << 12) * vbytes + (A::kFixed ? sizeof(int) << 6 : 0);
  auto kfn = k_small<A, kDec>;
  cudaError_t e = ensure_smem_limit((const void*)kfn, smem_max);
  if (e != cudaSuccess) return e;
  if (blocks <= 0) return cudaSuccess;
  kfn<<<blocks, 128, smem, s>>>(args);
  return cudaGetLastError();
}

template <bool kDec>
cudaError_t launch_pass_pipe_t(const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s) {
  const int threads = 1 << (pd.D - kRegBits);
  // two tile buffers, reduction slots, class slots
  const size_t smem = ((size_t)32 << pd.D) + kRedBytes + class_slot_bytes(pd);
  const size_t smem_max = ((size_t)32 << kStdTileBits) + kRedBytes + (sizeof(int) << (kStdTileBits - 1));
  PassKernel kfn;
  switch (fixed_role(args)) {
    case kRoleIntIn: kfn = k_pass_pipe<kDec, kRoleIntIn>; break;
    case kRoleIntOut: kfn = k_pass_pipe<kDec, kRoleIntOut>; break;
    case kRoleIntIn | kRoleIntOut: kfn = k_pass_pipe<kDec, kRoleIntIn | kRoleIntOut>; break;
    default: kfn = k_pass_pipe<kDec, 0>; break;
  }
  cudaError_t e = ensure_smem_limit((const void*)kfn, smem_max);
  if (e != cudaSuccess) return e;
  const long long grid = pd.ntiles < nsm ? pd.ntiles : nsm;
  kfn<<<(unsigned)grid, threads, smem, s>>>(pd, args);
  return cudaGetLastError();
}

}  // namespace tpd
