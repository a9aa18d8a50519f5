// Launch helpers shared by the per-storage-type kernel translation units.
#pragma once

#include <type_traits>

#include "tpd_launch.h"
#include "tpd_pass.cuh"

namespace tpd {

using PassKernel = void (*)(const PassDesc, const PassArgs);

// the instantiation for a pass's CTA size, occupancy and (fixed point) role
template <class A, bool kDec, int kRole>
PassKernel pick_pass_kernel(const PassDesc& pd, int threads) {
  if (threads > 256) return k_pass<A, kDec, 512, 1, kRole>;
  return pd.min_blocks >= 3 ? k_pass<A, kDec, 256, 3, kRole> : k_pass<A, kDec, 256, 2, kRole>;
}

// complex128 tiles of 2^13 elements planned as two-CTA clusters (min_blocks 2)
template <class A>
constexpr bool kClusterArith = std::is_same<A, FixedArith>::value || std::is_same<A, F64Arith>::value;

template <class A, bool kDec>
cudaError_t launch_pass_cl_t(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s) {
  const size_t smem = ((size_t)16 << (pd.D - 1)) + 256 + ((A::kFixed && args.q_in) ? sizeof(int) << kMaxPrevBits : 0);
  PassKernel kfn;
  if constexpr (A::kFixed) {
    switch ((args.q_in ? kRoleIntIn : 0) | (args.q_out ? kRoleIntOut : 0)) {
      case 0: kfn = k_pass_cl<A, kDec, 0>; break;
      case kRoleIntIn: kfn = k_pass_cl<A, kDec, kRoleIntIn>; break;
      case kRoleIntOut: kfn = k_pass_cl<A, kDec, kRoleIntOut>; break;
      default: kfn = k_pass_cl<A, kDec, kRoleIntIn | kRoleIntOut>; break;
    }
  } else {
    kfn = k_pass_cl<A, kDec, 0>;
  }
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ntiles_total <= 0) return cudaSuccess;
  if (2 * ntiles_total > 0x7fffffffll) return cudaErrorInvalidValue;
  kfn<<<(unsigned)(2 * ntiles_total), 256, smem, s>>>(pd, args);
  return cudaGetLastError();
}

template <class A, bool kDec>
cudaError_t launch_pass_t(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s) {
  const int threads = 1 << (pd.D - kRegBits);
  if constexpr (kClusterArith<A>) {
    if (pd.D == kMaxTileBits && pd.min_blocks == 2) return launch_pass_cl_t<A, kDec>(pd, args, ntiles_total, s);
  }
  const size_t vbytes = A::kFixed ? 16 : sizeof(typename A::V);
  // exchange area, reduction slots, and (fixed point reading int64 sums) the
  // gathered binary points -- the first pass keeps its occupancy without them
  const size_t smem =
      ((size_t)1 << pd.D) * vbytes + 256 + ((A::kFixed && args.q_in) ? sizeof(int) << kMaxPrevBits : 0);
  PassKernel kfn;
  if constexpr (A::kFixed) {
    switch ((args.q_in ? kRoleIntIn : 0) | (args.q_out ? kRoleIntOut : 0)) {
      case 0: kfn = pick_pass_kernel<A, kDec, 0>(pd, threads); break;
      case kRoleIntIn: kfn = pick_pass_kernel<A, kDec, kRoleIntIn>(pd, threads); break;
      case kRoleIntOut: kfn = pick_pass_kernel<A, kDec, kRoleIntOut>(pd, threads); break;
      default: kfn = pick_pass_kernel<A, kDec, kRoleIntIn | kRoleIntOut>(pd, threads); break;
    }
  } else {
    kfn = pick_pass_kernel<A, kDec, 0>(pd, threads);
  }
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (ntiles_total <= 0) return cudaSuccess;
  if (ntiles_total > 0x7fffffffll) return cudaErrorInvalidValue;
  kfn<<<(unsigned)ntiles_total, threads, smem, s>>>(pd, args);
  return cudaGetLastError();
}

template <class A, bool kDec>
cudaError_t launch_small_t(const SmallArgs& args, int blocks, int n_max, cudaStream_t s) {
  const size_t vbytes = A::kFixed ? 16 : sizeof(typename A::V);
  size_t smem = ((size_t)1 << (2 * n_max)) * vbytes;
  if (smem < 256) smem = 256;
  auto kfn = k_small<A, kDec>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (blocks <= 0) return cudaSuccess;
  kfn<<<blocks, 128, smem, s>>>(args);
  return cudaGetLastError();
}

template <bool kDec>
cudaError_t launch_pass_pipe_t(const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s) {
  const int threads = 1 << (pd.D - kRegBits);
  // two tile buffers, reduction slots, gathered binary points (passes reading int64 sums)
  const size_t smem = ((size_t)32 << pd.D) + 256 + (args.q_in ? sizeof(int) << kMaxPrevBits : 0);
  PassKernel kfn;
  switch ((args.q_in ? kRoleIntIn : 0) | (args.q_out ? kRoleIntOut : 0)) {
    case 0: kfn = k_pass_pipe<kDec, 0>; break;
    case kRoleIntIn: kfn = k_pass_pipe<kDec, kRoleIntIn>; break;
    case kRoleIntOut: kfn = k_pass_pipe<kDec, kRoleIntOut>; break;
    default: kfn = k_pass_pipe<kDec, kRoleIntIn | kRoleIntOut>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = pd.ntiles < nsm ? pd.ntiles : nsm;
  kfn<<<(unsigned)grid, threads, smem, s>>>(pd, args);
  return cudaGetLastError();
}

}  // namespace tpd
