// complex128 kernels: exact block fixed point and IEEE fp64 arithmetic.
#include "tpd_kernels_impl.cuh"

namespace tpd {

cudaError_t launch_pass_c128(int arith, bool dec, const PassDesc& pd, const PassArgs& args,
                             long long ntiles_total, cudaStream_t s) {
  if (arith == kArithFixed)
    return dec ? launch_pass_t<FixedArith, true>(pd, args, ntiles_total, s)
               : launch_pass_t<FixedArith, false>(pd, args, ntiles_total, s);
  return dec ? launch_pass_t<F64Arith, true>(pd, args, ntiles_total, s)
             : launch_pass_t<F64Arith, false>(pd, args, ntiles_total, s);
}

cudaError_t launch_small_c128(int arith, bool dec, const SmallArgs& args, int blocks, int n_max, cudaStream_t s) {
  if (arith == kArithFixed)
    return dec ? launch_small_t<FixedArith, true>(args, blocks, n_max, s)
               : launch_small_t<FixedArith, false>(args, blocks, n_max, s);
  return dec ? launch_small_t<F64Arith, true>(args, blocks, n_max, s)
             : launch_small_t<F64Arith, false>(args, blocks, n_max, s);
}

cudaError_t launch_pass_pipe_c128(bool dec, const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s) {
  const int threads = 1 << (pd.D - kRegBits);
  const size_t smem = ((size_t)32 << pd.D) + 256;   // two tile buffers + reduction slots
  const int role = (args.q_in ? kRoleIntIn : 0) | (args.q_out ? kRoleIntOut : 0);
  PassKernel kfn;
  switch (role) {
    case 0: kfn = dec ? k_pass_pipe<true, 0> : k_pass_pipe<false, 0>; break;
    case kRoleIntIn: kfn = dec ? k_pass_pipe<true, kRoleIntIn> : k_pass_pipe<false, kRoleIntIn>; break;
    case kRoleIntOut: kfn = dec ? k_pass_pipe<true, kRoleIntOut> : k_pass_pipe<false, kRoleIntOut>; break;
    default: kfn = dec ? k_pass_pipe<true, 3> : k_pass_pipe<false, 3>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long grid = pd.ntiles < nsm ? pd.ntiles : nsm;
  kfn<<<(unsigned)grid, threads, smem, s>>>(pd, args);
  return cudaGetLastError();
}

// One CTA buckets matrix indices by qubit count (counting sort in shared memory).
__global__ void __launch_bounds__(1024) k_bucket(const int* __restrict__ ns, int count, int* __restrict__ items,
                                                 int* __restrict__ offsets) {
  __shared__ int cnt[32];
  __shared__ int cur[32];
  const int tid = threadIdx.x;
  if (tid < 32) cnt[tid] = 0;
  __syncthreads();
  for (int i = tid; i < count; i += blockDim.x) {
    const int n = ns[i];
    if (n >= 0 && n < 32) atomicAdd(&cnt[n], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int n = 0; n < 32; ++n) { offsets[n] = acc; cur[n] = acc; acc += cnt[n]; }
    offsets[32] = acc;
  }
  __syncthreads();
  for (int i = tid; i < count; i += blockDim.x) {
    const int n = ns[i];
    if (n >= 0 && n < 32) items[atomicAdd(&cur[n], 1)] = i;
  }
}

cudaError_t launch_bucket(const int* ns_dev, int count, int* out_items, int* out_offsets, int* /*scratch*/,
                          cudaStream_t s) {
  k_bucket<<<1, 1024, 0, s>>>(ns_dev, count, out_items, out_offsets);
  return cudaGetLastError();
}

}  // namespace tpd
