// complex128 kernels: IEEE fp64 passes, whole small matrices, batching
// helpers; the block-fixed-point passes sit in tpd_kernels_fixed_{dec,com}.cu.
#include "tpd_kernels_impl.cuh"

#include <map>
#include <mutex>
#include <utility>

namespace tpd {

cudaError_t ensure_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;   // (kernel, device) -> limit set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[std::make_pair(fn, dev)];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int device_sm_count() {
  static std::mutex mu;
  static std::map<int, int> count;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(mu);
  int& c = count[dev];
  if (c == 0 && cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) c = 0;
  return c > 0 ? c : 1;
}

cudaError_t launch_pass_fixed_dec(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s);
cudaError_t launch_pass_fixed_com(const PassDesc& pd, const PassArgs& args, long long ntiles_total, cudaStream_t s);
cudaError_t launch_pass_pipe_fixed_dec(const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s);
cudaError_t launch_pass_pipe_fixed_com(const PassDesc& pd, const PassArgs& args, int nsm, cudaStream_t s);

cudaError_t launch_pass_c128(int arith, bool dec, const PassDesc& pd, const PassArgs& args,
                             long long ntiles_total, cudaStream_t s) {
  if (arith == kArithFixed)
    return dec ? launch_pass_fixed_dec(pd, args, ntiles_total, s) : launch_pass_fixed_com(pd, args, ntiles_total, s);
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
  return dec ? launch_pass_pipe_fixed_dec(pd, args, nsm, s) : launch_pass_pipe_fixed_com(pd, args, nsm, s);
}

// One CTA buckets matrix indices by qubit count (counting sort in shared memory).
__global__ void __launch_bounds__(1024) k_bucket(const int* __restrict__ ns, int count, const BucketHist hist,
                                                 int* __restrict__ items, unsigned* __restrict__ status) {
  __shared__ int cnt[kBatchMaxN + 1];
  __shared__ int cur[kBatchMaxN + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid <= kBatchMaxN) cnt[tid] = 0;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int i = tid; i < count; i += blockDim.x) {
    const int n = ns[i];
    if (n >= 1 && n <= kBatchMaxN) atomicAdd(&cnt[n], 1);
    else bad = 1;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int n = 0; n <= kBatchMaxN; ++n) {
      if (cnt[n] != hist.h[n]) bad = 1;
      cur[n] = acc;
      acc += cnt[n];
    }
    if (bad) atomicCAS(status, 0u, kBatchStatusBadSizes);
  }
  __syncthreads();
  for (int i = tid; i < count; i += blockDim.x) {
    if (bad) items[i] = -1;
    else items[atomicAdd(&cur[ns[i]], 1)] = i;
  }
}

cudaError_t launch_bucket(const int* ns_dev, int count, const BucketHist& hist, int* out_items, unsigned* status,
                          cudaStream_t s) {
  k_bucket<<<1, 1024, 0, s>>>(ns_dev, count, hist, out_items, status);
  return cudaGetLastError();
}

}  // namespace tpd
