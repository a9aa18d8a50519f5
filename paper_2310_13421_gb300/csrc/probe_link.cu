// Host link probe for the end-to-end call (tpd_decompose_host): bandwidth of
// host<->device transfers of a 4 GiB buffer through the copy engines
// (cudaMemcpyAsync; one stream, four streams, both directions at once) and
// through a kernel that reads or writes mapped pinned host memory directly,
// timed with CUDA events.  A device-to-device copy kernel is the reference.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o probe_link probe_link.cu
#include <cuda_runtime.h>
#include <cstdio>
#include <cstdlib>

__global__ void k_copy(const int4* __restrict__ src, int4* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

#define CK(x) do { cudaError_t ck_ = (x); if (ck_ != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(ck_), __LINE__); return 1; } } while (0)

int main() {
  const size_t bytes = (size_t)1 << 32;   // 4 GiB
  const size_t n = bytes / 16;
  int dev = 0, nsm = 0, pma = 0, pmaht = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, dev));
  CK(cudaDeviceGetAttribute(&pmaht, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev));
  printf("sms %d pageableMemoryAccess %d usesHostPageTables %d\n", nsm, pma, pmaht);
  void *h_in = nullptr, *h_out = nullptr, *d = nullptr, *d2 = nullptr;
  CK(cudaHostAlloc(&h_in, bytes, cudaHostAllocMapped));
  CK(cudaHostAlloc(&h_out, bytes, cudaHostAllocMapped));
  CK(cudaMalloc(&d, bytes));
  CK(cudaMalloc(&d2, bytes));
  memset(h_in, 1, bytes);
  memset(h_out, 0, bytes);
  void *hin_d = nullptr, *hout_d = nullptr;
  CK(cudaHostGetDevicePointer(&hin_d, h_in, 0));
  CK(cudaHostGetDevicePointer(&hout_d, h_out, 0));
  cudaStream_t s[4];
  for (int i = 0; i < 4; ++i) CK(cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
  auto timeit = [&](const char* name, auto fn) -> int {
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaDeviceSynchronize());
      CK(cudaEventRecord(a, s[0]));
      fn();
      for (int i = 1; i < 4; ++i) { cudaEvent_t ev; CK(cudaEventCreate(&ev)); CK(cudaEventRecord(ev, s[i])); CK(cudaStreamWaitEvent(s[0], ev, 0)); CK(cudaEventDestroy(ev)); }
      CK(cudaEventRecord(b, s[0]));
      CK(cudaEventSynchronize(b));
      float ms = 0; CK(cudaEventElapsedTime(&ms, a, b));
      printf("%-36s %8.3f ms  %7.1f GB/s\n", name, ms, bytes / (ms * 1e-3) / 1e9);
    }
    return 0;
  };
  const unsigned grid = nsm * 8;
  timeit("memcpy H2D (1 stream)", [&] { cudaMemcpyAsync(d, h_in, bytes, cudaMemcpyHostToDevice, s[0]); });
  timeit("memcpy D2H (1 stream)", [&] { cudaMemcpyAsync(h_out, d, bytes, cudaMemcpyDeviceToHost, s[0]); });
  timeit("memcpy H2D (4 streams, 4 chunks)", [&] {
    for (int i = 0; i < 4; ++i) cudaMemcpyAsync((char*)d + i * bytes / 4, (char*)h_in + i * bytes / 4, bytes / 4, cudaMemcpyHostToDevice, s[i]); });
  timeit("memcpy D2H (4 streams, 4 chunks)", [&] {
    for (int i = 0; i < 4; ++i) cudaMemcpyAsync((char*)h_out + i * bytes / 4, (char*)d + i * bytes / 4, bytes / 4, cudaMemcpyDeviceToHost, s[i]); });
  timeit("memcpy H2D + D2H concurrently", [&] {
    cudaMemcpyAsync(d, h_in, bytes, cudaMemcpyHostToDevice, s[0]);
    cudaMemcpyAsync(h_out, d2, bytes, cudaMemcpyDeviceToHost, s[1]); });
  timeit("kernel read host -> device", [&] { k_copy<<<grid, 256, 0, s[0]>>>((const int4*)hin_d, (int4*)d, n); });
  timeit("kernel device -> write host", [&] { k_copy<<<grid, 256, 0, s[0]>>>((const int4*)d, (int4*)hout_d, n); });
  timeit("kernel device -> device", [&] { k_copy<<<grid, 256, 0, s[0]>>>((const int4*)d, (int4*)d2, n); });
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  // check the kernel copies
  const unsigned char* o = (const unsigned char*)h_out;
  size_t bad = 0;
  for (size_t i = 0; i < bytes; i += 4099) bad += o[i] != 1;
  printf("check: %zu bad samples\n", bad);
  return 0;
}
