// tpd_decompose_noalloc: the decomposition for callers that cannot allocate
// device memory (see include/tpd.h).  Its workspace is a fixed array in the
// library's own device memory instead of a caller-provided buffer.
#include <cuda_runtime.h>

#include <mutex>

#include "tpd.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB

// Lives in every GPU that loads the library, until the process exits.  In
// host code this name is only a host-side stand-in: the device address comes
// from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (resolved once
// per device, with that device current).
tpd_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TPD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return TPD_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TPD_OK;
}

}  // namespace

static_assert(kNoAllocScratchBytes == TPD_NOALLOC_SCRATCH_BYTES, "header and library disagree on the limit");

extern "C" {

tpd_status tpd_decompose_noalloc(void* A, int n, int dtype, const tpd_options* opt, void* stream) {
  const size_t need = tpd_workspace_size(n, dtype, opt);
  if (need > kNoAllocScratchBytes) return TPD_ERR_WORKSPACE;   // this size needs tpd_decompose
  // Looked up on every device's first call, whether or not this call needs
  // the array, so that the set-up (which loads this file's device code and,
  // under lazy module loading, the array with it) happens on that first call.
  void* scratch = nullptr;
  const tpd_status st = scratch_address(&scratch);
  if (st != TPD_OK) return st;
  return tpd_decompose(A, n, dtype, opt, need > 0 ? scratch : nullptr, need > 0 ? kNoAllocScratchBytes : 0,
                       stream);
}

}  // extern "C"
