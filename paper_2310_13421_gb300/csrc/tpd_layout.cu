// Output-layout conversion and sum-of-squares reduction (memory-bound helpers
// around the decomposition).
//
// Layouts.  RC: the weight of string t at flat index r*N + c with
// t_j = 2 r_{n-j} + c_{n-j} (where the butterfly leaves it).  STRING: at the
// base-4 index s = sum_j t_j 4^(n-j) (t_1 most significant), i.e. bit 2b+1 of
// s is row bit r_b and bit 2b is column bit c_b: s interleaves the bits of c
// and r.  A CTA converts one block of 2^k x 2^k (rows x columns) that shares
// all higher index bits: in RC it is 2^k runs of 2^k contiguous elements, in
// STRING one run of 4^k contiguous elements (its s-bits below 2k are the
// interleaved low bits).  Both sides are read and written in full 128-byte
// lines through a shared-memory transpose.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tpd_launch.h"

namespace tpd {

namespace {

// spread the low 16 bits of x to the even bit positions
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// gather the even bit positions of x into the low 16 bits
__device__ __forceinline__ uint32_t compact16(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0f0f0f0fu;
  x = (x | (x >> 4)) & 0x00ff00ffu;
  x = (x | (x >> 8)) & 0x0000ffffu;
  return x;
}

// blockDim.x = 4^k threads, one element each; block b = the higher bits.
template <class T>
__global__ void __launch_bounds__(256) k_layout(const T* __restrict__ src, T* __restrict__ dst, int n, int k,
                                                int to_string) {
  __shared__ T tile[256];
  const uint32_t K = 1u << k;
  const uint32_t tid = threadIdx.x;
  // higher bits of the block: rh, ch (n-k bits each), interleaved in STRING order
  const uint64_t b = blockIdx.x + (uint64_t)blockIdx.y * gridDim.x;
  const uint32_t ch = compact16((uint32_t)b) | (compact16((uint32_t)(b >> 32)) << 16);
  const uint32_t rh = compact16((uint32_t)(b >> 1)) | (compact16((uint32_t)(b >> 33)) << 16);
  const uint64_t N = 1ull << n;
  const uint64_t rc_base = ((uint64_t)rh << k) * N + ((uint64_t)ch << k);   // row rh*K, column ch*K
  const uint64_t s_base = b << (2 * k);
  // thread's element in RC order within the block: (r_low, c_low) = (tid / K, tid % K)
  const uint32_t rl = tid >> k, cl = tid & (K - 1);
  const uint32_t sl = spread16(cl) | (spread16(rl) << 1);   // its position in STRING order
  if (to_string) {
    tile[sl] = src[rc_base + (uint64_t)rl * N + cl];       // read RC rows
    __syncthreads();
    dst[s_base + tid] = tile[tid];                          // write the STRING run
  } else {
    tile[tid] = src[s_base + tid];                          // read the STRING run
    __syncthreads();
    dst[rc_base + (uint64_t)rl * N + cl] = tile[sl];        // write RC rows
  }
}

// Sum of |x|^2 over `count` complex elements in fp64, deterministic: a fixed
// grid of kSumBlocks CTAs each sums a fixed strided subset in a fixed order,
// then one CTA sums the partials in a fixed order.
constexpr int kSumBlocks = 1024;
constexpr int kSumThreads = 256;

// acc + |x|^2 as two fused multiply-adds: on GB300 the fp64 pipe, not
// memory, bounds this kernel, so it gets the fewest fp64 instructions
template <class T>
__device__ __forceinline__ double add_abs2(double acc, const T& x) {
  const double re = x.x, im = x.y;
  return __fma_rn(im, im, __fma_rn(re, re, acc));
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// Each thread keeps kSumUnroll loads in flight (independent partial sums,
// combined in a fixed order at the end).
constexpr int kSumUnroll = 8;

template <class T>
__global__ void __launch_bounds__(kSumThreads) k_sumsq_partial(const T* __restrict__ x, uint64_t count,
                                                               double* __restrict__ partial) {
  __shared__ double sh[kSumThreads / 32];
  double acc[kSumUnroll];
#pragma unroll
  for (int u = 0; u < kSumUnroll; ++u) acc[u] = 0.0;
  const uint64_t stride = (uint64_t)kSumBlocks * kSumThreads;
  uint64_t i = (uint64_t)blockIdx.x * kSumThreads + threadIdx.x;
  for (; i + (kSumUnroll - 1) * stride < count; i += kSumUnroll * stride) {
    T r[kSumUnroll];
#pragma unroll
    for (int u = 0; u < kSumUnroll; ++u) r[u] = __ldcs(x + i + u * stride);
#pragma unroll
    for (int u = 0; u < kSumUnroll; ++u) acc[u] = add_abs2(acc[u], r[u]);
  }
  for (; i < count; i += stride) acc[0] = add_abs2(acc[0], x[i]);   // tail: fewer than kSumUnroll
  double v = 0.0;
#pragma unroll
  for (int u = 0; u < kSumUnroll; ++u) v += acc[u];
  const double t = block_sum(v, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kSumThreads) k_sumsq_final(const double* __restrict__ partial,
                                                             double* __restrict__ out) {
  __shared__ double sh[kSumThreads / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < kSumBlocks; i += kSumThreads) v += partial[i];
  const double t = block_sum(v, sh);
  if (threadIdx.x == 0) *out = t;
}

template <class T>
cudaError_t launch_layout_t(const void* src, void* dst, int n, int k, int to_string, cudaStream_t s) {
  const uint64_t blocks = 1ull << (2 * (n - k));
  const unsigned gx = blocks > 65536 ? 65536u : (unsigned)blocks;
  const unsigned gy = (unsigned)(blocks / gx);
  k_layout<T><<<dim3(gx, gy), 1u << (2 * k), 0, s>>>(static_cast<const T*>(src), static_cast<T*>(dst), n, k,
                                                    to_string);
  return cudaGetLastError();
}

template <class T>
__global__ void __launch_bounds__(256) k_gather(const T* __restrict__ mat, const unsigned long long* __restrict__ pos,
                                                unsigned long long count, T* __restrict__ out) {
  const unsigned long long i = blockIdx.x * 256ull + threadIdx.x;
  if (i < count) out[i] = mat[pos[i]];
}

// ---------------------------------------------------------------- nonzero list
//
// The paper's output form (Alg. 1/2: the list L of strings with nonzero
// weight), in string order.  Blocks of 256 consecutive string indices (the
// blocks of k_layout) count their entries, one CTA turns the counts into
// offsets, and the blocks write their entries at those offsets: the order is
// the string order, independent of scheduling.
template <class T>
__device__ __forceinline__ bool keep(const T& w, double tol) {
  const double re = w.x, im = w.y;
  return !(fabs(re) <= tol && fabs(im) <= tol);            // NaN is kept
}

// element of the CTA's block held by this thread, in string order (s = s_base + tid)
template <class T>
__device__ __forceinline__ T string_element(const T* __restrict__ W, int n, int k, uint64_t b, uint32_t tid,
                                            T* tile) {
  const uint32_t K = 1u << k;
  const uint32_t ch = compact16((uint32_t)b) | (compact16((uint32_t)(b >> 32)) << 16);
  const uint32_t rh = compact16((uint32_t)(b >> 1)) | (compact16((uint32_t)(b >> 33)) << 16);
  const uint64_t N = 1ull << n;
  const uint64_t rc_base = ((uint64_t)rh << k) * N + ((uint64_t)ch << k);
  const uint32_t rl = tid >> k, cl = tid & (K - 1);
  const uint32_t sl = spread16(cl) | (spread16(rl) << 1);
  tile[sl] = W[rc_base + (uint64_t)rl * N + cl];              // coalesced RC read
  __syncthreads();
  return tile[tid];
}

template <class T>
__global__ void __launch_bounds__(256) k_nz_count(const T* __restrict__ W, int n, int k, double tol,
                                                  unsigned* __restrict__ counts) {
  __shared__ T tile[256];
  const uint64_t b = blockIdx.x + (uint64_t)blockIdx.y * gridDim.x;
  const T w = string_element(W, n, k, b, threadIdx.x, tile);
  const int c = __syncthreads_count(keep(w, tol));
  if (threadIdx.x == 0) counts[b] = (unsigned)c;
}

// exclusive scan of nb counts into offsets (one CTA of 1024 threads), total into *total
__global__ void __launch_bounds__(1024) k_nz_scan(const unsigned* __restrict__ counts, uint64_t nb,
                                                  unsigned long long* __restrict__ offsets,
                                                  unsigned long long* __restrict__ total) {
  __shared__ unsigned long long part[1024];
  const uint64_t per = (nb + 1023) / 1024;
  const uint64_t lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
  unsigned long long sum = 0;
  for (uint64_t i = lo; i < hi; ++i) sum += counts[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {                      // inclusive scan of the chunk sums
    const unsigned long long v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0ull;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0ull;
  for (uint64_t i = lo; i < hi; ++i) { offsets[i] = run; run += counts[i]; }
  if (threadIdx.x == 1023) *total = part[1023];
}

template <class T>
__global__ void __launch_bounds__(256) k_nz_write(const T* __restrict__ W, int n, int k, double tol,
                                                  const unsigned long long* __restrict__ offsets,
                                                  unsigned long long capacity,
                                                  unsigned long long* __restrict__ strings, T* __restrict__ weights) {
  __shared__ T tile[256];
  __shared__ unsigned warp_base[8];
  const uint64_t b = blockIdx.x + (uint64_t)blockIdx.y * gridDim.x;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T w = string_element(W, n, k, b, tid, tile);
  const bool kp = keep(w, tol);
  // blocks of n < 3 qubits have fewer than 32 threads
  const unsigned active = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  const unsigned ball = __ballot_sync(active, kp);
  if (lane == 0) warp_base[warp] = __popc(ball);
  __syncthreads();
  if (tid == 0) {
    unsigned acc = 0;
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) {
      const unsigned c = warp_base[i];
      warp_base[i] = acc;
      acc += c;
    }
  }
  __syncthreads();
  if (kp) {
    const unsigned long long pos = offsets[b] + warp_base[warp] + __popc(ball & ((1u << lane) - 1u));
    if (pos < capacity) {
      strings[pos] = (b << (2 * k)) + tid;
      weights[pos] = w;
    }
  }
}

template <class T>
cudaError_t launch_nonzero_t(const void* W, int n, double tol, unsigned long long* strings, void* weights,
                             unsigned long long capacity, unsigned long long* total, void* ws, cudaStream_t s) {
  const int k = n < 4 ? n : 4;
  const uint64_t blocks = 1ull << (2 * (n - k));
  const unsigned gx = blocks > 65536 ? 65536u : (unsigned)blocks;
  const unsigned gy = (unsigned)(blocks / gx);
  unsigned* counts = static_cast<unsigned*>(ws);
  unsigned long long* offsets =
      reinterpret_cast<unsigned long long*>(static_cast<char*>(ws) + ((blocks * 4 + 255) & ~255ull));
  const T* w = static_cast<const T*>(W);
  k_nz_count<T><<<dim3(gx, gy), 1u << (2 * k), 0, s>>>(w, n, k, tol, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nz_scan<<<1, 1024, 0, s>>>(counts, blocks, offsets, total);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_nz_write<T><<<dim3(gx, gy), 1u << (2 * k), 0, s>>>(w, n, k, tol, offsets, capacity, strings,
                                                      static_cast<T*>(weights));
  return cudaGetLastError();
}

}  // namespace

size_t nonzero_workspace_bytes(int n) {
  const int k = n < 4 ? n : 4;
  const uint64_t blocks = 1ull << (2 * (n - k));
  return ((blocks * 4 + 255) & ~255ull) + blocks * 8;
}

cudaError_t launch_nonzero(const void* W, int n, int elem_bytes, double tol, unsigned long long* strings,
                           void* weights, unsigned long long capacity, unsigned long long* total, void* ws,
                           cudaStream_t s) {
  return elem_bytes == 16 ? launch_nonzero_t<double2>(W, n, tol, strings, weights, capacity, total, ws, s)
                          : launch_nonzero_t<float2>(W, n, tol, strings, weights, capacity, total, ws, s);
}

cudaError_t launch_gather(const void* mat, const unsigned long long* pos, unsigned long long count, int elem_bytes,
                          void* out, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const unsigned long long blocks = (count + 255) / 256;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  if (elem_bytes == 16)
    k_gather<double2><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double2*>(mat), pos, count,
                                                       static_cast<double2*>(out));
  else
    k_gather<float2><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float2*>(mat), pos, count,
                                                      static_cast<float2*>(out));
  return cudaGetLastError();
}

cudaError_t launch_layout(const void* src, void* dst, int n, int elem_bytes, int to_string, cudaStream_t s) {
  const int k = n < 4 ? n : 4;      // 16 columns: 256 B (complex128) / 128 B (complex64) runs
  return elem_bytes == 16 ? launch_layout_t<double2>(src, dst, n, k, to_string, s)
                          : launch_layout_t<float2>(src, dst, n, k, to_string, s);
}

size_t sumsq_workspace_bytes() { return kSumBlocks * sizeof(double); }

cudaError_t launch_sumsq(const void* x, unsigned long long count, int elem_bytes, double* out, void* ws,
                         cudaStream_t s) {
  double* partial = static_cast<double*>(ws);
  if (elem_bytes == 16)
    k_sumsq_partial<double2><<<kSumBlocks, kSumThreads, 0, s>>>(static_cast<const double2*>(x), count, partial);
  else
    k_sumsq_partial<float2><<<kSumBlocks, kSumThreads, 0, s>>>(static_cast<const float2*>(x), count, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sumsq_final<<<1, kSumThreads, 0, s>>>(partial, out);
  return cudaGetLastError();
}

}  // namespace tpd
