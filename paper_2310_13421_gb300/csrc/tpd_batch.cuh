// Persistent batched Pauli decomposition / composition: a whole batch of
// matrices of mixed qubit counts in ONE kernel launch (the batch form of
// Sec. III's algorithm: every matrix independently, Eqs. 3-5).
//
// CTAs claim work items in order from a device counter (the work list is
// described in tpd_launch.h: bucketing, then per qubit count the passes of
// its matrices software-pipelined so that a matrix's later passes find its
// data in L2, or whole small matrices).  A tile of pass p > 0 of matrix m
// reads what the tiles of pass p-1 of m wrote, so it waits until m's
// completion counter of pass p-1 is full.  All those tiles were claimed
// earlier (p-1 runs `lag` rounds ahead).
//
// Claim ahead: a CTA claims its next item when it starts the current one, so
// the counter's round trip overlaps the current item's lookups.  A CTA thus
// holds at most two claimed items, the current and the next (not begun), and
// only running CTAs hold claims.  Every item waits only on lower items, and
// the lowest unfinished item is always some CTA's current item (a CTA's next
// item lies above its current one), whose dependencies are all finished: the
// waits end.  They are nonetheless bounded: after kSpinLimit polls the CTA
// records TPD_ERR_TIMEOUT in the status word and skips the item, and every
// later item is skipped as soon as the status word is set, so the launch
// always finishes and the context stays usable.
//
// Publication: the CTA finishes a tile's stores, barriers, and one thread (of
// warp 1, so that warp 0 goes straight on to the next item) issues a
// gpu-scope fence and increments the counter; the waiting thread polls with
// ld.acquire.gpu and the CTA barriers before loading, and the loads of data
// written in this launch go through L2 (ld.global.cg).
#pragma once

#include <type_traits>

#include "tpd_kernels_impl.cuh"

namespace tpd {

constexpr unsigned kSpinLimit = 1u << 21;       // polls, with back-off up to 0.5 us: ~1-3 s

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// Wait until *p >= need.  false when the status word is (or becomes) set, or
// when the poll limit runs out (the status word is then set to TIMEOUT).
static __device__ __noinline__ bool wait_count(const unsigned* p, unsigned need, unsigned* status) {
  unsigned sleep_ns = 32;
  for (unsigned it = 0;; ++it) {
    if (ld_acquire_gpu(p) >= need) return true;
    if (ld_volatile(status) != 0) return false;
    if (it >= kSpinLimit) {
      atomicCAS(status, 0u, kBatchStatusTimeout);
      return false;
    }
    __nanosleep(sleep_ns);
    if (sleep_ns < 512) sleep_ns *= 2;
  }
}

// Work item 0: counting sort of the matrix indices by qubit count into
// bp.items, and of their pointers into bp.bptrs (ascending n, as the host
// laid out the segments), checking the counts against the host's histogram.
static __device__ __noinline__ void bucket_item(const BatchParams& bp, int tid, int nthr) {
  __shared__ int cnt[kBatchMaxN + 1];
  __shared__ int cur[kBatchMaxN + 1];
  __shared__ int bad;
  if (tid <= kBatchMaxN) cnt[tid] = 0;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int i = tid; i < bp.count; i += nthr) {
    const int n = __ldg(bp.ns + i);
    if (n >= 1 && n <= kBatchMaxN) atomicAdd(&cnt[n], 1);
    else bad = 1;
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int n = 0; n <= kBatchMaxN; ++n) {
      if (cnt[n] != bp.hist[n]) bad = 1;
      cur[n] = acc;
      acc += cnt[n];
    }
  }
  __syncthreads();
  if (!bad)
    for (int i = tid; i < bp.count; i += nthr) {
      const int n = __ldg(bp.ns + i);
      const int pos = atomicAdd(&cur[n], 1);
      bp.items[pos] = i;
      bp.bptrs[pos] = __ldg(reinterpret_cast<const unsigned long long*>(bp.ptrs) + i);
    }
  __syncthreads();
  if (tid == 0) {
    if (bad) atomicCAS(bp.ctrl + kCtrlStatus, 0u, kBatchStatusBadSizes);
    __threadfence();
    atomicExch(bp.ctrl + kCtrlBucket, 1u);
  }
}

template <class A, bool kDec>
__device__ __forceinline__ void batch_pass_tile(const BatchSeg& sg, int p, const PassDesc& pd, void* matp,
                                                long long j, long long tile, unsigned char* smem, int lane,
                                                int warp) {
  const PassArgs& args = sg.args[p];
  const int16_t* q_in = args.q_in ? args.q_in + j * args.q_in_stride : nullptr;
  int16_t* q_out = args.q_out ? args.q_out + j * args.q_out_stride : nullptr;
  if constexpr (A::kFixed) {
    const int role = (p > 0 ? kRoleIntIn : 0) | (p + 1 < sg.npass ? kRoleIntOut : 0);
    switch (role) {
      case 0: pass_tile<A, kDec, 0, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp); break;
      case kRoleIntIn:
        pass_tile<A, kDec, kRoleIntIn, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
        break;
      case kRoleIntOut:
        pass_tile<A, kDec, kRoleIntOut, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
        break;
      default:
        pass_tile<A, kDec, kRoleIntIn | kRoleIntOut, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
        break;
    }
  } else {
    pass_tile<A, kDec, 0, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
  }
}

// kStdThreads threads; dynamic shared memory: 2^12 x 16 bytes + kRedBytes + 2^11 ints (a
// D = 12 tile or a whole n <= 6 matrix, reduction slots, class slots of the
// block fixed point).  Thread 0 keeps the claimed-ahead item in s_next (its own
// slot: kept out of registers, which the tile needs) and hands it to the CTA
// through s_work at the top of the loop.
template <class A, bool kDec>
__global__ void __launch_bounds__(kStdThreads, kOccLow) k_batch(const __grid_constant__ BatchParams bp) {
  using Store = typename A::Store;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_work, s_next;
  __shared__ int s_ok;
  __shared__ void* s_mat;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* status = bp.ctrl + kCtrlStatus;
  bool seen_bucket = false;
  if (tid == 0) s_next = atomicAdd(bp.ctrl + kCtrlWork, 1u);
  for (;;) {
    if (tid == 0) s_work = s_next;
    __syncthreads();
    const long long w = s_work;
    if (w >= bp.total) break;
    if (w == 0) {
      if (tid == 0) s_next = atomicAdd(bp.ctrl + kCtrlWork, 1u);
      bucket_item(bp, tid, blockDim.x);       // ends with barriers: s_work may be rewritten after it
      seen_bucket = true;
      continue;
    }
    int si = 0;
    while (si + 1 < bp.nseg && w >= bp.seg[si + 1].first) ++si;
    const BatchSeg& sg = bp.seg[si];
    const long long rel = w - sg.first;
    long long j = rel, tile = 0;              // small matrices: one item each
    int p = 0;
    if (sg.kind == kSegPipe) {
      const long long per_round = (long long)sg.npass * sg.tiles;
      const long long round = rel / per_round;
      const long long sub = rel - round * per_round;
      p = (int)(sub / sg.tiles);
      tile = sub - p * sg.tiles;
      j = round - (long long)p * sg.lag;
      if (j < 0 || j >= sg.nmat) {            // empty slot of the pipeline's ramp
        if (tid == 0) s_next = atomicAdd(bp.ctrl + kCtrlWork, 1u);
        __syncthreads();                      // everyone has read s_work
        continue;
      }
    }
    unsigned* done = bp.ctrl + kCtrlDone + sg.done;
    if (tid == 0) {
      // The claim, the status word, the matrix pointer (once the bucketing is
      // known to be done) and the first poll of the dependency are issued
      // back to back, so their round trips overlap; only a dependency not yet
      // met takes the polling loop.
      const unsigned nxt = atomicAdd(bp.ctrl + kCtrlWork, 1u);   // claimed ahead
      const unsigned st0 = ld_volatile(status);
      unsigned long long mp = seen_bucket ? __ldcg(bp.bptrs + sg.item_start + j) : 0ull;
      bool ok = st0 == 0;
      if (ok && !seen_bucket) {
        // the bucketing sets the status word (sizes disagreeing) before it
        // releases its flag: read it again after acquiring the flag
        ok = wait_count(bp.ctrl + kCtrlBucket, 1u, status) && ld_volatile(status) == 0;
        if (ok) mp = __ldcg(bp.bptrs + sg.item_start + j);
      }
      if (ok && p > 0) {
        const unsigned* dep = done + (long long)(p - 1) * sg.nmat + j;
        const unsigned need = (unsigned)(sg.tiles + sg.wait_extra);
        if (ld_acquire_gpu(dep) < need) ok = wait_count(dep, need, status);
      }
      s_mat = reinterpret_cast<void*>(mp);
      s_ok = ok;
      s_next = nxt;
    }
    __syncthreads();
    seen_bucket = true;
    if (s_ok) {
      void* matp = s_mat;
      if (sg.kind == kSegSmall) {
        // whole small matrices of the complex64 fixed-point form: the compensated kernel
        using SmallA = typename std::conditional<A::kFixed32, F32CArith, A>::type;
        small_matrix<SmallA, kDec>(reinterpret_cast<Store*>(matp), sg.n, 0, bp.scale_mode, smem, tid, blockDim.x);
      } else {
        batch_pass_tile<A, kDec>(sg, p, bp.desc[sg.desc + p], matp, j, tile, smem, lane, warp);
      }
    }
    __syncthreads();                          // the tile's stores are done (and smem is free)
    if (tid == 32 && sg.kind == kSegPipe && p + 1 < sg.npass) {   // warp 0 goes on to the next item
      __threadfence();
      atomicAdd(done + (long long)p * sg.nmat + j, 1u);
    }
  }
}

template <class A, bool kDec>
cudaError_t launch_batch_t(const BatchParams& bp, int* grid_out, cudaStream_t s) {
  const size_t smem = ((size_t)16 << kStdTileBits) + kRedBytes + (sizeof(int) << (kStdTileBits - 1));
  auto kfn = k_batch<A, kDec>;
  cudaError_t e = ensure_smem_limit((const void*)kfn, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kStdThreads, smem)) != cudaSuccess) return e;
  long long grid = (long long)nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > bp.total) grid = bp.total;
  if (grid_out) *grid_out = (int)grid;
  kfn<<<(unsigned)grid, kStdThreads, smem, s>>>(bp);
  return cudaGetLastError();
}

}  // namespace tpd
