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
// Publication: the CTA finishes an item's stores, barriers, and one thread
// (of warp 1, so that warp 0 goes straight on to the next item) issues a
// gpu-scope fence and adds the item's tile count to the counter; the waiting
// thread polls with ld.acquire.gpu and the CTA barriers before loading, and
// the loads of data written in this launch go through L2 (ld.global.cg).
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
    // the compiled layouts of the batch's largest matrices (n = 9, 10: a first
    // pass of 5 or 6 levels, a last pass of 4); identical results to the
    // run-time layout below
    const int sh = sg.shape[p];
    if (sh == kShapeFirst6 && role == kRoleIntOut) {
      pass_tile<A, kDec, kRoleIntOut, true>(GeoCT<ShapeT<kShapeFirst6>>(pd), args, matp, q_in, q_out, tile, smem,
                                            lane, warp);
      return;
    }
    if (sh == kShapeFirst5 && role == kRoleIntOut) {
      pass_tile<A, kDec, kRoleIntOut, true>(GeoCT<ShapeT<kShapeFirst5>>(pd), args, matp, q_in, q_out, tile, smem,
                                            lane, warp);
      return;
    }
    if (sh == kShapeMid4 && role == kRoleIntIn) {
      pass_tile<A, kDec, kRoleIntIn, true>(GeoCT<ShapeT<kShapeMid4>>(pd), args, matp, q_in, q_out, tile, smem, lane,
                                           warp);
      return;
    }
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
// block fixed point).  Thread 0 alone decodes each item (segment, pass,
// matrix, tiles), claims the next one and does the lookups, and hands the
// result to the CTA through shared memory behind one barrier; the claimed-ahead
// item waits in s_next (its own slot: kept out of registers, which the tile
// needs).
constexpr int kItemEnd = 0, kItemBucket = 1, kItemSkip = 2, kItemRun = 3;

template <class A, bool kDec>
__global__ void __launch_bounds__(kStdThreads, kOccLow) k_batch(const __grid_constant__ BatchParams bp) {
  using Store = typename A::Store;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_next;
  __shared__ int s_kind, s_si, s_p;
  __shared__ long long s_j, s_tile;
  __shared__ void* s_mat;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* status = bp.ctrl + kCtrlStatus;
  bool seen_bucket = false;                   // (thread 0's)
  if (tid == 0) s_next = atomicAdd(bp.ctrl + kCtrlWork, 1u);
  for (;;) {
    if (tid == 0) {
      const long long w = s_next;
      int kind = kItemRun, si = 0, p = 0;
      long long j = 0, tile = 0;
      if (w >= bp.total) {
        kind = kItemEnd;
      } else if (w == 0) {
        kind = kItemBucket;
        s_next = atomicAdd(bp.ctrl + kCtrlWork, 1u);
      } else {
        while (si + 1 < bp.nseg && w >= bp.seg[si + 1].first) ++si;
        const BatchSeg& sg = bp.seg[si];
        j = w - sg.first;                     // small matrices: one item each
        if (sg.kind == kSegPipe) {
          // item indices are below 2^31 (checked on the host): 32-bit division
          const unsigned rel = (unsigned)(w - sg.first);
          const unsigned ipp = (unsigned)(sg.tiles / sg.tpi);   // items per pass of a matrix
          const unsigned per_round = (unsigned)sg.npass * ipp;
          const unsigned round = rel / per_round;
          const unsigned sub = rel - round * per_round;
          p = (int)(sub / ipp);
          tile = (long long)(sub - (unsigned)p * ipp) * sg.tpi;
          j = (long long)round - (long long)p * sg.lag;
          if (j < 0 || j >= sg.nmat) {        // empty slot of the pipeline's ramp
            kind = kItemSkip;
            s_next = atomicAdd(bp.ctrl + kCtrlWork, 1u);
          }
        }
        if (kind == kItemRun) {
          // The claim, the status word, the matrix pointer (once the bucketing
          // is known to be done) and the first poll of the dependency are
          // issued back to back, so their round trips overlap; only a
          // dependency not yet met takes the polling loop.
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
          if (ok && sg.kind == kSegPipe && p > 0) {
            const unsigned* dep = bp.ctrl + kCtrlDone + sg.done + (long long)(p - 1) * sg.nmat + j;
            const unsigned need = (unsigned)(sg.tiles + sg.wait_extra);
            if (ld_acquire_gpu(dep) < need) ok = wait_count(dep, need, status);
          }
          seen_bucket = true;
          s_mat = reinterpret_cast<void*>(mp);
          s_next = nxt;
          if (!ok) kind = kItemSkip;
        }
      }
      s_kind = kind; s_si = si; s_p = p; s_j = j; s_tile = tile;
    }
    __syncthreads();
    const int kind = s_kind;
    if (kind == kItemEnd) break;
    if (kind == kItemBucket) {
      bucket_item(bp, tid, blockDim.x);       // ends with barriers
      if (tid == 0) seen_bucket = true;
      continue;
    }
    // The item's state is re-read from shared memory where it is used (the
    // s_* slots stay valid until the barrier that ends the item), so that
    // nothing but the tile counter stays live across a tile's registers.
    auto vol_int = [](const int& x) { return *reinterpret_cast<const volatile int*>(&x); };
    auto vol_ll = [](const long long& x) { return *reinterpret_cast<const volatile long long*>(&x); };
    if (kind == kItemRun) {
      const BatchSeg& sg = bp.seg[s_si];
      if (sg.kind == kSegSmall) {
        // whole small matrices of the complex64 fixed-point form: the compensated kernel
        using SmallA = typename std::conditional<A::kFixed32, F32CArith, A>::type;
        small_matrix<SmallA, kDec>(reinterpret_cast<Store*>(s_mat), sg.n, 0, bp.scale_mode, smem, tid, blockDim.x);
      } else {
        for (int k = 0;; ++k) {
          const BatchSeg& sgk = bp.seg[vol_int(s_si)];
          const int pk = vol_int(s_p);
          void* const matp = *reinterpret_cast<void* const volatile*>(&s_mat);
          batch_pass_tile<A, kDec>(sgk, pk, bp.desc[sgk.desc + pk], matp, vol_ll(s_j), vol_ll(s_tile) + k, smem,
                                   lane, warp);
          if (k + 1 >= bp.seg[vol_int(s_si)].tpi) break;
          __syncthreads();                     // the tile is done with shared memory
        }
      }
    }
    // Completion of a pass item, published by one thread of warp 1 (warp 0
    // goes on to the next item): its counter, read before the barrier that
    // frees the s_* slots for thread 0.
    unsigned* pub = nullptr;
    unsigned pub_n = 0;
    if (tid == 32 && kind == kItemRun) {
      const BatchSeg& sg = bp.seg[vol_int(s_si)];
      const int p = vol_int(s_p);
      if (sg.kind == kSegPipe && p + 1 < sg.npass) {
        pub = bp.ctrl + kCtrlDone + sg.done + (long long)p * sg.nmat + vol_ll(s_j);
        pub_n = (unsigned)sg.tpi;
      }
    }
    __syncthreads();                          // the item's stores are done (and smem is free)
    if (pub != nullptr) {
      __threadfence();
      atomicAdd(pub, pub_n);
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
