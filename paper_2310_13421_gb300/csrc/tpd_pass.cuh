// One pass of the Pauli butterfly over a group of qubit levels (Sec. III,
// Eqs. 3-5), in place, one CTA per tile.  See tpd_plan.h for tiles and stages
// and tpd_arith.cuh for the arithmetics.
//
// Flow of a CTA:
//   1. skip the tile if the previous pass flagged it all-zero (zero-CMW
//      pruning of Alg. 1/2: a zero block has only zero weights below it);
//   2. load its 16 elements per thread from HBM with the stage-0 mapping
//      (lanes on the lowest tile bits: 128-byte runs);
//   3. fixed point: CTA-wide max exponent -> common binary point; optional
//      all-zero test (then nothing is written);
//   4. per stage: apply the stage's levels in registers / across lanes, then
//      exchange through shared memory into the next stage's mapping;
//   5. round back to the storage type, store in place with the last stage's
//      mapping, and flag the next pass's tiles that received a nonzero.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "tpd_arith.cuh"
#include "tpd_launch.h"
#include "tpd_plan.h"

namespace tpd {


constexpr uint32_t kFull = 0xffffffffu;

// -------------------------------------------------------------- two-CTA clusters
//
// A complex128 tile of 2^13 elements runs as a cluster of two 256-thread CTAs
// (kCl = true) instead of one 512-thread CTA: the stage layouts are the
// 512-thread ones, with the CTA's rank in the cluster as the highest warp
// bit, so the register budget stays at two CTAs per SM.  Each CTA keeps half
// of the exchange area -- the elements whose tile bit on that warp bit (in
// the stage being entered) equals its rank -- and writes the other half into
// its peer's shared memory.  Protocol per tile: every thread arrives
// (relaxed) at the cluster barrier on entry and waits right after issuing its
// global loads, so the peer is running before any access to its shared
// memory; every exchange and the block-wide reduction end their remote
// writes with a full cluster barrier before anything reads them, and no
// remote access follows the last barrier, so either CTA may exit after it.
// Decisions that end a tile early (all-zero, Inf/NaN) are taken from
// cluster-wide values, so both CTAs take the same path and meet the same
// barriers.
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}
// the same shared-memory location in the other CTA of the cluster
template <class T>
__device__ __forceinline__ T* peer_smem(T* p) {
  return cooperative_groups::this_cluster().map_shared_rank(p, cluster_rank() ^ 1u);
}

// Loads of data a pass reads.  kCg = false: the read-only path (ld.global.nc),
// valid when nothing in the same launch writes the data; kCg = true: loads
// cached in L2 only (ld.global.cg), for the persistent batched kernel whose
// later passes read what other CTAs of the same launch wrote (after an
// acquire on their completion counters).
template <bool kCg, class T>
__device__ __forceinline__ T ld_in(const T* p) {
  if constexpr (kCg) return __ldcg(p);
  else return __ldg(p);
}

// 2^e as a double, built from its bits (normal range only)
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}

__device__ __forceinline__ long long thread_goff(const PassDesc& pd, const Stage& st, int lane, int warp) {
  long long g = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i)
    if ((lane >> i) & 1) g += 1ll << pd.gbit[st.lane[i]];
  for (int i = 0; i < pd.D - kMinTileBits; ++i)
    if ((warp >> i) & 1) g += 1ll << pd.gbit[st.warp[i]];
  return g;
}

__device__ __forceinline__ int thread_sidx(const PassDesc& pd, const Stage& st, int lane, int warp) {
  int s = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i) s |= ((lane >> i) & 1) << st.lane[i];
  for (int i = 0; i < pd.D - kMinTileBits; ++i) s |= ((warp >> i) & 1) << st.warp[i];
  return s;
}

__device__ __forceinline__ int thread_next(const PassDesc& pd, const Stage& st, int lane, int warp) {
  int s = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i)
    if ((lane >> i) & 1) s += pd.next_w[st.lane[i]];
  for (int i = 0; i < pd.D - kMinTileBits; ++i)
    if ((warp >> i) & 1) s += pd.next_w[st.warp[i]];
  return s;
}

// offset of register e from 4 per-bit weights (e is a compile-time constant after unrolling)
template <class T>
__device__ __forceinline__ T reg_off(int e, T w0, T w1, T w2, T w3) {
  return ((e & 1) ? w0 : T(0)) + ((e & 2) ? w1 : T(0)) + ((e & 4) ? w2 : T(0)) + ((e & 8) ? w3 : T(0));
}

// -------------------------------------------------------------- levels

// i (a - b): the arithmetic's fused form where it has one
template <class A, class = void>
struct HasIsub : std::false_type {};
template <class A>
struct HasIsub<A, decltype((void)A::isub(typename A::V{}, typename A::V{}))> : std::true_type {};
template <class A>
__device__ __forceinline__ typename A::V isub(typename A::V a, typename A::V b) {
  if constexpr (HasIsub<A>::value) return A::isub(a, b);
  else return A::mul_i(A::sub(a, b));
}

// In-register level: register bits RC (column) and RR (row).
template <class A, bool kDec, int RC, int RR>
__device__ __forceinline__ void pair_level(typename A::V (&v)[kElems]) {
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    if ((e >> RC) & 1) continue;
    if ((e >> RR) & 1) continue;
    const int e01 = e | (1 << RC), e10 = e | (1 << RR), e11 = e | (1 << RC) | (1 << RR);
    const typename A::V a00 = v[e], a01 = v[e01], a10 = v[e10], a11 = v[e11];
    if (kDec) {
      v[e] = A::add(a00, a11);                  // I
      v[e01] = A::add(a01, a10);                // X
      v[e10] = isub<A>(a01, a10);               // Y
      v[e11] = A::sub(a00, a11);                // Z
    } else {
      const typename A::V iy = A::mul_i(a10);   // positions hold I, X, Y, Z
      v[e] = A::add(a00, a11);                  // I + Z
      v[e01] = A::sub(a01, iy);                 // X - iY
      v[e10] = A::add(a01, iy);                 // X + iY
      v[e11] = A::sub(a00, a11);                // I - Z
    }
  }
}

// Cross-lane level: column bit on lane bit `lbit`, row bit on register bit RB.
// Both lanes of a pair compute the same sums as pair_level, in the same order.
template <class A, bool kDec, int RB>
__device__ __forceinline__ void shfl_level(typename A::V (&v)[kElems], int lbit, int lane) {
  const int mask = 1 << lbit;
  const bool cb = (lane >> lbit) & 1;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    if ((e >> RB) & 1) continue;
    const int e1i = e | (1 << RB);
    const typename A::V e0 = v[e], e1 = v[e1i];
    const typename A::V p0 = A::shfl(e0, mask), p1 = A::shfl(e1, mask);
    if (kDec) {
      // column 0 holds a00 (row 0), a10 (row 1); column 1 holds a01, a11
      v[e] = A::add(e0, p1);                    // I at (0,0) / X at (0,1)
      const typename A::V d = A::sub(p0, e1);   // a01 - a10 / a00 - a11
      v[e1i] = cb ? d : A::mul_i(d);            // Y at (1,0) / Z at (1,1)
    } else {
      // column 0 holds I, Y; column 1 holds X, Z
      const typename A::V t1 = cb ? A::mul_mi(p1) : p1;
      const typename A::V t2 = cb ? A::neg(e1) : A::mul_i(e1);
      v[e] = A::add(e0, t1);                    // I + Z / X - iY
      v[e1i] = A::add(p0, t2);                  // X + iY / I - Z
    }
  }
}

template <class A, bool kDec>
__device__ __forceinline__ void stage_levels(typename A::V (&v)[kElems], const Stage& st, int lane) {
  if (st.npair >= 1) pair_level<A, kDec, 0, 1>(v);
  if (st.npair >= 2) pair_level<A, kDec, 2, 3>(v);
  const int r0 = 2 * st.npair;
  for (int s = 0; s < st.nshfl; ++s) {
    const int lb = st.shfl_lane[s];
    switch (r0 + s) {
      case 0: shfl_level<A, kDec, 0>(v, lb, lane); break;
      case 1: shfl_level<A, kDec, 1>(v, lb, lane); break;
      case 2: shfl_level<A, kDec, 2>(v, lb, lane); break;
      default: shfl_level<A, kDec, 3>(v, lb, lane); break;
    }
  }
}

// Shared-memory exchange from stage `a`'s mapping to stage `b`'s.  kCl: the
// tile is split over a two-CTA cluster (see above): an element goes to the
// CTA whose rank equals its tile bit on b's highest warp bit, at its tile
// index with that bit removed.
template <bool kCl = false, class V>
__device__ __forceinline__ void exchange(V (&v)[kElems], const PassDesc& pd, const Stage& a,
                                         const Stage& b, V* sm, int lane, int warp, bool sync_first) {
  if constexpr (kCl) {
    if (sync_first) cluster_sync();           // both CTAs have read the previous exchange
    const int cb = b.warp[3];                 // >= 3: lanes hold tile bits 0..2
    const int lowm = (1 << cb) - 1;
    auto squeeze = [&](int x) { return (x & lowm) | ((x >> 1) & ~lowm); };
    V* const mine = sm;
    V* const peer = peer_smem(sm);
    const int rank = (int)cluster_rank();
    {
      const int t = thread_sidx(pd, a, lane, warp);
      const int lt = squeeze(t), ot = (t >> cb) & 1;
      const int w0 = squeeze(1 << a.reg[0]), w1 = squeeze(1 << a.reg[1]);
      const int w2 = squeeze(1 << a.reg[2]), w3 = squeeze(1 << a.reg[3]);
      const int o0 = a.reg[0] == cb, o1 = a.reg[1] == cb, o2 = a.reg[2] == cb, o3 = a.reg[3] == cb;
#pragma unroll
      for (int e = 0; e < kElems; ++e) {
        const int own = ot ^ reg_off(e, o0, o1, o2, o3);
        (own == rank ? mine : peer)[lt + reg_off(e, w0, w1, w2, w3)] = v[e];
      }
    }
    cluster_sync();
    {
      const int lt = squeeze(thread_sidx(pd, b, lane, warp));
      const int w0 = squeeze(1 << b.reg[0]), w1 = squeeze(1 << b.reg[1]);
      const int w2 = squeeze(1 << b.reg[2]), w3 = squeeze(1 << b.reg[3]);
#pragma unroll
      for (int e = 0; e < kElems; ++e) v[e] = mine[lt + reg_off(e, w0, w1, w2, w3)];
    }
    return;
  }
  if (sync_first) __syncthreads();
  {
    const int t = thread_sidx(pd, a, lane, warp);
    const int w0 = 1 << a.reg[0], w1 = 1 << a.reg[1], w2 = 1 << a.reg[2], w3 = 1 << a.reg[3];
#pragma unroll
    for (int e = 0; e < kElems; ++e) sm[t + reg_off(e, w0, w1, w2, w3)] = v[e];
  }
  __syncthreads();
  {
    const int t = thread_sidx(pd, b, lane, warp);
    const int w0 = 1 << b.reg[0], w1 = 1 << b.reg[1], w2 = 1 << b.reg[2], w3 = 1 << b.reg[3];
#pragma unroll
    for (int e = 0; e < kElems; ++e) v[e] = sm[t + reg_off(e, w0, w1, w2, w3)];
  }
}

// Stages, rounding and the in-place store, for arithmetic A on loaded data.
template <class A, bool kDec, bool kCl = false, class Raw>
__device__ __forceinline__ void finish_tile(const PassDesc& pd, const PassArgs& args, void* matp,
                                            const Raw (&raw)[kElems], double mul, long long base,
                                            int nbase, unsigned char* smem, int lane, int warp) {
  using V = typename A::V;
  using Store = typename A::Store;
  V v[kElems];
#pragma unroll
  for (int e = 0; e < kElems; ++e) v[e] = A::load(raw[e]);
  V* sm = reinterpret_cast<V*>(smem);
  for (int s = 0; s < pd.nstage; ++s) {
    if (s > 0) exchange<kCl>(v, pd, pd.st[s - 1], pd.st[s], sm, lane, warp, s > 1);
    stage_levels<A, kDec>(v, pd.st[s], lane);
  }
  const Stage& sl = pd.st[pd.nstage - 1];
  Store* mat = reinterpret_cast<Store*>(matp);
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, sl, lane, warp);
  const uint32_t w0 = 1u << pd.gbit[sl.reg[0]], w1 = 1u << pd.gbit[sl.reg[1]];
  const uint32_t w2 = 1u << pd.gbit[sl.reg[2]], w3 = 1u << pd.gbit[sl.reg[3]];
  const bool flags = args.flags_out != nullptr;
  int nt = 0, n0 = 0, n1 = 0, n2 = 0, n3 = 0;
  bool lanes_inside = true;
  if (flags) {
    nt = nbase + thread_next(pd, sl, lane, warp);
    n0 = pd.next_w[sl.reg[0]]; n1 = pd.next_w[sl.reg[1]];
    n2 = pd.next_w[sl.reg[2]]; n3 = pd.next_w[sl.reg[3]];
#pragma unroll
    for (int i = 0; i < kLaneBits; ++i) lanes_inside &= (pd.next_w[sl.lane[i]] == 0);
  }
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    const Store o = A::store(v[e], OutScale{0, 1.0}, mul);
    const bool nz = flags && A::nonzero(o);
    mat[g + reg_off(e, w0, w1, w2, w3)] = o;
    if (flags) {
      const int id = nt + reg_off(e, n0, n1, n2, n3);
      if (lanes_inside) {
        if (__any_sync(kFull, nz) && lane == 0) args.flags_out[id] = 1;
      } else if (nz) {
        args.flags_out[id] = 1;
      }
    }
  }
}

template <bool kCg = false, class Store>
__device__ __forceinline__ void load_tile(const PassDesc& pd, const void* matp, long long base, int lane, int warp,
                                          Store (&raw)[kElems]) {
  const Stage& s0 = pd.st[0];
  const Store* mat = reinterpret_cast<const Store*>(matp);
  // element indices in 32 bits: a matrix has at most 4^16 = 2^32 elements
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, s0, lane, warp);
  const uint32_t w0 = 1u << pd.gbit[s0.reg[0]], w1 = 1u << pd.gbit[s0.reg[1]];
  const uint32_t w2 = 1u << pd.gbit[s0.reg[2]], w3 = 1u << pd.gbit[s0.reg[3]];
#pragma unroll
  for (int e = 0; e < kElems; ++e) raw[e] = ld_in<kCg>(mat + (g + reg_off(e, w0, w1, w2, w3)));
}

// ============================================================== fixed point
//
// A pass of the complex128 fixed-point path reads either IEEE doubles (the
// first pass) or the int64 sums the previous pass stored in place together
// with one binary point per previous tile (value = v * 2^q), and writes
// either int64 sums plus its own tiles' binary points (a pass that does not
// end the plan) or IEEE doubles rounded once (the last pass).  Between
// passes the data stay 16-byte int64 pairs, so only the first pass converts
// from double and only the last back to double.
//
// Headroom: every stored |v| < 2^62.  A reading pass of K levels aligns all
// its elements to q_in = max(q_src) + K, i.e. shifts each right by at least
// K bits (toward zero, so that conjugate inputs stay exactly conjugate),
// after which 2^K-term sums stay below 2^62.

__device__ __forceinline__ bool q_is_valid(int q) { return q > kQValidMin; }

// v / 2^sh rounded toward zero (sh >= 0; 0 once sh >= 64)
__device__ __forceinline__ long long shr_tz(long long v, unsigned sh) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  unsigned long long a = ((unsigned long long)v ^ s) - s;
  asm("shr.b64 %0, %0, %1;" : "+l"(a) : "r"(sh));   // PTX clamps the amount at 64
  return (long long)((a ^ s) - s);
}

// floor(v / 2^sh) (sh >= 0; 0 or -1 once sh >= 64)
__device__ __forceinline__ long long shr_floor(long long v, unsigned sh) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(sh));   // PTX clamps the amount at 64
  return r;
}

// Alignment of the int64 sums of a previous pass to the tile's binary point.
// Rounding toward minus infinity costs 2-3 instructions against ~11 for
// toward zero; the error is below 2^-(62-K) of the tile's largest element.
#ifdef TPD_ALIGN_TOWARD_ZERO
#define TPD_ALIGN shr_tz
#else
#define TPD_ALIGN shr_floor
#endif

// Which unit converts each component between double and int64 (identical
// results either way): integer instructions, or the fp64 conversion unit.
#if defined(TPD_CVT_BOTH)
#define TPD_TO_FIXED_RE FixedArith::to_fixed_cvt
#define TPD_TO_FIXED_IM FixedArith::to_fixed_cvt
#define TPD_TO_DOUBLE_RE FixedArith::to_double_cvt
#define TPD_TO_DOUBLE_IM FixedArith::to_double_cvt
#elif defined(TPD_CVT_RE)
#define TPD_TO_FIXED_RE FixedArith::to_fixed_cvt
#define TPD_TO_FIXED_IM FixedArith::to_fixed
#define TPD_TO_DOUBLE_RE FixedArith::to_double_cvt
#define TPD_TO_DOUBLE_IM FixedArith::to_double_int
#else
#define TPD_TO_FIXED_RE FixedArith::to_fixed
#define TPD_TO_FIXED_IM FixedArith::to_fixed
#define TPD_TO_DOUBLE_RE FixedArith::to_double_int
#define TPD_TO_DOUBLE_IM FixedArith::to_double_int
#endif

// Tiles meeting an Inf or NaN run the IEEE fp64 butterfly instead.  Out of
// line (never taken for finite data) so the hot path stays small in the
// instruction cache.  Elements are re-read: doubles as such, int64 sums of a
// previous pass converted with their tile's binary point.
template <bool kDec, bool kCg = false, bool kCl = false>
__device__ __noinline__ void ieee_tile(const PassDesc& pd, const PassArgs& args, void* matp, const int* q_in,
                                       int* q_out, long long tile, long long base, long long pbase, int nbase,
                                       unsigned char* smem, int lane, int warp) {
  double2 raw[kElems];
  load_tile<kCg>(pd, matp, base, lane, warp, raw);
  if (q_in != nullptr) {
    const Stage& s0 = pd.st[0];
    long long pt = pbase;
#pragma unroll
    for (int i = 0; i < kLaneBits; ++i)
      if ((lane >> i) & 1) pt += pd.prev_w[s0.lane[i]];
    for (int i = 0; i < pd.D - kMinTileBits; ++i)
      if ((warp >> i) & 1) pt += pd.prev_w[s0.warp[i]];
    const int p0 = pd.prev_w[s0.reg[0]], p1 = pd.prev_w[s0.reg[1]], p2 = pd.prev_w[s0.reg[2]],
              p3 = pd.prev_w[s0.reg[3]];
    for (int e = 0; e < kElems; ++e) {
      const int q = ld_in<kCg>(q_in + pt + reg_off(e, p0, p1, p2, p3));
      if (q == kQIeee) continue;
      if (!q_is_valid(q)) { raw[e] = make_double2(0.0, 0.0); continue; }
      raw[e].x = FixedArith::to_double_int(__double_as_longlong(raw[e].x), -q);
      raw[e].y = FixedArith::to_double_int(__double_as_longlong(raw[e].y), -q);
    }
  }
  const bool last = q_out == nullptr;
  const double mul = kDec ? pow2d(-pd.K) : (last ? pow2d(args.out_pow2) * args.out_mul : 1.0);
  finish_tile<F64Arith, kDec, kCl>(pd, args, matp, raw, mul, base, nbase, smem, lane, warp);
  if (!last && threadIdx.x == 0 && (!kCl || cluster_rank() == 0)) q_out[tile] = kQIeee;
}

// The tile's elements in the stage-0 mapping from a shared-memory copy.
template <class Store>
__device__ __forceinline__ void load_tile_smem(const PassDesc& pd, const unsigned char* buf, int lane, int warp,
                                               Store (&raw)[kElems]) {
  const Stage& s0 = pd.st[0];
  const Store* b = reinterpret_cast<const Store*>(buf);
  const int t = thread_sidx(pd, s0, lane, warp);
  const int w0 = 1 << s0.reg[0], w1 = 1 << s0.reg[1], w2 = 1 << s0.reg[2], w3 = 1 << s0.reg[3];
#pragma unroll
  for (int e = 0; e < kElems; ++e) raw[e] = b[t + reg_off(e, w0, w1, w2, w3)];
}

// Role of a fixed-point pass (kRoleIntIn / kRoleIntOut of tpd_launch.h), a
// compile-time choice so that each kernel carries only its own conversions
// (smaller code, fewer registers).

// xbuf: shared-memory exchange area (2^D x 16 bytes); red: 64 ints;
// inbuf: the tile already copied to shared memory (stage-0 positions), or
// nullptr to read it from global memory.
// kCl: one CTA of a two-CTA cluster (warp: the virtual warp, rank * 8 + the
// CTA's own warp; red: this CTA's reduction slots).
template <bool kDec, int kRole, bool kCg = false, bool kCl = false>
__device__ __forceinline__ void fixed_tile(const PassDesc& pd, const PassArgs& args, void* matp, const int* q_in,
                                           int* q_out, long long tile, long long base, long long pbase, int nbase,
                                           const unsigned char* inbuf, unsigned char* xbuf, int* red, int lane,
                                           int warp) {
  using V = FixedArith::V;
  const int nwarps = 1 << (pd.D - kMinTileBits - (kCl ? 1 : 0));   // this CTA's warps
  const int lwarp = kCl ? (warp & 7) : warp;
  unsigned char* smem = xbuf;
  V v[kElems];
  int qin;
  if constexpr (!(kRole & kRoleIntIn)) {
    // ---- first pass: IEEE doubles onto the tile's binary point
    double2 raw[kElems];
    if (inbuf) load_tile_smem(pd, inbuf, lane, warp, raw);
    else load_tile<kCg>(pd, matp, base, lane, warp, raw);
    if constexpr (kCl) cluster_wait();                   // the peer CTA is running
    uint32_t hmax = 0, nzw = 0;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const uint32_t hx = (uint32_t)__double2hiint(raw[e].x) & 0x7fffffffu;
      const uint32_t hy = (uint32_t)__double2hiint(raw[e].y) & 0x7fffffffu;
      hmax = max(hmax, max(hx, hy));
    }
    if (args.skip_zero) {
#pragma unroll
      for (int e = 0; e < kElems; ++e)
        nzw |= (uint32_t)__double2hiint(raw[e].x) << 1 | (uint32_t)__double2loint(raw[e].x) |
               (uint32_t)__double2hiint(raw[e].y) << 1 | (uint32_t)__double2loint(raw[e].y);
      nzw = __reduce_or_sync(kFull, nzw);
    }
    const uint32_t wmax = __reduce_max_sync(kFull, hmax >> 20);
    int emax = 0, nz = 0;
    if constexpr (kCl) {
      // this CTA's warp maxima into its own slots 0..15 and the peer's 32..47
      int* pred = peer_smem(red);
      if (lane == 0) {
        red[lwarp] = (int)wmax; red[16 + lwarp] = (int)nzw;
        pred[32 + lwarp] = (int)wmax; pred[48 + lwarp] = (int)nzw;
      }
      cluster_sync();
      for (int w = 0; w < nwarps; ++w) {
        emax = max(emax, max(red[w], red[32 + w]));
        nz |= red[16 + w] | red[48 + w];
      }
    } else {
      if (lane == 0) { red[warp] = (int)wmax; red[16 + warp] = (int)nzw; }
      __syncthreads();
      for (int w = 0; w < nwarps; ++w) { emax = max(emax, red[w]); nz |= red[16 + w]; }
    }
    if (args.skip_zero && nz == 0) return;                // all +-0: outputs are zero already
    if (emax == 2047) {                                   // Inf/NaN in the tile
      ieee_tile<kDec, kCg, kCl>(pd, args, matp, nullptr, q_out, tile, base, pbase, nbase, smem, lane, warp);
      return;
    }
    // x * 2^S with S = 1084 - K - emax_eff puts the largest element below 2^(62-K)
    const int emax_eff = max(emax, 1);
    const int shift_base = 9 - pd.K - emax_eff;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      v[e].re = TPD_TO_FIXED_RE(raw[e].x, shift_base);
      v[e].im = TPD_TO_FIXED_IM(raw[e].y, shift_base);
    }
    qin = emax_eff + pd.K - 1084;                          // = -S
  } else {
    // ---- later pass: int64 sums with their previous tile's binary point
    longlong2 raw[kElems];
    if (inbuf) load_tile_smem(pd, inbuf, lane, warp, raw);
    else load_tile<kCg>(pd, matp, base, lane, warp, raw);
    if constexpr (kCl) cluster_wait();                   // the peer CTA is running
    // The tile's elements come from 2^prev_nb previous tiles (<= 2^kMaxPrevBits):
    // their binary points are loaded once each into shared memory (qs), and
    // each element finds its own there by its combination index.
    const Stage& s0 = pd.st[0];
    int* qs = red + 64;
    int qmax = kQValidMin, ieee = 0;
    {
      // (each CTA of a cluster gathers all of them: both see the same maximum)
      const int nq = 1 << pd.prev_nb, nthr = 32 * nwarps;
      for (int j = lane + 32 * lwarp; j < nq; j += nthr) {
        long long idx = pbase;
        for (int k = 0; k < pd.prev_nb; ++k)
          if ((j >> k) & 1) idx += pd.prev_cw[k];
        const int q = ld_in<kCg>(q_in + idx);
        qs[j] = q;
        qmax = max(qmax, q);
        ieee |= (q == kQIeee);
      }
    }
    int qj = 0;
#pragma unroll
    for (int i = 0; i < kLaneBits; ++i)
      if ((lane >> i) & 1) qj += pd.prev_qw[s0.lane[i]];
    for (int i = 0; i < pd.D - kMinTileBits; ++i)
      if ((warp >> i) & 1) qj += pd.prev_qw[s0.warp[i]];
    const int j0 = pd.prev_qw[s0.reg[0]], j1 = pd.prev_qw[s0.reg[1]], j2 = pd.prev_qw[s0.reg[2]],
              j3 = pd.prev_qw[s0.reg[3]];
    // kQIeee sits below kQValidMin, so it never wins the max
    qmax = __reduce_max_sync(kFull, qmax);
    ieee = __reduce_or_sync(kFull, ieee);
    if (lane == 0) { red[lwarp] = qmax; red[16 + lwarp] = ieee; }
    __syncthreads();
    qmax = kQValidMin; ieee = 0;
    for (int w = 0; w < nwarps; ++w) { qmax = max(qmax, red[w]); ieee |= red[16 + w]; }
    if (ieee) {
      ieee_tile<kDec, kCg, kCl>(pd, args, matp, q_in, q_out, tile, base, pbase, nbase, smem, lane, warp);
      return;
    }
    if (qmax == kQValidMin) {                              // every source tile was zero
      if (args.skip_zero) return;
      qmax = 0;
    }
    qin = qmax + pd.K;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const int q = qs[qj + reg_off(e, j0, j1, j2, j3)];   // written before the barrier above
      if (q_is_valid(q)) {
        const unsigned sh = (unsigned)(qin - q);
        v[e].re = TPD_ALIGN(raw[e].x, sh);
        v[e].im = TPD_ALIGN(raw[e].y, sh);
      } else {
        v[e].re = 0; v[e].im = 0;
      }
    }
  }

  // ---- the pass's levels
  V* sm = reinterpret_cast<V*>(smem);
  for (int s = 0; s < pd.nstage; ++s) {
    if (s > 0) exchange<kCl>(v, pd, pd.st[s - 1], pd.st[s], sm, lane, warp, s > 1);
    stage_levels<FixedArith, kDec>(v, pd.st[s], lane);
  }
  const int qout = qin - (kDec ? pd.K : 0);                // the 1/2 of Eq. 4 per level

  // ---- store in place
  const Stage& sl = pd.st[pd.nstage - 1];
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, sl, lane, warp);
  const uint32_t w0 = 1u << pd.gbit[sl.reg[0]], w1 = 1u << pd.gbit[sl.reg[1]];
  const uint32_t w2 = 1u << pd.gbit[sl.reg[2]], w3 = 1u << pd.gbit[sl.reg[3]];
  const bool flags = args.flags_out != nullptr;
  int nt = 0, n0 = 0, n1 = 0, n2 = 0, n3 = 0;
  bool lanes_inside = true;
  if (flags) {
    nt = nbase + thread_next(pd, sl, lane, warp);
    n0 = pd.next_w[sl.reg[0]]; n1 = pd.next_w[sl.reg[1]];
    n2 = pd.next_w[sl.reg[2]]; n3 = pd.next_w[sl.reg[3]];
#pragma unroll
    for (int i = 0; i < kLaneBits; ++i) lanes_inside &= (pd.next_w[sl.lane[i]] == 0);
  }
  if constexpr ((kRole & kRoleIntOut) != 0) {
    longlong2* mat = reinterpret_cast<longlong2*>(matp);
#pragma unroll
    for (int e = 0; e < kElems; ++e) mat[g + reg_off(e, w0, w1, w2, w3)] = make_longlong2(v[e].re, v[e].im);
    if (threadIdx.x == 0 && (!kCl || cluster_rank() == 0)) q_out[tile] = qout;
  } else {
    double2* mat = reinterpret_cast<double2*>(matp);
    const int T = -(qout + args.out_pow2);
    const bool resid = args.out_mul != 1.0;                // non-power-of-two composition scale (rare)
    if (FixedArith::fast_range(T) && !resid) {             // the whole tile rounds in the normal range
      // real parts through the fp64 conversion unit, imaginary parts through
      // integer instructions (identical roundings): the two pipes share the
      // conversions (measured on GB300: n = 14 last pass 1.82 -> 1.67 ms;
      // all of them on either pipe is slower)
#pragma unroll
      for (int e = 0; e < kElems; ++e)
        mat[g + reg_off(e, w0, w1, w2, w3)] =
            make_double2(FixedArith::to_double_cvt_fast(v[e].re, T), FixedArith::to_double_fast(v[e].im, T));
    } else {
#pragma unroll
      for (int e = 0; e < kElems; ++e) {
        double2 o;
        o.x = TPD_TO_DOUBLE_RE(v[e].re, T);
        o.y = TPD_TO_DOUBLE_IM(v[e].im, T);
        if (resid) { o.x *= args.out_mul; o.y *= args.out_mul; }
        mat[g + reg_off(e, w0, w1, w2, w3)] = o;
      }
    }
  }
  if (flags) {
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const bool nz = (v[e].re | v[e].im) != 0;
      const int id = nt + reg_off(e, n0, n1, n2, n3);
      if (lanes_inside) {
        if (__any_sync(kFull, nz) && lane == 0) args.flags_out[id] = 1;
      } else if (nz) {
        args.flags_out[id] = 1;
      }
    }
  }
}

// ============================================================== fixed point, float storage
//
// Every pass of the complex64 fixed-point form reads floats, sums the tile's
// K levels exactly in int64 on the tile's own binary point, and rounds the
// results to float (RNE) as it stores: one rounding per pass, nothing handed
// between passes but the floats.  Tiles meeting an Inf or NaN run the IEEE
// float butterfly instead.
template <bool kDec, bool kCg>
__device__ __forceinline__ void fixed32_tile(const PassDesc& pd, const PassArgs& args, void* matp, long long base,
                                             int nbase, unsigned char* smem, int* red, int lane, int warp) {
  using V = Fixed32Arith::V;
  const int nwarps = 1 << (pd.D - kMinTileBits);
  float2 raw[kElems];
  load_tile<kCg>(pd, matp, base, lane, warp, raw);
  uint32_t hmax = 0, nzw = 0;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    const uint32_t hx = __float_as_uint(raw[e].x) & 0x7fffffffu, hy = __float_as_uint(raw[e].y) & 0x7fffffffu;
    hmax = max(hmax, max(hx, hy));
    nzw |= hx | hy;
  }
  const uint32_t wmax = __reduce_max_sync(kFull, hmax >> 23);
  nzw = __reduce_or_sync(kFull, nzw);
  if (lane == 0) { red[warp] = (int)wmax; red[16 + warp] = (int)nzw; }
  __syncthreads();
  int emax = 0, nz = 0;
  for (int w = 0; w < nwarps; ++w) { emax = max(emax, red[w]); nz |= red[16 + w]; }
  if (args.skip_zero && nz == 0) return;                  // all +-0: outputs are zero already
  if (emax == 255) {                                      // Inf/NaN in the tile
    finish_tile<F32Arith, kDec>(pd, args, matp, raw, kDec ? pow2d(-pd.K) : pow2d(args.out_pow2) * args.out_mul,
                                base, nbase, smem, lane, warp);
    return;
  }
  const int emax_eff = max(emax, 1);
  const int rs_base = emax_eff + pd.K;
  V v[kElems];
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    v[e].re = Fixed32Arith::to_fixed(raw[e].x, rs_base);
    v[e].im = Fixed32Arith::to_fixed(raw[e].y, rs_base);
  }
  V* sm = reinterpret_cast<V*>(smem);
  for (int s = 0; s < pd.nstage; ++s) {
    if (s > 0) exchange(v, pd, pd.st[s - 1], pd.st[s], sm, lane, warp, s > 1);
    stage_levels<Fixed32Arith, kDec>(v, pd.st[s], lane);
  }
  // value = sum * 2^-S (S = 188 - K - emax_eff), times 2^-K for the 1/2 of
  // Eq. 4 per level, times 2^out_pow2 for a composition's scale
  const int T = 188 - pd.K - emax_eff + (kDec ? pd.K : 0) - args.out_pow2;
  const bool resid = args.out_mul != 1.0;
  const bool fast = Fixed32Arith::fast_range(T);
  const Stage& sl = pd.st[pd.nstage - 1];
  float2* mat = reinterpret_cast<float2*>(matp);
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, sl, lane, warp);
  const uint32_t w0 = 1u << pd.gbit[sl.reg[0]], w1 = 1u << pd.gbit[sl.reg[1]];
  const uint32_t w2 = 1u << pd.gbit[sl.reg[2]], w3 = 1u << pd.gbit[sl.reg[3]];
  const bool flags = args.flags_out != nullptr;
  int nt = 0, n0 = 0, n1 = 0, n2 = 0, n3 = 0;
  bool lanes_inside = true;
  if (flags) {
    nt = nbase + thread_next(pd, sl, lane, warp);
    n0 = pd.next_w[sl.reg[0]]; n1 = pd.next_w[sl.reg[1]];
    n2 = pd.next_w[sl.reg[2]]; n3 = pd.next_w[sl.reg[3]];
#pragma unroll
    for (int i = 0; i < kLaneBits; ++i) lanes_inside &= (pd.next_w[sl.lane[i]] == 0);
  }
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    // real parts on the conversion unit, imaginary parts with integer
    // instructions (identical roundings; n = 15: 31.3 -> 28.3 ms)
    float2 o = make_float2(fast ? Fixed32Arith::to_float_cvt_fast(v[e].re, T) : Fixed32Arith::to_float(v[e].re, T),
                           Fixed32Arith::to_float(v[e].im, T));
    if (resid) { o.x = __fmul_rn(o.x, (float)args.out_mul); o.y = __fmul_rn(o.y, (float)args.out_mul); }
    mat[g + reg_off(e, w0, w1, w2, w3)] = o;
    if (flags) {
      const bool nzo = (v[e].re | v[e].im) != 0;
      const int id = nt + reg_off(e, n0, n1, n2, n3);
      if (lanes_inside) {
        if (__any_sync(kFull, nzo) && lane == 0) args.flags_out[id] = 1;
      } else if (nzo) {
        args.flags_out[id] = 1;
      }
    }
  }
}

// One tile of a pass: its position from the tile id, then the arithmetic's
// load / levels / store.  smem: the exchange area (2^D x 16 bytes; half of it
// per CTA of a two-CTA cluster) followed by 64 ints of reduction slots.
template <class A, bool kDec, int kRole, bool kCg, bool kCl = false>
__device__ __forceinline__ void pass_tile(const PassDesc& pd, const PassArgs& args, void* matp, const int* q_in,
                                          int* q_out, long long tile, unsigned char* smem, int lane, int warp) {
  using Store = typename A::Store;
  static_assert(!(kCl && A::kFixed32), "two-CTA clusters serve complex128 tiles only");
  int* red = reinterpret_cast<int*>(smem + ((size_t)16 << (pd.D - (kCl ? 1 : 0))));
  long long base = 0, pbase = 0;
  int nbase = 0;
  for (int j = 0; j < pd.nrest; ++j)
    if ((tile >> j) & 1) {
      base += 1ll << pd.rest_gbit[j];
      nbase += (int)pd.next_rest_w[j];
      pbase += pd.prev_rest_w[j];
    }

  if constexpr (A::kFixed) {
    fixed_tile<kDec, kRole, kCg, kCl>(pd, args, matp, q_in, q_out, tile, base, pbase, nbase, nullptr, smem, red,
                                      lane, warp);
  } else if constexpr (A::kFixed32) {
    fixed32_tile<kDec, kCg>(pd, args, matp, base, nbase, smem, red, lane, warp);
  } else {
    Store raw[kElems];
    load_tile<kCg>(pd, matp, base, lane, warp, raw);
    if constexpr (kCl) cluster_wait();                   // the peer CTA is running
    if (args.skip_zero) {
      int nz = 0;
#pragma unroll
      for (int e = 0; e < kElems; ++e) nz |= A::nonzero(raw[e]);
      nz = __syncthreads_or(nz);
      if constexpr (kCl) {                               // cluster-wide: slot 0 here, slot 1 at the peer
        if (threadIdx.x == 0) { red[0] = nz; peer_smem(red)[1] = nz; }
        cluster_sync();
        nz = red[0] | red[1];
      }
      if (!nz) return;
    }
    finish_tile<A, kDec, kCl>(pd, args, matp, raw, args.out_mul, base, nbase, smem, lane, warp);
  }
}

// Tiles of up to 2^12 elements run 256-thread CTAs, several per SM; 2^13
// element tiles run 512-thread CTAs.
// kMinBlocks: CTAs of kThreads the compiler must fit on one SM (register
// budget); the planner picks 3 for the conversion-heavy first and last
// fixed-point passes and 2 elsewhere.  kRole: fixed point only (see above).
template <class A, bool kDec, int kThreads, int kMinBlocks, int kRole = 0>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_pass(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long tile = (long long)blockIdx.x + (long long)blockIdx.y * gridDim.x;
  void* matp = args.mat;
  const int* q_in = args.q_in;
  int* q_out = args.q_out;
  if (args.chunked) {                      // one L2-sized chunk of the matrix: spread the CTA index
    unsigned long long t = args.chunk_or;
    for (int k = 0; k < args.nfree; ++k)
      if ((tile >> k) & 1) t |= 1ull << args.chunk_free[k];
    tile = (long long)t;
  }
  if (args.ptrs != nullptr) {              // batched: tiles of matrix items[m] are contiguous in the grid
    const long long m = tile / args.tiles_per_mat;
    tile -= m * args.tiles_per_mat;
    const int idx = args.items[m];
    if (idx < 0) return;                   // bucketing found ns_dev inconsistent: touch nothing
    matp = args.ptrs[idx];
    if (q_in) q_in += m * args.q_in_stride;
    if (q_out) q_out += m * args.q_out_stride;
  }
  if (tile >= pd.ntiles) return;
  if (args.flags_in != nullptr && args.flags_in[tile] == 0) return;
  if (args.need != nullptr && args.need[tile] == 0) return;
  pass_tile<A, kDec, kRole, false>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
}

// Complex128 tiles of 2^13 elements as two-CTA clusters of 256 threads (see
// the top of this file): grid = 2 x tiles, tile = cluster index.
template <class A, bool kDec, int kRole = 0>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 2)
    k_pass_cl(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31;
  const int warp = (int)(cluster_rank() << 3) | (tid >> 5);   // the 512-thread layout's warp
  long long tile = (long long)(blockIdx.x >> 1);
  void* matp = args.mat;
  const int* q_in = args.q_in;
  int* q_out = args.q_out;
  if (args.chunked) {
    unsigned long long t = args.chunk_or;
    for (int k = 0; k < args.nfree; ++k)
      if ((tile >> k) & 1) t |= 1ull << args.chunk_free[k];
    tile = (long long)t;
  }
  if (args.ptrs != nullptr) {
    const long long m = tile / args.tiles_per_mat;
    tile -= m * args.tiles_per_mat;
    const int idx = args.items[m];
    if (idx < 0) return;
    matp = args.ptrs[idx];
    if (q_in) q_in += m * args.q_in_stride;
    if (q_out) q_out += m * args.q_out_stride;
  }
  // both CTAs of a cluster share the tile, so they leave here together
  if (tile >= pd.ntiles) return;
  if (args.flags_in != nullptr && args.flags_in[tile] == 0) return;
  if (args.need != nullptr && args.need[tile] == 0) return;
  cluster_arrive_relaxed();
  pass_tile<A, kDec, kRole, false, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
}

// -------------------------------------------------------------- persistent, double buffered
//
// Fixed point, one matrix, tiles of up to 2^12 elements: one CTA per SM walks
// the tiles (tile += gridDim.x).  Each thread copies ITS elements of the next
// tile into the spare shared-memory buffer with cp.async while the CTA works
// on the current one, so HBM stays busy across the compute phase.  The waits
// are the hardware's (cp.async.wait_group + barrier), with no spin loops.

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ long long tile_base(const PassDesc& pd, long long tile) {
  long long base = 0;
  for (int j = 0; j < pd.nrest; ++j)
    if ((tile >> j) & 1) base += 1ll << pd.rest_gbit[j];
  return base;
}

// This thread's 16 elements of `tile` (stage-0 positions) into buf.
__device__ __forceinline__ void prefetch_tile(const PassDesc& pd, const void* matp, long long tile,
                                              unsigned char* buf, int lane, int warp) {
  const Stage& s0 = pd.st[0];
  const char* mat = reinterpret_cast<const char*>(matp);
  const long long g = tile_base(pd, tile) + thread_goff(pd, s0, lane, warp);
  const long long w0 = 1ll << pd.gbit[s0.reg[0]], w1 = 1ll << pd.gbit[s0.reg[1]];
  const long long w2 = 1ll << pd.gbit[s0.reg[2]], w3 = 1ll << pd.gbit[s0.reg[3]];
  const int t = thread_sidx(pd, s0, lane, warp);
  const int v0 = 1 << s0.reg[0], v1 = 1 << s0.reg[1], v2 = 1 << s0.reg[2], v3 = 1 << s0.reg[3];
#pragma unroll
  for (int e = 0; e < kElems; ++e)
    cp_async16(buf + 16 * (t + reg_off(e, v0, v1, v2, v3)), mat + 16 * (g + reg_off(e, w0, w1, w2, w3)));
  cp_async_commit();
}

template <bool kDec, int kRole>
__global__ void __launch_bounds__(256, 1)
    k_pass_pipe(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t tb = (size_t)16 << pd.D;
  unsigned char* buf0 = smem;
  unsigned char* buf1 = smem + tb;
  int* red = reinterpret_cast<int*>(smem + 2 * tb);
  long long tile = blockIdx.x;
  if (tile >= pd.ntiles) return;
  prefetch_tile(pd, args.mat, tile, buf0, lane, warp);
  bool odd = false;
  for (; tile < pd.ntiles; tile += gridDim.x, odd = !odd) {
    unsigned char* cur = odd ? buf1 : buf0;
    unsigned char* spare = odd ? buf0 : buf1;
    const long long nxt = tile + gridDim.x;
    if (nxt < pd.ntiles) {
      prefetch_tile(pd, args.mat, nxt, spare, lane, warp);
      cp_async_wait<1>();                 // this thread's copies of the current tile have landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();                      // ... and everyone's
    long long base = 0, pbase = 0;
    int nbase = 0;
    for (int j = 0; j < pd.nrest; ++j)
      if ((tile >> j) & 1) {
        base += 1ll << pd.rest_gbit[j];
        nbase += (int)pd.next_rest_w[j];
        pbase += pd.prev_rest_w[j];
      }
    fixed_tile<kDec, kRole>(pd, args, args.mat, args.q_in, args.q_out, tile, base, pbase, nbase, cur, cur, red,
                            lane, warp);
    __syncthreads();                      // the current buffer is refilled next iteration
  }
}

// -------------------------------------------------------------- whole small matrices
// One CTA per matrix of n <= 6 qubits held entirely in shared memory; every
// level is a sweep over the 4^(n-1) quads.  Used for n <= 4 and in batches.

template <class A, bool kDec>
__device__ __forceinline__ void small_levels(typename A::V* sm, int n, int tid, int nthr) {
  const int quads = 1 << (2 * n - 2);
  for (int beta = 0; beta < n; ++beta) {
    const int rbit = n + beta;
    for (int q = tid; q < quads; q += nthr) {
      // insert zero bits at beta and n+beta
      const int lo = q & ((1 << beta) - 1);
      const int q1 = q >> beta;
      const int mid = q1 & ((1 << (n - 1)) - 1);
      const int hi = q1 >> (n - 1);
      const int i00 = lo | (mid << (beta + 1)) | (hi << (rbit + 1));
      const int i01 = i00 | (1 << beta), i10 = i00 | (1 << rbit), i11 = i01 | (1 << rbit);
      const typename A::V a00 = sm[i00], a01 = sm[i01], a10 = sm[i10], a11 = sm[i11];
      if (kDec) {
        sm[i00] = A::add(a00, a11);
        sm[i01] = A::add(a01, a10);
        sm[i10] = A::mul_i(A::sub(a01, a10));
        sm[i11] = A::sub(a00, a11);
      } else {
        const typename A::V iy = A::mul_i(a10);
        sm[i00] = A::add(a00, a11);
        sm[i01] = A::sub(a01, iy);
        sm[i10] = A::add(a01, iy);
        sm[i11] = A::sub(a00, a11);
      }
    }
    __syncthreads();
  }
}

template <class A, bool kDec>
__device__ __forceinline__ void small_run(typename A::Store* mat, int n, int skip, int scale_mode,
                                          unsigned char* smem, int tid, int nthr, int emax_in) {
  using V = typename A::V;
  V* sm = reinterpret_cast<V*>(smem);
  const int count = 1 << (2 * n);
  int shift_base = 0, outT = 0;
  if constexpr (A::kFixed) {
    const int emax_eff = max(emax_in, 1);
    shift_base = 9 - n - emax_eff;
    // fixed = x * 2^S with headroom for n levels; the output is sum * 2^-S,
    // times 2^-n for the decomposition (the 1/2 of Eq. 4 per level) or for a
    // composition scaled to the adjoint.
    const int S = 1084 - n - emax_eff;
    outT = (kDec || scale_mode) ? S + n : S;
  }
  for (int i = tid; i < count; i += nthr) {
    const typename A::Store x = mat[i];
    if constexpr (A::kFixed) {
      V t; t.re = A::to_fixed(x.x, shift_base); t.im = A::to_fixed(x.y, shift_base);
      sm[i] = t;
    } else {
      sm[i] = A::load(x);
    }
  }
  __syncthreads();
  small_levels<A, kDec>(sm, n, tid, nthr);
  const double mul = (kDec || scale_mode) ? pow2d(-n) : 1.0;
  for (int i = tid; i < count; i += nthr) {
    typename A::Store o;
    if constexpr (A::kFixed) {
      o.x = A::to_double(sm[i].re, outT);
      o.y = A::to_double(sm[i].im, outT);
    } else {
      o = A::store(sm[i], OutScale{0, 1.0}, mul);
    }
    mat[i] = o;
  }
}

// A whole matrix of n <= 6 qubits by the CTA's nthr threads (all of them call
// it): max exponent / nonzero test, then small_run (IEEE fallback for Inf/NaN).
template <class A, bool kDec>
__device__ __forceinline__ void small_matrix(typename A::Store* mat, int n, int skip_zero, int scale_mode,
                                             unsigned char* smem, int tid, int nthr) {
  using Store = typename A::Store;
  const int count = 1 << (2 * n);
  // max exponent / nonzero over the whole matrix
  uint32_t emax = 0, nzw = 0;
  for (int i = tid; i < count; i += nthr) {
    const Store x = mat[i];
    uint32_t hx, hy, lx, ly;
    if constexpr (sizeof(Store) == 16) {
      hx = (uint32_t)__double2hiint(((const double2&)x).x) & 0x7fffffffu;
      hy = (uint32_t)__double2hiint(((const double2&)x).y) & 0x7fffffffu;
      lx = (uint32_t)__double2loint(((const double2&)x).x);
      ly = (uint32_t)__double2loint(((const double2&)x).y);
      emax = max(emax, max(hx >> 20, hy >> 20));
    } else {
      hx = __float_as_uint(((const float2&)x).x) & 0x7fffffffu;
      hy = __float_as_uint(((const float2&)x).y) & 0x7fffffffu;
      lx = ly = 0;
    }
    nzw |= hx | hy | lx | ly;
  }
  const int nz = __syncthreads_or((int)(nzw != 0));
  if (skip_zero && !nz) return;
  uint32_t* red = reinterpret_cast<uint32_t*>(smem);
  emax = __reduce_max_sync(kFull, emax);
  if ((tid & 31) == 0) red[tid >> 5] = emax;
  __syncthreads();
  uint32_t em = 0;
  for (int w = 0; w < (nthr + 31) / 32; ++w) em = max(em, red[w]);
  __syncthreads();
  if constexpr (A::kFixed) {
    if (em == 2047) {
      small_run<F64Arith, kDec>(mat, n, skip_zero, scale_mode, smem, tid, nthr, 0);
      return;
    }
  }
  small_run<A, kDec>(mat, n, skip_zero, scale_mode, smem, tid, nthr, (int)em);
}

template <class A, bool kDec>
__global__ void __launch_bounds__(256) k_small(const SmallArgs args) {
  using Store = typename A::Store;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  int idx = blockIdx.x;
  if (args.items) idx = args.items[idx];
  if (idx < 0) return;                     // bucketing found ns_dev inconsistent: touch nothing
  Store* mat = reinterpret_cast<Store*>(args.ptrs ? args.ptrs[idx] : args.mat);
  const int n = args.ptrs ? args.ns[idx] : args.n;
  small_matrix<A, kDec>(mat, n, args.skip_zero, args.scale_mode, smem, tid, nthr);
}

}  // namespace tpd
