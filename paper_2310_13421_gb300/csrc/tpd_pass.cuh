// One pass of the Pauli butterfly over a group of qubit levels (Sec. III,
// Eqs. 3-5), in place, one CTA per tile.  See tpd_plan.h for tiles and stages
// and tpd_arith.cuh for the arithmetics.
//
// Flow of a CTA:
//   1. skip the tile if the previous pass flagged it all-zero (zero-CMW
//      pruning of Alg. 1/2: a zero block has only zero weights below it);
//   2. load its 16 elements per thread from HBM with the stage-0 mapping
//      (lanes on the lowest tile bits: 128-byte runs);
//   3. block fixed point: the largest exponent of each class of elements the
//      pass adds together -> one binary point per class; optional all-zero
//      test (then nothing is written);
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
#include "tpd_shape.h"

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

// -------------------------------------------------------------- pass geometry
//
// The device functions below read a pass's layout through a geometry object
// `pd`: either the run-time PassDesc itself (any plan) or a GeoCT, which
// gives the in-tile layout of a compiled shape (tpd_shape.h) as constants and
// forwards the rest (global bit positions, tile-id and class-index weights)
// to the run-time descriptor.  Both spell the same members (pd.D, pd.K,
// pd.nstage, pd.st[s].reg[i], pd.cls_w[i], pd.gbit[i], ...), so one body of
// code serves both; with a GeoCT, once the loops over stages and bits are
// unrolled, every layout lookup is a constant.

template <class Sh>
struct StageCT {
  struct Reg {
    int s;
    __device__ __forceinline__ int operator[](int i) const { return (int)((Sh::kReg >> (16 * s + 4 * i)) & 15); }
  };
  struct Lane {
    int s;
    __device__ __forceinline__ int operator[](int i) const { return (int)((Sh::kLane >> (20 * s + 4 * i)) & 15); }
  };
  struct Warp {
    int s;
    __device__ __forceinline__ int operator[](int i) const { return (int)((Sh::kWarp >> (16 * s + 4 * i)) & 15); }
  };
  struct ShflLane {
    int s;
    __device__ __forceinline__ int operator[](int j) const { return (int)((Sh::kShfl >> (12 * s + 3 * j)) & 7); }
  };
  Reg reg;
  Lane lane;
  Warp warp;
  ShflLane shfl_lane;
  int npair, nshfl;
  __device__ __forceinline__ explicit StageCT(int s)
      : reg{s}, lane{s}, warp{s}, shfl_lane{s}, npair((int)((Sh::kStg >> (8 * s)) & 3)),
        nshfl((int)((Sh::kStg >> (8 * s + 2)) & 7)) {}
};

template <class Sh>
struct GeoCT {
  static constexpr int D = Sh::kD;
  static constexpr int K = Sh::kK;
  static constexpr int nstage = Sh::kNStage;
  struct Cls {
    __device__ __forceinline__ int operator[](int i) const { return 1 << (int)((Sh::kCls >> (4 * i)) & 15); }
  };
  struct Stages {
    __device__ __forceinline__ StageCT<Sh> operator[](int s) const { return StageCT<Sh>(s); }
  };
  Cls cls_w;
  Stages st;
  const PassDesc& raw;
  const int8_t (&gbit)[kMaxTileBits];
  const int32_t (&next_w)[kMaxTileBits];
  const uint32_t (&src_w)[kMaxTileBits];
  const int32_t& nrest;
  const int8_t (&rest_gbit)[2 * kMaxQubits];
  const int64_t (&next_rest_w)[2 * kMaxQubits];
  const uint32_t (&src_rest_w)[2 * kMaxQubits];
  __device__ __forceinline__ explicit GeoCT(const PassDesc& p)
      : raw(p), gbit(p.gbit), next_w(p.next_w), src_w(p.src_w), nrest(p.nrest), rest_gbit(p.rest_gbit),
        next_rest_w(p.next_rest_w), src_rest_w(p.src_rest_w) {}
};

// the run-time descriptor behind a geometry
__device__ __forceinline__ const PassDesc& raw_desc(const PassDesc& p) { return p; }
template <class Sh>
__device__ __forceinline__ const PassDesc& raw_desc(const GeoCT<Sh>& g) { return g.raw; }

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

template <class G, class S>
__device__ __forceinline__ long long thread_goff(const G& pd, const S& st, int lane, int warp) {
  long long g = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i)
    if ((lane >> i) & 1) g += 1ll << pd.gbit[st.lane[i]];
#pragma unroll
  for (int i = 0; i < pd.D - kMinTileBits; ++i)
    if ((warp >> i) & 1) g += 1ll << pd.gbit[st.warp[i]];
  return g;
}

template <class G, class S>
__device__ __forceinline__ int thread_sidx(const G& pd, const S& st, int lane, int warp) {
  int s = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i) s |= ((lane >> i) & 1) << st.lane[i];
#pragma unroll
  for (int i = 0; i < pd.D - kMinTileBits; ++i) s |= ((warp >> i) & 1) << st.warp[i];
  return s;
}

template <class G, class S>
__device__ __forceinline__ int thread_next(const G& pd, const S& st, int lane, int warp) {
  int s = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i)
    if ((lane >> i) & 1) s += pd.next_w[st.lane[i]];
#pragma unroll
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
// The two lanes of a pair swap their row-1 elements (one shuffle per pair):
// the column-0 lane then holds (a00, a11), the column-1 lane (a01, a10), and
// each computes the two outputs of its pair -- the same operations on the same
// operands as pair_level.  The row-1 outputs stay in the lane that computed
// them, so after the level register RB of a thread holds the element of its
// partner lane's position ("twisted"): the exchange or store that follows
// places it there (twist_add / twist_xor).
template <class A, bool kDec, int RB>
__device__ __forceinline__ void shfl_level(typename A::V (&v)[kElems], int lbit, int lane) {
  const int mask = 1 << lbit;
  const bool cb = (lane >> lbit) & 1;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    if ((e >> RB) & 1) continue;
    const int e1i = e | (1 << RB);
    const typename A::V e0 = v[e];
    const typename A::V r = A::shfl(v[e1i], mask);   // a11 / a10 (decomposition); Z / Y (composition)
    if (kDec) {
      v[e] = A::add(e0, r);                     // I = a00 + a11 at (0,0) / X = a01 + a10 at (0,1)
      const typename A::V d = A::sub(e0, r);    // a00 - a11 / a01 - a10
      v[e1i] = cb ? A::mul_i(d) : d;            // Z for (1,1) / Y for (1,0)
    } else {
      // column 0 holds I, Y; column 1 holds X, Z
      v[e] = A::add(e0, cb ? A::mul_mi(r) : r);          // a00 = I + Z / a01 = X - iY
      v[e1i] = A::add(e0, cb ? A::mul_i(r) : A::neg(r));  // a11 = I - Z / a10 = X + iY
    }
  }
}

// After a stage's shuffle levels, register bit 2 npair + s of every thread
// also stands for its lane bit shfl_lane[s] flipped (see shfl_level): the
// element in register e sits at the position of lane (lane ^ Tw(e)).  The
// index weights of those register bits absorb it: an additive index (shared
// memory, global element, next-pass tile) gains -+ the lane bit's weight for
// a thread whose lane bit is 1 / 0 (twist_add); an XOR-linear one (the class)
// gains the lane bit's class bit (twist_xor).
template <class S, class T, class LaneW>
__device__ __forceinline__ void twist_add(const S& st, int lane, T& w0, T& w1, T& w2, T& w3, LaneW lane_w) {
#pragma unroll
  for (int s = 0; s < kRegBits; ++s) {
    if (s < st.nshfl) {
      const int lb = st.shfl_lane[s];
      const T d = lane_w(st.lane[lb]);
      const T sd = ((lane >> lb) & 1) ? T(T(0) - d) : d;
      const int rb = 2 * st.npair + s;
      if (rb == 0) w0 += sd;
      else if (rb == 1) w1 += sd;
      else if (rb == 2) w2 += sd;
      else w3 += sd;
    }
  }
}
template <class S, class T, class LaneW>
__device__ __forceinline__ void twist_xor(const S& st, T& w0, T& w1, T& w2, T& w3, LaneW lane_w) {
#pragma unroll
  for (int s = 0; s < kRegBits; ++s) {
    if (s < st.nshfl) {
      const T d = lane_w(st.lane[st.shfl_lane[s]]);
      const int rb = 2 * st.npair + s;
      if (rb == 0) w0 ^= d;
      else if (rb == 1) w1 ^= d;
      else if (rb == 2) w2 ^= d;
      else w3 ^= d;
    }
  }
}

template <class A, bool kDec, class S>
__device__ __forceinline__ void stage_levels(typename A::V (&v)[kElems], const S& st, int lane) {
  if (st.npair >= 1) pair_level<A, kDec, 0, 1>(v);
  if constexpr (kRegBits >= 4) {
    if (st.npair >= 2) pair_level<A, kDec, 2, 3>(v);
  }
  const int r0 = 2 * st.npair;
#pragma unroll
  for (int s = 0; s < st.nshfl; ++s) {
    const int lb = st.shfl_lane[s];
    switch (r0 + s) {
      case 0: shfl_level<A, kDec, 0>(v, lb, lane); break;
      case 1: shfl_level<A, kDec, 1>(v, lb, lane); break;
      case 2: shfl_level<A, kDec, 2>(v, lb, lane); break;
      default:
        if constexpr (kRegBits >= 4) shfl_level<A, kDec, 3>(v, lb, lane);
        break;
    }
  }
}

// Shared-memory exchange from stage `a`'s mapping to stage `b`'s.  kCl: the
// tile is split over a two-CTA cluster (see above): an element goes to the
// CTA whose rank equals its tile bit on b's highest warp bit, at its tile
// index with that bit removed.
template <bool kCl = false, class V, class G, class S1, class S2>
__device__ __forceinline__ void exchange(V (&v)[kElems], const G& pd, const S1& a, const S2& b, V* sm, int lane,
                                         int warp, bool sync_first) {
  if constexpr (kCl) {
    if (sync_first) cluster_sync();           // both CTAs have read the previous exchange
    const int cb = b.warp[kClWarpBit];        // >= 3: lanes hold tile bits 0..2
    const int lowm = (1 << cb) - 1;
    auto squeeze = [&](int x) { return (x & lowm) | ((x >> 1) & ~lowm); };
    V* const mine = sm;
    V* const peer = peer_smem(sm);
    const int rank = (int)cluster_rank();
    if (a.nshfl == 0) {
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
    } else {
      // twisted registers (shuffle levels): each element's full tile index,
      // then its CTA and its index there
      const int t = thread_sidx(pd, a, lane, warp);
      int w0 = 1 << a.reg[0], w1 = 1 << a.reg[1], w2 = 1 << a.reg[2], w3 = 1 << a.reg[3];
      twist_add(a, lane, w0, w1, w2, w3, [](int pos) { return 1 << pos; });
#pragma unroll
      for (int e = 0; e < kElems; ++e) {
        const int te = t + reg_off(e, w0, w1, w2, w3);
        (((te >> cb) & 1) == rank ? mine : peer)[squeeze(te)] = v[e];
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
    int w0 = 1 << a.reg[0], w1 = 1 << a.reg[1], w2 = 1 << a.reg[2], w3 = 1 << a.reg[3];
    twist_add(a, lane, w0, w1, w2, w3, [](int pos) { return 1 << pos; });
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
template <class A, bool kDec, bool kCl = false, class G, class Raw>
__device__ __forceinline__ void finish_tile(const G& pd, const PassArgs& args, void* matp,
                                            const Raw (&raw)[kElems], double mul, long long base,
                                            int nbase, unsigned char* smem, int lane, int warp) {
  using V = typename A::V;
  using Store = typename A::Store;
  V v[kElems];
#pragma unroll
  for (int e = 0; e < kElems; ++e) v[e] = A::load(raw[e]);
  V* sm = reinterpret_cast<V*>(smem);
#pragma unroll
  for (int s = 0; s < pd.nstage; ++s) {
    if (s > 0) exchange<kCl>(v, pd, pd.st[s - 1], pd.st[s], sm, lane, warp, s > 1);
    stage_levels<A, kDec>(v, pd.st[s], lane);
  }
  const auto& sl = pd.st[pd.nstage - 1];
  Store* mat = reinterpret_cast<Store*>(matp);
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, sl, lane, warp);
  uint32_t w0 = 1u << pd.gbit[sl.reg[0]], w1 = 1u << pd.gbit[sl.reg[1]];
  uint32_t w2 = 1u << pd.gbit[sl.reg[2]], w3 = 1u << pd.gbit[sl.reg[3]];
  twist_add(sl, lane, w0, w1, w2, w3, [&](int pos) { return 1u << pd.gbit[pos]; });
  const bool flags = args.flags_out != nullptr;
  int nt = 0, n0 = 0, n1 = 0, n2 = 0, n3 = 0;
  bool lanes_inside = true;
  if (flags) {
    nt = nbase + thread_next(pd, sl, lane, warp);
    n0 = pd.next_w[sl.reg[0]]; n1 = pd.next_w[sl.reg[1]];
    n2 = pd.next_w[sl.reg[2]]; n3 = pd.next_w[sl.reg[3]];
    twist_add(sl, lane, n0, n1, n2, n3, [&](int pos) { return (int)pd.next_w[pos]; });
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

template <bool kCg = false, class G, class Store>
__device__ __forceinline__ void load_tile(const G& pd, const void* matp, long long base, int lane, int warp,
                                          Store (&raw)[kElems]) {
  const auto& s0 = pd.st[0];
  const Store* mat = reinterpret_cast<const Store*>(matp);
  // element indices in 32 bits: a matrix has at most 4^16 = 2^32 elements
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, s0, lane, warp);
  const uint32_t w0 = 1u << pd.gbit[s0.reg[0]], w1 = 1u << pd.gbit[s0.reg[1]];
  const uint32_t w2 = 1u << pd.gbit[s0.reg[2]], w3 = 1u << pd.gbit[s0.reg[3]];
#pragma unroll
  for (int e = 0; e < kElems; ++e) raw[e] = ld_in<kCg>(mat + (g + reg_off(e, w0, w1, w2, w3)));
}

// ============================================================== block fixed point
//
// A pass of the block fixed point reads IEEE numbers and writes IEEE numbers.
// Its tile splits into classes (PassDesc::cls_w): the 2^K elements the pass's
// levels add together, i.e. those agreeing on x_j = r_j xor c_j of every
// level j of the pass and on every passenger bit.  Each class goes onto its
// own binary point, set by the largest exponent field E_c among the
// components of its elements, so that its largest element lands below
// 2^(62-K) and the 2^K-term sums of the pass are exact in int64; each output
// is rounded once, to nearest even, when the pass stores it.  Components far
// below their class's largest (more than 9-K binades for complex128,
// 38-K for complex64) are truncated toward zero on loading, an error
// below 2^-(62-K) of that largest.  Elements of different X-masks never share
// a binary point, so a weight's error is bounded by the magnitudes of its own
// class, not by those of a large neighbour (a strong diagonal beside weak
// couplings).  Truncation toward zero and rounding to nearest are odd
// functions, and a class and its conjugate partner (the same positions with
// the row and column bits of the unprocessed levels swapped) hold conjugate
// values with the same E_c, so conjugate symmetry is kept exactly: Hermitian
// matrices give exactly real weights.

// Class of a thread's register 0 in stage st: XOR of its lane and warp bits' class bits.
template <class G, class S>
__device__ __forceinline__ int cls_thread(const G& pd, const S& st, int lane, int warp) {
  int c = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i)
    if ((lane >> i) & 1) c ^= pd.cls_w[st.lane[i]];
#pragma unroll
  for (int i = 0; i < pd.D - kMinTileBits; ++i)
    if ((warp >> i) & 1) c ^= pd.cls_w[st.warp[i]];
  return c;
}

// class offset of register e from the class bits of the 4 register bits
// (e is a compile-time constant after unrolling)
__device__ __forceinline__ int reg_cls(int e, int w0, int w1, int w2, int w3) {
  return ((e & 1) ? w0 : 0) ^ ((e & 2) ? w1 : 0) ^ ((e & 4) ? w2 : 0) ^ ((e & 8) ? w3 : 0);
}

// Class maxima of a tile held in the stage-0 mapping: slots[c] becomes the
// largest exponent field (exp_of) of class c's elements.  The slots must be 0
// on entry.  A stage's in-register levels put a level's column and row bit on
// register bits (0,1) and (2,3), so e, e^3 (and e^12, e^15) share a class: one
// atomic per class and thread.
// Slot values of elements: the exponent field of an IEEE element, or the
// source binary point + kQSlot of an int64 one (0: a zero source).
constexpr int kQSlot = 4096;
struct ExpSlot64 {
  __device__ __forceinline__ static int of(const double2& x) {
    return (int)(max((uint32_t)__double2hiint(x.x) & 0x7fffffffu, (uint32_t)__double2hiint(x.y) & 0x7fffffffu) >> 20);
  }
};
struct ExpSlot32 {
  __device__ __forceinline__ static int of(const float2& x) {
    return (int)(max(__float_as_uint(x.x) & 0x7fffffffu, __float_as_uint(x.y) & 0x7fffffffu) >> 23);
  }
};
struct QSlot {
  __device__ __forceinline__ static int of(int q) { return q > kQValidMin ? q + kQSlot : 0; }
};

// One atomic per in-thread class: with kNp in-register levels in the stage,
// e, e^3 (and e^12, e^15) share a class.
template <int kNp, class S, class T>
__device__ __forceinline__ void class_atomics(const T (&x)[kElems], int* slots, int ct, int c0, int c1, int c2,
                                              int c3) {
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    if (kNp >= 1 && (e & 2)) continue;
    if (kNp >= 2 && (e & 8)) continue;
    int m = S::of(x[e]);
    if (kNp >= 1) m = max(m, S::of(x[e ^ 3]));
    if (kNp >= 2) m = max(m, max(S::of(x[e ^ 12]), S::of(x[e ^ 15])));
    if (m) atomicMax(slots + (ct ^ reg_cls(e, c0, c1, c2, c3)), m);
  }
}

// class_atomics for the stage's in-register level count, a uniform branch
// to straight-line code for each count
template <class S, class T>
__device__ __forceinline__ void class_atomics_any(int np, const T (&x)[kElems], int* slots, int ct, int c0, int c1,
                                                  int c2, int c3) {
  if constexpr (kRegBits >= 4) {
    if (np >= 2) {
      class_atomics<2, S>(x, slots, ct, c0, c1, c2, c3);
      return;
    }
  }
  if (np >= 1) class_atomics<1, S>(x, slots, ct, c0, c1, c2, c3);
  else class_atomics<0, S>(x, slots, ct, c0, c1, c2, c3);
}

// Returns the largest exponent field of the thread's elements, and in lo
// the smallest nonzero one (0x7fffffff if none).
template <class S, class G, class Raw, class ExpOf>
__device__ __forceinline__ uint32_t class_max(const G& pd, const Raw (&raw)[kElems], int* slots, int lane,
                                              int warp, ExpOf exp_of, int& lo) {
  const auto& s0 = pd.st[0];
  const int ct = cls_thread(pd, s0, lane, warp);
  const int c0 = pd.cls_w[s0.reg[0]], c1 = pd.cls_w[s0.reg[1]], c2 = pd.cls_w[s0.reg[2]],
            c3 = pd.cls_w[s0.reg[3]];
  uint32_t hmax = 0, hmin = 0x7fffffffu;
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    const uint32_t x = exp_of(raw[e]);
    hmax = max(hmax, x);
    hmin = min(hmin, x ? x : 0x7fffffffu);
  }
  lo = (int)hmin;
  // (the exponents are recomputed rather than kept: 16 registers fewer)
  class_atomics_any<S>(s0.npair, raw, slots, ct, c0, c1, c2, c3);
  return hmax;
}

__device__ __forceinline__ uint32_t exp_f64(const double2& x) {
  return max((uint32_t)__double2hiint(x.x) & 0x7fffffffu, (uint32_t)__double2hiint(x.y) & 0x7fffffffu) >> 20;
}
__device__ __forceinline__ uint32_t exp_f32(const float2& x) {
  return max(__float_as_uint(x.x) & 0x7fffffffu, __float_as_uint(x.y) & 0x7fffffffu) >> 23;
}

// Source-class index (previous pass's binary-point array) of a thread's
// register 0 in stage st: XOR of its lane and warp bits' contributions.
template <class G, class S>
__device__ __forceinline__ uint32_t src_thread(const G& pd, const S& st, int lane, int warp) {
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i)
    if ((lane >> i) & 1) c ^= pd.src_w[st.lane[i]];
#pragma unroll
  for (int i = 0; i < pd.D - kMinTileBits; ++i)
    if ((warp >> i) & 1) c ^= pd.src_w[st.warp[i]];
  return c;
}

__device__ __forceinline__ uint32_t reg_src(int e, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  return ((e & 1) ? w0 : 0u) ^ ((e & 2) ? w1 : 0u) ^ ((e & 4) ? w2 : 0u) ^ ((e & 8) ? w3 : 0u);
}

__device__ __forceinline__ bool q_is_valid(int q) { return q > kQValidMin; }

// floor(v / 2^sh) (sh >= 0; 0 or -1 once sh >= 64)
__device__ __forceinline__ long long shr_floor(long long v, unsigned sh) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(sh));   // PTX clamps the amount at 64
  return r;
}

// v / 2^sh rounded toward zero (sh >= 0; 0 once sh >= 64): an odd function,
// so conjugate sums stay exactly conjugate
__device__ __forceinline__ long long shr_tz(long long v, unsigned sh) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  unsigned long long a = ((unsigned long long)v ^ s) - s;
  asm("shr.b64 %0, %0, %1;" : "+l"(a) : "r"(sh));   // PTX clamps the amount at 64
  return (long long)((a ^ s) - s);
}

// Tiles meeting an Inf or NaN run the IEEE fp64 butterfly instead (rounded
// every level, the paper's arithmetic), so non-finite inputs propagate as in
// IEEE arithmetic.  Out of line: never taken for finite data.  Elements are
// re-read: IEEE numbers as such, int64 sums of a previous pass converted with
// their class's binary point; a pass that hands on int64 sums marks all its
// classes of this tile as holding IEEE numbers.
template <bool kDec, bool kCg = false, bool kCl = false>
__device__ __noinline__ void ieee_tile(const PassDesc& pd, const PassArgs& args, void* matp, const int16_t* q_in,
                                       int16_t* q_out, long long tile, long long base, uint32_t sbase, int nbase,
                                       unsigned char* smem, int lane, int warp) {
  double2 raw[kElems];
  load_tile<kCg>(pd, matp, base, lane, warp, raw);
  if (q_in != nullptr) {
    const Stage& s0 = pd.st[0];
    const uint32_t sb = sbase ^ src_thread(pd, s0, lane, warp);
    const uint32_t w0 = pd.src_w[s0.reg[0]], w1 = pd.src_w[s0.reg[1]], w2 = pd.src_w[s0.reg[2]],
                   w3 = pd.src_w[s0.reg[3]];
    for (int e = 0; e < kElems; ++e) {
      const int q = ld_in<kCg>(q_in + (sb ^ reg_src(e, w0, w1, w2, w3)));
      if (q == kQIeee) continue;
      if (!q_is_valid(q)) { raw[e] = make_double2(0.0, 0.0); continue; }
      raw[e].x = FixedArith::to_double_int(__double_as_longlong(raw[e].x), -q);
      raw[e].y = FixedArith::to_double_int(__double_as_longlong(raw[e].y), -q);
    }
  }
  const bool last = q_out == nullptr;
  const double mul = kDec ? pow2d(-pd.K) : (last ? pow2d(args.out_pow2) * args.out_mul : 1.0);
  finish_tile<F64Arith, kDec, kCl>(pd, args, matp, raw, mul, base, nbase, smem, lane, warp);
  if (!last && (!kCl || cluster_rank() == 0)) {
    const long long ncls = 1ll << (pd.D - pd.K);
    for (long long c = threadIdx.x; c < ncls; c += blockDim.x) q_out[(tile << (pd.D - pd.K)) + c] = (int16_t)kQIeee;
  }
}

// The tile's elements in the stage-0 mapping from a shared-memory copy.
template <class G, class Store>
__device__ __forceinline__ void load_tile_smem(const G& pd, const unsigned char* buf, int lane, int warp,
                                               Store (&raw)[kElems]) {
  const auto& s0 = pd.st[0];
  const Store* b = reinterpret_cast<const Store*>(buf);
  const int t = thread_sidx(pd, s0, lane, warp);
  const int w0 = 1 << s0.reg[0], w1 = 1 << s0.reg[1], w2 = 1 << s0.reg[2], w3 = 1 << s0.reg[3];
#pragma unroll
  for (int e = 0; e < kElems; ++e) raw[e] = b[t + reg_off(e, w0, w1, w2, w3)];
}

// Flags of the next pass's tiles that receive a nonzero (zero skipping).
template <class G, class NonZero>
__device__ __forceinline__ void flag_next(const G& pd, const PassArgs& args, int nbase, int lane, int warp,
                                          NonZero nz_of) {
  const auto& sl = pd.st[pd.nstage - 1];
  const int nt = nbase + thread_next(pd, sl, lane, warp);
  int n0 = pd.next_w[sl.reg[0]], n1 = pd.next_w[sl.reg[1]], n2 = pd.next_w[sl.reg[2]], n3 = pd.next_w[sl.reg[3]];
  twist_add(sl, lane, n0, n1, n2, n3, [&](int pos) { return (int)pd.next_w[pos]; });
  bool lanes_inside = true;
#pragma unroll
  for (int i = 0; i < kLaneBits; ++i) lanes_inside &= (pd.next_w[sl.lane[i]] == 0);
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    const bool nz = nz_of(e);
    const int id = nt + reg_off(e, n0, n1, n2, n3);
    if (lanes_inside) {
      if (__any_sync(kFull, nz) && lane == 0) args.flags_out[id] = 1;
    } else if (nz) {
      args.flags_out[id] = 1;
    }
  }
}

// Tile-wide reduction of the flags (OR) and of the range [lo, hi] of the
// nonzero class slots, through red[0..S) / red[S..2S) / red[2S..3S), S = kRedStride (one
// entry per warp; a two-CTA cluster writes its entries into both CTAs at the
// one-CTA layout's warp index and meets at a cluster barrier).
template <bool kCl>
__device__ __forceinline__ void tile_reduce(int* red, int warp, int lane, int nwarps_total, int& tb, int& lo,
                                            int& hi) {
  tb = __reduce_or_sync(kFull, tb);
  lo = (int)__reduce_min_sync(kFull, (unsigned)lo);
  hi = (int)__reduce_max_sync(kFull, (unsigned)hi);
  if (lane == 0) {
    red[warp] = tb; red[kRedStride + warp] = lo; red[2 * kRedStride + warp] = hi;
    if constexpr (kCl) {
      int* pr = peer_smem(red);
      pr[warp] = tb; pr[kRedStride + warp] = lo; pr[2 * kRedStride + warp] = hi;
    }
  }
  if constexpr (kCl) cluster_sync();
  else __syncthreads();
  // lane w reads warp w's entries; one warp-wide reduction each
  const bool in = lane < nwarps_total;
  tb = (int)__reduce_or_sync(kFull, in ? (unsigned)red[lane] : 0u);
  lo = (int)__reduce_min_sync(kFull, in ? (unsigned)red[kRedStride + lane] : 0x7fffffffu);
  hi = (int)__reduce_max_sync(kFull, in ? (unsigned)red[2 * kRedStride + lane] : 0u);
}

// Asynchronous copies of a tile's elements into shared memory (the
// prefetching pass forms): each thread copies its own stage-0 elements.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class G>
__device__ __forceinline__ long long tile_base(const G& pd, long long tile) {
  long long base = 0;
  for (int j = 0; j < pd.nrest; ++j)
    if ((tile >> j) & 1) base += 1ll << pd.rest_gbit[j];
  return base;
}

// This thread's 16 elements of `tile` (stage-0 positions) into buf.
template <class G>
__device__ __forceinline__ void prefetch_tile(const G& pd, const void* matp, long long tile, unsigned char* buf,
                                              int lane, int warp) {
  const auto& s0 = pd.st[0];
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

// One complex128 tile of the block fixed point, in the role kRole (IEEE
// numbers or int64 sums in, IEEE numbers or int64 sums out).
// xbuf: exchange area (2^D x 16 bytes; a two-CTA cluster: half of it per
// CTA); red: 64 ints; cls: 2^(D-K) class slots; inbuf: the tile already in
// shared memory (stage-0 positions), or nullptr to read it from global memory.
// sbase: the tile-id bits' part of the source-class index (kRoleIntIn).
// kCl: one CTA of a two-CTA cluster (warp: the virtual warp, rank * 8 + the
// CTA's own warp); each CTA keeps the class maxima of its own elements and
// merges the peer's through distributed shared memory.
//
// Class slots: IEEE input, the class's largest exponent field E (binary point
// q_in = max(E, 1) + K - 1084, where the largest lands below 2^(62-K));
// int64 input, the largest source binary point + kQSlot (q_in = that point +
// K: every element shifts right by at least K bits, toward zero, after which
// the 2^K-term sums stay below 2^62), 0 for a class whose sources are all zero.

template <bool kDec, int kRole, bool kCg = false, bool kCl = false, class G>
__device__ __forceinline__ void fixed_tile(const G& pd, const PassArgs& args, void* matp, const int16_t* q_in,
                                           int16_t* q_out, long long tile, long long base, uint32_t sbase,
                                           int nbase, const unsigned char* inbuf, unsigned char* xbuf, int* red,
                                           int* cls, int lane, int warp, long long pf_tile = -1) {
  using V = FixedArith::V;
  // pf_tile >= 0 (persistent form): once every thread is done with the
  // exchange area, copy that tile's elements into it for the next round
  auto prefetch_next = [&]() {
    if (pf_tile >= 0) {
      __syncthreads();
      prefetch_tile(pd, matp, pf_tile, xbuf, lane, warp);
    }
  };
  constexpr bool kIntIn = (kRole & kRoleIntIn) != 0;
  constexpr bool kIntOut = (kRole & kRoleIntOut) != 0;
  const int nthr = blockDim.x;
  const int nwarps_total = 1 << (pd.D - kMinTileBits);   // warps of the tile (both CTAs of a cluster)
  const int ncls = 1 << (pd.D - pd.K);
  for (int i = threadIdx.x; i < ncls; i += nthr) cls[i] = 0;
  int slot_lo, slot_hi;                                  // range of the tile's nonzero class slots
  const auto& s0 = pd.st[0];
  const int ct = cls_thread(pd, s0, lane, warp);
  const int c0 = pd.cls_w[s0.reg[0]], c1 = pd.cls_w[s0.reg[1]], c2 = pd.cls_w[s0.reg[2]],
            c3 = pd.cls_w[s0.reg[3]];
  const int np = s0.npair;
  V v[kElems];
  int tb;                                                // tile flags: 1 nonzero, 2 Inf / NaN
  if constexpr (!kIntIn) {
    // ---- IEEE doubles: class maxima of the exponent fields
    double2 raw[kElems];
    if (inbuf) load_tile_smem(pd, inbuf, lane, warp, raw);
    else load_tile<kCg>(pd, matp, base, lane, warp, raw);
    if constexpr (kCl) cluster_wait();                   // the peer CTA is running
    __syncthreads();                                     // class slots cleared
    int lo;
    const uint32_t hmax = class_max<ExpSlot64>(pd, raw, cls, lane, warp, exp_f64, lo);
    uint32_t nzw = 0;
    if (args.skip_zero) {
#pragma unroll
      for (int e = 0; e < kElems; ++e)
        nzw |= (uint32_t)__double2hiint(raw[e].x) << 1 | (uint32_t)__double2loint(raw[e].x) |
               (uint32_t)__double2hiint(raw[e].y) << 1 | (uint32_t)__double2loint(raw[e].y);
    }
    tb = (nzw != 0 ? 1 : 0) | (hmax == 2047 ? 2 : 0);
    int hi = (int)hmax;
    tile_reduce<kCl>(red, warp, lane, nwarps_total, tb, lo, hi);   // both CTAs' atomics and flags are in
    slot_lo = lo;
    slot_hi = hi;
    if ((args.skip_zero && !(tb & 1)) || (tb & 2)) {
      if (tb & 2)
        ieee_tile<kDec, kCg, kCl>(raw_desc(pd), args, matp, q_in, q_out, tile, base, sbase, nbase, xbuf, lane, warp);
      prefetch_next();
      return;                                            // (else all +-0: the outputs are zero already)
    }
    if constexpr (kCl) {
      const int* pcls = peer_smem(cls);
      for (int i = threadIdx.x; i < ncls; i += nthr) cls[i] = max(cls[i], pcls[i]);
      cluster_sync();                                    // both CTAs are done with the peer's slots
    }
    // onto the classes' binary points: x * 2^S_c, S_c = 1084 - K - max(E_c, 1)
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const int sb = 9 - pd.K - max(cls[ct ^ reg_cls(e, c0, c1, c2, c3)], 1);
      v[e].re = FixedArith::to_fixed(raw[e].x, sb);
      v[e].im = FixedArith::to_fixed(raw[e].y, sb);
    }
  } else {
    // ---- int64 sums of a previous pass, each with its source class's binary point
    longlong2 raw[kElems];
    int qs[kElems];
    if (inbuf) load_tile_smem(pd, inbuf, lane, warp, raw);
    else load_tile<kCg>(pd, matp, base, lane, warp, raw);
    {
      const uint32_t sb = sbase ^ src_thread(pd, s0, lane, warp);
      const uint32_t w0 = pd.src_w[s0.reg[0]], w1 = pd.src_w[s0.reg[1]], w2 = pd.src_w[s0.reg[2]],
                     w3 = pd.src_w[s0.reg[3]];
#pragma unroll
      for (int e = 0; e < kElems; ++e) qs[e] = ld_in<kCg>(q_in + (sb ^ reg_src(e, w0, w1, w2, w3)));
    }
    if constexpr (kCl) cluster_wait();                   // the peer CTA is running
    __syncthreads();                                     // class slots cleared
    int any_valid = 0, any_ieee = 0, lo = 0x7fffffff, hi = 0;
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const bool ok = q_is_valid(qs[e]);
      any_valid |= ok;
      any_ieee |= qs[e] == kQIeee;
      lo = min(lo, ok ? qs[e] + kQSlot : 0x7fffffff);
      hi = max(hi, ok ? qs[e] + kQSlot : 0);
    }
    class_atomics_any<QSlot>(np, qs, cls, ct, c0, c1, c2, c3);
    tb = (any_valid ? 1 : 0) | (any_ieee ? 2 : 0);
    tile_reduce<kCl>(red, warp, lane, nwarps_total, tb, lo, hi);
    slot_lo = lo;
    slot_hi = hi;
    if (tb & 2) {
      ieee_tile<kDec, kCg, kCl>(raw_desc(pd), args, matp, q_in, q_out, tile, base, sbase, nbase, xbuf, lane, warp);
      prefetch_next();
      return;
    }
    if (args.skip_zero && !(tb & 1)) {                   // every source class was zero
      prefetch_next();
      return;
    }
    if constexpr (kCl) {
      const int* pcls = peer_smem(cls);
      for (int i = threadIdx.x; i < ncls; i += nthr) cls[i] = max(cls[i], pcls[i]);
      cluster_sync();
    }
    // realign onto q_in_c = (largest source point) + K.  Conjugate partners
    // (Hermitian inputs) have equal real parts and opposite imaginary parts:
    // the real parts may round toward -inf (two instructions), the imaginary
    // parts round toward zero (an odd function), and conjugate sums stay
    // exactly conjugate
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const int q = qs[e];
      if (q_is_valid(q)) {
        const unsigned sh = (unsigned)(cls[ct ^ reg_cls(e, c0, c1, c2, c3)] - kQSlot + pd.K - q);
        v[e].re = shr_floor(raw[e].x, sh);
        v[e].im = shr_tz(raw[e].y, sh);
      } else {
        v[e].re = 0; v[e].im = 0;
      }
    }
  }
  // binary point of class c: q_in_c; the outputs hold q_in_c - K (decomposition:
  // the 1/2 of Eq. 4 per level) or q_in_c (composition)
  auto q_of_slot = [&](int slot) {
    if constexpr (kIntIn) return slot - kQSlot + pd.K;
    else return max(slot, 1) + pd.K - 1084;
  };
  if constexpr (kIntOut) {
    if (!kCl || cluster_rank() == 0) {
      int16_t* qo = q_out + (tile << (pd.D - pd.K));
      for (int c = threadIdx.x; c < ncls; c += nthr) {
        const int slot = cls[c];
        qo[c] = (int16_t)((kIntIn && slot == 0) ? kQValidMin : q_of_slot(slot) - (kDec ? pd.K : 0));
      }
    }
  }

  // ---- the pass's levels, exact
  V* sm = reinterpret_cast<V*>(xbuf);
#pragma unroll
  for (int s = 0; s < pd.nstage; ++s) {
    if (s > 0) exchange<kCl>(v, pd, pd.st[s - 1], pd.st[s], sm, lane, warp, s > 1);
    if (s == pd.nstage - 1) prefetch_next();             // the last stage works in registers
    stage_levels<FixedArith, kDec>(v, pd.st[s], lane);
  }

  // ---- store in place: int64 sums, or rounded once
  const auto& sl = pd.st[pd.nstage - 1];
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, sl, lane, warp);
  uint32_t w0 = 1u << pd.gbit[sl.reg[0]], w1 = 1u << pd.gbit[sl.reg[1]];
  uint32_t w2 = 1u << pd.gbit[sl.reg[2]], w3 = 1u << pd.gbit[sl.reg[3]];
  twist_add(sl, lane, w0, w1, w2, w3, [&](int pos) { return 1u << pd.gbit[pos]; });
  if constexpr (kIntOut) {
    longlong2* mat = reinterpret_cast<longlong2*>(matp);
#pragma unroll
    for (int e = 0; e < kElems; ++e) mat[g + reg_off(e, w0, w1, w2, w3)] = make_longlong2(v[e].re, v[e].im);
  } else {
    // value = sum * 2^q_out_c * 2^out_pow2 (a composition's scale)
    const int cl = cls_thread(pd, sl, lane, warp);
    int l0 = pd.cls_w[sl.reg[0]], l1 = pd.cls_w[sl.reg[1]], l2 = pd.cls_w[sl.reg[2]], l3 = pd.cls_w[sl.reg[3]];
    twist_xor(sl, l0, l1, l2, l3, [&](int pos) { return (int)pd.cls_w[pos]; });
    const bool resid = args.out_mul != 1.0;              // non-power-of-two composition scale (rare)
    double2* mat = reinterpret_cast<double2*>(matp);
    // T of a class, -(q_out + out_pow2), falls as its slot rises; zero
    // classes (all of whose sums are 0) round to 0 at any T
    const int tadj = -(kDec ? pd.K : 0) + args.out_pow2;
    const bool fast = !resid && (slot_hi < slot_lo || (FixedArith::fast_range(-(q_of_slot(slot_hi) + tadj)) &&
                                                       FixedArith::fast_range(-(q_of_slot(slot_lo) + tadj))));
    if (fast) {
      // real parts through the fp64 conversion unit, imaginary parts through
      // integer instructions (identical roundings): the two pipes share the
      // conversions
#pragma unroll
      for (int e = 0; e < kElems; ++e) {
        const int T = -(q_of_slot(cls[cl ^ reg_cls(e, l0, l1, l2, l3)]) + tadj);
        mat[g + reg_off(e, w0, w1, w2, w3)] =
            make_double2(FixedArith::to_double_cvt_fast(v[e].re, T), FixedArith::to_double_fast(v[e].im, T));
      }
    } else {
      for (int e = 0; e < kElems; ++e) {
        const int T = -(q_of_slot(cls[cl ^ reg_cls(e, l0, l1, l2, l3)]) + tadj);
        mat[g + reg_off(e, w0, w1, w2, w3)] = FixedArith::to_double2_rare(v[e].re, v[e].im, T, args.out_mul);
      }
    }
  }
  if (args.flags_out != nullptr) flag_next(pd, args, nbase, lane, warp, [&](int e) { return (v[e].re | v[e].im) != 0; });
}

// One complex64 tile of the block fixed point: class c on the binary point
// S_c = 188 - K - max(E_c, 1) (E_c its largest float exponent field): x * 2^S_c
// is exact for components within 2^(38-K) of the class's largest, the
// largest lands below 2^(62-K), the sums are exact in int64, and every output
// is rounded to float once (RNE).  Tiles meeting an Inf or NaN run the IEEE
// float butterfly instead.
template <bool kDec, bool kCg, class G>
__device__ __forceinline__ void fixed32_tile(const G& pd, const PassArgs& args, void* matp, long long base,
                                             int nbase, unsigned char* smem, int* red, int* cls, int lane, int warp) {
  using V = Fixed32Arith::V;
  const int nthr = blockDim.x, nwarps = nthr >> 5;
  const int ncls = 1 << (pd.D - pd.K);
  for (int i = threadIdx.x; i < ncls; i += nthr) cls[i] = 0;
  float2 raw[kElems];
  load_tile<kCg>(pd, matp, base, lane, warp, raw);
  __syncthreads();                                       // class slots cleared
  int lo_unused;
  const uint32_t hmax = class_max<ExpSlot32>(pd, raw, cls, lane, warp, exp_f32, lo_unused);
  uint32_t nzw = 0;
  if (args.skip_zero) {
#pragma unroll
    for (int e = 0; e < kElems; ++e) nzw |= (__float_as_uint(raw[e].x) | __float_as_uint(raw[e].y)) << 1;
  }
  int t = (nzw != 0 ? 1 : 0) | (hmax == 255 ? 2 : 0), hi_unused = 0;
  tile_reduce<false>(red, warp, lane, nwarps, t, lo_unused, hi_unused);
  if (args.skip_zero && !(t & 1)) return;                // all +-0: the outputs are zero already
  if (t & 2) {                                           // Inf/NaN in the tile
    finish_tile<F32Arith, kDec>(pd, args, matp, raw, kDec ? pow2d(-pd.K) : pow2d(args.out_pow2) * args.out_mul,
                                base, nbase, smem, lane, warp);
    return;
  }
  V v[kElems];
  {
    const auto& s0 = pd.st[0];
    const int ct = cls_thread(pd, s0, lane, warp);
    const int c0 = pd.cls_w[s0.reg[0]], c1 = pd.cls_w[s0.reg[1]], c2 = pd.cls_w[s0.reg[2]],
              c3 = pd.cls_w[s0.reg[3]];
#pragma unroll
    for (int e = 0; e < kElems; ++e) {
      const int rs_base = max(cls[ct ^ reg_cls(e, c0, c1, c2, c3)], 1) + pd.K;
      v[e].re = Fixed32Arith::to_fixed(raw[e].x, rs_base);
      v[e].im = Fixed32Arith::to_fixed(raw[e].y, rs_base);
    }
  }
  V* sm = reinterpret_cast<V*>(smem);
#pragma unroll
  for (int s = 0; s < pd.nstage; ++s) {
    if (s > 0) exchange(v, pd, pd.st[s - 1], pd.st[s], sm, lane, warp, s > 1);
    stage_levels<Fixed32Arith, kDec>(v, pd.st[s], lane);
  }
  // value = sum * 2^-S_c, times 2^-K for the 1/2 of Eq. 4 per level, times
  // 2^out_pow2 for a composition's scale
  const int tbase = 188 - pd.K + (kDec ? pd.K : 0) - args.out_pow2;
  const bool resid = args.out_mul != 1.0;
  const auto& sl = pd.st[pd.nstage - 1];
  float2* mat = reinterpret_cast<float2*>(matp);
  const uint32_t g = (uint32_t)base + (uint32_t)thread_goff(pd, sl, lane, warp);
  uint32_t w0 = 1u << pd.gbit[sl.reg[0]], w1 = 1u << pd.gbit[sl.reg[1]];
  uint32_t w2 = 1u << pd.gbit[sl.reg[2]], w3 = 1u << pd.gbit[sl.reg[3]];
  twist_add(sl, lane, w0, w1, w2, w3, [&](int pos) { return 1u << pd.gbit[pos]; });
  const int cl = cls_thread(pd, sl, lane, warp);
  int l0 = pd.cls_w[sl.reg[0]], l1 = pd.cls_w[sl.reg[1]], l2 = pd.cls_w[sl.reg[2]], l3 = pd.cls_w[sl.reg[3]];
  twist_xor(sl, l0, l1, l2, l3, [&](int pos) { return (int)pd.cls_w[pos]; });
#pragma unroll
  for (int e = 0; e < kElems; ++e) {
    const int T = tbase - max(cls[cl ^ reg_cls(e, l0, l1, l2, l3)], 1);
    // real parts on the conversion unit, imaginary parts with integer
    // instructions (identical roundings)
    const bool fast = Fixed32Arith::fast_range(T) || v[e].re == 0;
    float2 o = make_float2(fast ? Fixed32Arith::to_float_cvt_fast(v[e].re, T) : Fixed32Arith::to_float(v[e].re, T),
                           Fixed32Arith::to_float(v[e].im, T));
    if (resid) { o.x = __fmul_rn(o.x, (float)args.out_mul); o.y = __fmul_rn(o.y, (float)args.out_mul); }
    mat[g + reg_off(e, w0, w1, w2, w3)] = o;
  }
  if (args.flags_out != nullptr) flag_next(pd, args, nbase, lane, warp, [&](int e) { return (v[e].re | v[e].im) != 0; });
}

// One tile of a pass: its position from the tile id, then the arithmetic's
// load / levels / store.  smem: the exchange area (2^D x 16 bytes; half of it
// per CTA of a two-CTA cluster), 64 ints of reduction slots, then (block fixed
// point) 2^(D-K) class slots.
template <class A, bool kDec, int kRole, bool kCg, bool kCl = false, class G>
__device__ __forceinline__ void pass_tile(const G& pd, const PassArgs& args, void* matp, const int16_t* q_in,
                                          int16_t* q_out, long long tile, unsigned char* smem, int lane, int warp) {
  using Store = typename A::Store;
  static_assert(!(kCl && A::kFixed32), "two-CTA clusters serve complex128 tiles only");
  int* red = reinterpret_cast<int*>(smem + ((size_t)16 << (pd.D - (kCl ? 1 : 0))));
  int* cls = red + kRedInts;
  long long base = 0;
  int nbase = 0;
  uint32_t sbase = 0;
  for (int j = 0; j < pd.nrest; ++j)
    if ((tile >> j) & 1) {
      base += 1ll << pd.rest_gbit[j];
      nbase += (int)pd.next_rest_w[j];
      sbase ^= pd.src_rest_w[j];
    }

  if constexpr (A::kFixed) {
    fixed_tile<kDec, kRole, kCg, kCl>(pd, args, matp, q_in, q_out, tile, base, sbase, nbase, nullptr, smem, red,
                                      cls, lane, warp);
  } else if constexpr (A::kFixed32) {
    fixed32_tile<kDec, kCg>(pd, args, matp, base, nbase, smem, red, cls, lane, warp);
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
// budget); the planner picks it per pass.
// kShape: a compiled layout (tpd_shape.h) the launcher has matched to pd, or
// -1 (the layout read from pd at run time).
template <class A, bool kDec, int kThreads, int kMinBlocks, int kRole = 0, int kShape = -1>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    k_pass(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long tile = (long long)blockIdx.x + (long long)blockIdx.y * gridDim.x;
  void* matp = args.mat;
  const int16_t* q_in = args.q_in;
  int16_t* q_out = args.q_out;
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
  if constexpr (kShape < 0) {
    pass_tile<A, kDec, kRole, false>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
  } else {
    static_assert((1 << (ShapeT<kShape>::kD - kRegBits)) <= kThreads, "compiled shapes are tiles of one CTA");
    pass_tile<A, kDec, kRole, false>(GeoCT<ShapeT<kShape>>(pd), args, matp, q_in, q_out, tile, smem, lane, warp);
  }
}

// Complex128 tiles of 2^13 elements as two-CTA clusters of 256 threads (see
// the top of this file): grid = 2 x tiles, tile = cluster index.
template <class A, bool kDec, int kRole = 0, int kShape = -1>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kClThreads, 2)
    k_pass_cl(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31;
  const int warp = (int)(cluster_rank() << kClWarpBit) | (tid >> 5);   // the one-CTA layout's warp
  long long tile = (long long)(blockIdx.x >> 1);
  void* matp = args.mat;
  const int16_t* q_in = args.q_in;
  int16_t* q_out = args.q_out;
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
  if constexpr (kShape < 0)
    pass_tile<A, kDec, kRole, false, true>(pd, args, matp, q_in, q_out, tile, smem, lane, warp);
  else
    pass_tile<A, kDec, kRole, false, true>(GeoCT<ShapeT<kShape>>(pd), args, matp, q_in, q_out, tile, smem, lane,
                                           warp);
}

// -------------------------------------------------------------- persistent, double buffered
//
// Fixed point, one matrix, tiles of up to 2^12 elements: one CTA per SM walks
// the tiles (tile += gridDim.x).  Each thread copies ITS elements of the next
// tile into the spare shared-memory buffer with cp.async while the CTA works
// on the current one, so HBM stays busy across the compute phase.  The waits
// are the hardware's (cp.async.wait_group + barrier), with no spin loops.

template <bool kDec, int kRole>
__global__ void __launch_bounds__(kStdThreads, 1)
    k_pass_pipe(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t tb = (size_t)16 << pd.D;
  unsigned char* buf0 = smem;
  unsigned char* buf1 = smem + tb;
  int* red = reinterpret_cast<int*>(smem + 2 * tb);
  int* cls = red + kRedInts;
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
    long long base = 0;
    int nbase = 0;
    uint32_t sbase = 0;
    for (int j = 0; j < pd.nrest; ++j)
      if ((tile >> j) & 1) {
        base += 1ll << pd.rest_gbit[j];
        nbase += (int)pd.next_rest_w[j];
        sbase ^= pd.src_rest_w[j];
      }
    fixed_tile<kDec, kRole>(pd, args, args.mat, args.q_in, args.q_out, tile, base, sbase, nbase, cur, cur, red, cls,
                            lane, warp);
    __syncthreads();                      // the current buffer is refilled next iteration
  }
}

// Persistent form of the block-fixed-point pass for a compiled layout (one
// matrix, every tile: no zero skipping, partial masks or L2 chunks): a CTA
// walks the tiles tile += gridDim.x, two CTAs per SM.  Each tile arrives in the
// exchange area through cp.async, issued by the previous tile once its last
// exchange has been read, so the copy runs while that tile's last stage, its
// rounding and its stores execute; the waits are cp.async.wait_group and
// barriers only.
template <bool kDec, int kRole, int kShape>
__global__ void __launch_bounds__(kStdThreads, kOccLow)
    k_pass_pf(const __grid_constant__ PassDesc pd, const __grid_constant__ PassArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const GeoCT<ShapeT<kShape>> g(pd);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* buf = smem;
  int* red = reinterpret_cast<int*>(smem + ((size_t)16 << ShapeT<kShape>::kD));
  int* cls = red + kRedInts;
  long long tile = blockIdx.x;
  if (tile >= pd.ntiles) return;
  prefetch_tile(g, args.mat, tile, buf, lane, warp);
  for (; tile < pd.ntiles; tile += gridDim.x) {
    cp_async_wait<0>();
    __syncthreads();                      // the tile is in shared memory, everyone's copies included
    long long base = 0;
    int nbase = 0;
    uint32_t sbase = 0;
    for (int j = 0; j < pd.nrest; ++j)
      if ((tile >> j) & 1) {
        base += 1ll << pd.rest_gbit[j];
        nbase += (int)pd.next_rest_w[j];
        sbase ^= pd.src_rest_w[j];
      }
    const long long nxt = tile + gridDim.x;
    fixed_tile<kDec, kRole>(g, args, args.mat, args.q_in, args.q_out, tile, base, sbase, nbase, buf, buf, red, cls,
                            lane, warp, nxt < pd.ntiles ? nxt : -1);
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

// All n levels of a whole matrix in shared memory.  Block fixed point: the
// element (r, c) belongs to the class r xor c (its X-mask: every level keeps
// it), and cls[x] holds that class's largest exponent field.
template <class A, bool kDec>
__device__ __forceinline__ void small_run(typename A::Store* mat, int n, int scale_mode, unsigned char* smem,
                                          const int* cls, int tid, int nthr) {
  using V = typename A::V;
  V* sm = reinterpret_cast<V*>(smem);
  const int count = 1 << (2 * n), cmask = (1 << n) - 1;
  for (int i = tid; i < count; i += nthr) {
    const typename A::Store x = mat[i];
    if constexpr (A::kFixed) {
      // x * 2^S with S = 1084 - n - E: headroom for the 2^n-term sums of n levels
      const int sb = 9 - n - max(cls[(i >> n) ^ (i & cmask)], 1);
      V t;
      t.re = A::to_fixed(x.x, sb);
      t.im = A::to_fixed(x.y, sb);
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
      // the output is sum * 2^-S, times 2^-n for the decomposition (the 1/2
      // of Eq. 4 per level) or for a composition scaled to the adjoint
      const int S = 1084 - n - max(cls[(i >> n) ^ (i & cmask)], 1);
      const int T = (kDec || scale_mode) ? S + n : S;
      o.x = A::to_double(sm[i].re, T);
      o.y = A::to_double(sm[i].im, T);
    } else {
      o = A::store(sm[i], OutScale{0, 1.0}, mul);
    }
    mat[i] = o;
  }
}

// A whole matrix of n <= 6 qubits by the CTA's nthr threads (all of them call
// it): nonzero test (and, block fixed point, the class maxima and the IEEE
// fallback for Inf/NaN), then small_run.  smem: 4^n elements of A::V, then
// (block fixed point) 2^n class slots.
template <class A, bool kDec>
__device__ __forceinline__ void small_matrix(typename A::Store* mat, int n, int skip_zero, int scale_mode,
                                             unsigned char* smem, int tid, int nthr) {
  using Store = typename A::Store;
  const int count = 1 << (2 * n);
  if constexpr (A::kFixed) {
    int* cls = reinterpret_cast<int*>(smem + ((size_t)16 << (2 * n)));
    const int cmask = (1 << n) - 1;
    for (int i = tid; i <= cmask; i += nthr) cls[i] = 0;
    __syncthreads();
    uint32_t hmax = 0, nzw = 0;
    for (int i = tid; i < count; i += nthr) {
      const double2 x = mat[i];
      const uint32_t ex = exp_f64(x);
      hmax = max(hmax, ex);
      nzw |= (uint32_t)__double2hiint(x.x) << 1 | (uint32_t)__double2loint(x.x) |
             (uint32_t)__double2hiint(x.y) << 1 | (uint32_t)__double2loint(x.y);
      if (ex) atomicMax(cls + ((i >> n) ^ (i & cmask)), (int)ex);
    }
    const int nz = __syncthreads_or(nzw != 0);
    const int inf = __syncthreads_or(hmax == 2047);
    if (skip_zero && !nz) return;
    if (inf) {
      small_run<F64Arith, kDec>(mat, n, scale_mode, smem, nullptr, tid, nthr);
      return;
    }
    small_run<A, kDec>(mat, n, scale_mode, smem, cls, tid, nthr);
  } else {
    uint32_t nzw = 0;
    for (int i = tid; i < count; i += nthr) {
      const Store x = mat[i];
      if constexpr (sizeof(Store) == 16) {
        nzw |= (uint32_t)__double2hiint(((const double2&)x).x) << 1 | (uint32_t)__double2loint(((const double2&)x).x) |
               (uint32_t)__double2hiint(((const double2&)x).y) << 1 | (uint32_t)__double2loint(((const double2&)x).y);
      } else {
        nzw |= (__float_as_uint(((const float2&)x).x) | __float_as_uint(((const float2&)x).y)) << 1;
      }
    }
    const int nz = __syncthreads_or(nzw != 0);
    if (skip_zero && !nz) return;
    small_run<A, kDec>(mat, n, scale_mode, smem, nullptr, tid, nthr);
  }
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
