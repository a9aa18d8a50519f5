// Sparse input: the decomposition of a matrix given by its nonzero entries
// (COO), level by level as in the paper's iterative algorithm (Alg. 2, the
// CMWs of Eq. 4), keeping only nonzero entries -- the zero-CMW pruning that
// gives the paper's O(m n p) cost for m nonzero entries and p contributing
// strings (Sec. IV).
//
// An entry is (key, value): key = the element's flat index r*N + c in the
// "RC" numbering, where after a qubit level beta the row / column bits
// (r_beta, c_beta) hold that level's Pauli label (I (0,0), X (0,1), Y (1,0),
// Z (1,1)) instead of the index bits.  One level maps an entry at (r_beta,
// c_beta) to two entries of its quad (Eq. 4 without the 1/2, applied once at
// the end as 2^-n):
//     a00 -> I +v, Z +v     a11 -> I +v, Z -v
//     a01 -> X +v, Y +iv    a10 -> X +v, Y -iv
// Entries with equal keys are summed in a hash table, zero sums dropped.
//
// Exactness: values are int64 on one binary point per X-mask x = r xor c
// (x * 2^S_x, S_x = 1084 - n - the largest exponent among the entries of that
// X-mask, like a fixed-point pass with K = n).  A level never changes an
// entry's X-mask (Eq. 4: I, Z keep r_beta xor c_beta = 0, X, Y keep 1), so
// every sum adds values on one binary point: the sums are exact and
// independent of the order the atomics land in, and a weight's truncation
// error is bounded by its own X-mask's entries.  The weights are rounded to
// double once, at the end.  The output list is
// sorted by string index (bitonic sort), so it does not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tpd_launch.h"

namespace tpd {

namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;      // keys are < 4^15

__device__ __forceinline__ uint32_t hash32(uint32_t k) {
  k ^= k >> 16; k *= 0x7feb352du; k ^= k >> 15; k *= 0x846ca68bu; k ^= k >> 16;
  return k;
}

// emax[x] = the largest exponent field among the entries of X-mask x = r xor c
// (emax: 2^n ints, zero on entry; the index is masked to n bits, so that rows
// or columns outside 0..2^n-1 cannot address outside the array)
__global__ void k_sp_emax(const int* __restrict__ rows, const int* __restrict__ cols,
                          const double2* __restrict__ vals, unsigned long long m, int n, int* __restrict__ emax) {
  const int xmask = (1 << n) - 1;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < m;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int ex = (int)((unsigned long long)__double_as_longlong(vals[i].x) >> 52) & 0x7FF;
    const int ey = (int)((unsigned long long)__double_as_longlong(vals[i].y) >> 52) & 0x7FF;
    const int e = max(ex, ey);
    if (e) atomicMax(emax + ((rows[i] ^ cols[i]) & xmask), e);
  }
}

// x * 2^S truncated toward zero, S = 1084 - n - emax_eff (|result| < 2^(62-n)):
// x = m * 2^(max(e,1) - 1075), and (m << 11) >> rs = x * 2^S for
// rs = 2 + n + emax_eff - max(e, 1) >= 3
__device__ __forceinline__ long long sp_to_fixed(double x, int n, int emax_eff) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(bits >> 52) & 0x7FF;
  const unsigned long long mnt = (bits & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
  const unsigned rs = (unsigned)(2 + n + emax_eff - max(e, 1));
  unsigned long long mag;
  const unsigned long long ml = mnt << 11;                         // < 2^64
  asm("shr.b64 %0, %1, %2;" : "=l"(mag) : "l"(ml), "r"(rs));       // clamps above 64: 0
  const unsigned long long s = (unsigned long long)((long long)bits >> 63);
  return (long long)((mag ^ s) - s);
}

// v * 2^-T rounded to nearest even (integer instructions, normal range or Inf / subnormal)
__device__ __forceinline__ double sp_to_double(long long v, int T) {
  if (v == 0) return 0.0;
  const unsigned long long s = (unsigned long long)(v >> 63);
  unsigned long long a = ((unsigned long long)v ^ s) - s;
  const int lz = __clzll((long long)a);
  a <<= lz;
  const int be = 1086 - lz - T;
  unsigned long long bits;
  if (be >= 1) {
    unsigned long long mant = a >> 11;
    const unsigned rem = (unsigned)a & 0x7FFu;
    mant += (unsigned long long)((rem > 0x400u) | ((rem == 0x400u) & (unsigned)mant));
    bits = be > 2046 ? 0x7FF0000000000000ull : ((unsigned long long)(be - 1) << 52) + mant;
    if (bits > 0x7FF0000000000000ull) bits = 0x7FF0000000000000ull;
  } else {
    const int rsh = 12 - be;
    if (rsh > 64) bits = 0;
    else if (rsh == 64) bits = a > 0x8000000000000000ull ? 1ull : 0ull;
    else {
      const unsigned long long mant = a >> rsh, rem = a & ((1ull << rsh) - 1), half = 1ull << (rsh - 1);
      bits = mant + (unsigned long long)((rem > half) | ((rem == half) & (mant & 1ull)));
    }
  }
  return __longlong_as_double((long long)(bits | (s & 0x8000000000000000ull)));
}

// initial entries: key = r*N + c, value on its X-mask's binary point
__global__ void k_sp_init(const int* __restrict__ rows, const int* __restrict__ cols, const double2* __restrict__ vals,
                          unsigned long long m, int n, const int* __restrict__ emax, uint32_t* __restrict__ keys,
                          longlong2* __restrict__ v) {
  const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int emax_eff = max(emax[(rows[i] ^ cols[i]) & ((1 << n) - 1)], 1);
  keys[i] = ((uint32_t)rows[i] << n) | (uint32_t)cols[i];
  v[i] = make_longlong2(sp_to_fixed(vals[i].x, n, emax_eff), sp_to_fixed(vals[i].y, n, emax_eff));
}

__device__ __forceinline__ void sp_insert(uint32_t key, long long re, long long im, uint32_t* __restrict__ tkeys,
                                          unsigned long long* __restrict__ tv, uint32_t mask,
                                          unsigned long long* __restrict__ overflow) {
  uint32_t slot = hash32(key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const uint32_t prev = atomicCAS(tkeys + slot, kEmpty, key);
    if (prev == kEmpty || prev == key) {
      atomicAdd(tv + 2 * slot, (unsigned long long)re);        // two's complement: exact int64 sums
      atomicAdd(tv + 2 * slot + 1, (unsigned long long)im);
      return;
    }
    slot = (slot + 1) & mask;
  }
  atomicExch(overflow, 1ull);                                  // table full (cannot happen when sized 2x)
}

// one qubit level: every entry emits its two children into the table
__global__ void k_sp_level(const uint32_t* __restrict__ keys, const longlong2* __restrict__ v,
                           const unsigned long long* __restrict__ count, unsigned long long cap, int n, int beta,
                           uint32_t* __restrict__ tkeys, unsigned long long* __restrict__ tv, uint32_t mask,
                           unsigned long long* __restrict__ overflow) {
  const unsigned long long E = min(*count, cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < E;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    const longlong2 x = v[i];
    const uint32_t cb = (k >> beta) & 1u, rb = (k >> (n + beta)) & 1u;
    const uint32_t base = k & ~((1u << beta) | (1u << (n + beta)));
    const uint32_t kI = base, kX = base | (1u << beta), kY = base | (1u << (n + beta)),
                   kZ = base | (1u << beta) | (1u << (n + beta));
    if (rb == cb) {
      sp_insert(kI, x.x, x.y, tkeys, tv, mask, overflow);                       // I += v
      if (rb) sp_insert(kZ, -x.x, -x.y, tkeys, tv, mask, overflow);             // Z -= a11
      else sp_insert(kZ, x.x, x.y, tkeys, tv, mask, overflow);                  // Z += a00
    } else {
      sp_insert(kX, x.x, x.y, tkeys, tv, mask, overflow);                       // X += v
      if (cb) sp_insert(kY, -x.y, x.x, tkeys, tv, mask, overflow);              // Y += i a01
      else sp_insert(kY, x.y, -x.x, tkeys, tv, mask, overflow);                 // Y -= i a10
    }
  }
}

// nonzero table entries -> the next level's entry list (any order); every
// slot is cleared after it is read, so the table starts the next level empty
__global__ void k_sp_compact(uint32_t* __restrict__ tkeys, unsigned long long* __restrict__ tv, uint32_t slots,
                             uint32_t* __restrict__ keys, longlong2* __restrict__ v,
                             unsigned long long* __restrict__ count_out, unsigned long long cap,
                             unsigned long long* __restrict__ overflow) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += gridDim.x * blockDim.x) {
    const uint32_t key = tkeys[s];
    if (key == kEmpty) continue;
    const long long re = (long long)tv[2 * s], im = (long long)tv[2 * s + 1];
    tkeys[s] = kEmpty;
    tv[2 * s] = 0ull;
    tv[2 * s + 1] = 0ull;
    if ((re | im) == 0) continue;                              // zero CMW: pruned
    const unsigned long long pos = atomicAdd(count_out, 1ull);
    if (pos < cap) { keys[pos] = key; v[pos] = make_longlong2(re, im); }
    else atomicExch(overflow, 1ull);
  }
}

// Counters (unsigned long long): [0] overflow flag, [1 + beta] entries
// entering level beta (beta = 0..n-1), [1 + n] the final entries.
constexpr int kSpCounters = 18;                                // n <= 15

// entries of the first level (the input's nonzeros, at most the capacity)
__global__ void k_sp_start(unsigned long long* ctr, unsigned long long m, unsigned long long cap) {
  ctr[1] = m < cap ? m : cap;
  if (m > cap) ctr[0] = 1ull;
}

// status word: TPD_ERR_WORKSPACE (4) if some level had more entries than the capacity
__global__ void k_sp_status(const unsigned long long* ctr, unsigned* status) { *status = ctr[0] ? 4u : 0u; }

// RC key -> base-4 string index (bit 2b = c_b, bit 2b+1 = r_b)
__device__ __forceinline__ unsigned long long sp_string(uint32_t key, int n) {
  unsigned long long s = 0;
  for (int b = 0; b < n; ++b) {
    s |= (unsigned long long)((key >> b) & 1u) << (2 * b);
    s |= (unsigned long long)((key >> (n + b)) & 1u) << (2 * b + 1);
  }
  return s;
}

// The final entries, sorted by string index: a bitonic sort over the
// entries padded to Pd = the power of two >= E (padding keys = max), E read on
// the device.  Steps whose stride is below kSpChunk run inside a CTA on its
// chunk of the keys in shared memory; the launches for sizes above Pd return
// at once, so the host plans the launches for the largest possible E.
constexpr int kSpChunk = 2048;                 // keys per CTA in shared memory
constexpr int kSpLocalThreads = kSpChunk / 2;  // one compare-exchange pair per thread

__device__ __forceinline__ unsigned long long sp_padded(const unsigned long long* final_count,
                                                        unsigned long long cap) {
  const unsigned long long E = min(*final_count, cap);
  unsigned long long P = 1;
  while (P < E) P <<= 1;
  return P;
}

// string keys of the final entries into the sort buffer (padding = max)
__global__ void k_sp_keys(const uint32_t* __restrict__ keys, const unsigned long long* __restrict__ final_count,
                          unsigned long long cap, int n, unsigned long long* __restrict__ skey,
                          uint32_t* __restrict__ sidx) {
  const unsigned long long E = min(*final_count, cap), P = sp_padded(final_count, cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < P;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    skey[i] = i < E ? sp_string(keys[i], n) : ~0ull;
    sidx[i] = (uint32_t)i;
  }
}

// one compare-exchange step (j >= kSpChunk, k) over the global buffer
__global__ void k_sp_bitonic(unsigned long long* __restrict__ skey, uint32_t* __restrict__ sidx,
                             const unsigned long long* __restrict__ final_count, unsigned long long cap,
                             unsigned long long j, unsigned long long k) {
  const unsigned long long P = sp_padded(final_count, cap);
  if (k > P) return;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < P;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long l = i ^ j;
    if (l <= i) continue;
    const bool up = (i & k) == 0;
    const unsigned long long a = skey[i], b = skey[l];
    if ((a > b) == up) {
      skey[i] = b; skey[l] = a;
      const uint32_t t = sidx[i]; sidx[i] = sidx[l]; sidx[l] = t;
    }
  }
}

// the steps j < kSpChunk of sizes k in [k_lo, k_hi] on each CTA's chunk, in
// shared memory (k_lo = 2, k_hi = kSpChunk: the chunks' own sort; k_lo =
// k_hi = k > kSpChunk: the end of a merge of size k)
__global__ void __launch_bounds__(kSpLocalThreads) k_sp_local(unsigned long long* __restrict__ skey,
                                                              uint32_t* __restrict__ sidx,
                                                              const unsigned long long* __restrict__ final_count,
                                                              unsigned long long cap, unsigned long long k_lo,
                                                              unsigned long long k_hi) {
  __shared__ unsigned long long sk[kSpChunk];
  __shared__ uint32_t si[kSpChunk];
  const unsigned long long P = sp_padded(final_count, cap);
  const unsigned long long base = (unsigned long long)blockIdx.x * kSpChunk;
  if (base >= P || k_lo > P) return;
  const unsigned cnt = (unsigned)min((unsigned long long)kSpChunk, P - base);   // a power of two
  for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) { sk[t] = skey[base + t]; si[t] = sidx[base + t]; }
  __syncthreads();
  const unsigned long long kmax = min(k_hi, P);
  for (unsigned long long k = k_lo; k <= kmax; k <<= 1) {
    for (unsigned long long j = min(k >> 1, (unsigned long long)kSpChunk >> 1); j > 0; j >>= 1) {
      const unsigned t = threadIdx.x;
      const unsigned i = (unsigned)((t / j) * 2 * j + (t % j));
      const unsigned l = i + (unsigned)j;
      if (l < cnt) {
        const bool up = ((base + i) & k) == 0;
        const unsigned long long a = sk[i], b = sk[l];
        if ((a > b) == up) {
          sk[i] = b; sk[l] = a;
          const uint32_t x = si[i]; si[i] = si[l]; si[l] = x;
        }
      }
      __syncthreads();
    }
  }
  for (unsigned t = threadIdx.x; t < cnt; t += blockDim.x) { skey[base + t] = sk[t]; sidx[base + t] = si[t]; }
}

__global__ void k_sp_emit(const uint32_t* __restrict__ keys, const longlong2* __restrict__ v,
                          const unsigned long long* __restrict__ final_count,
                          unsigned long long cap, const unsigned long long* __restrict__ skey,
                          const uint32_t* __restrict__ sidx, int n, const int* __restrict__ emax,
                          unsigned long long capacity, unsigned long long* __restrict__ strings,
                          double2* __restrict__ weights, unsigned long long* __restrict__ out_count) {
  const unsigned long long E = min(*final_count, cap);
  const uint32_t xmask = (1u << n) - 1;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < E && i < capacity;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t key = keys[sidx[i]];
    const longlong2 x = v[sidx[i]];
    // S_x of the input, and the 1/2 of Eq. 4 per level (the labels keep x = r xor c)
    const int T = 1084 - max(emax[((key >> n) ^ key) & xmask], 1);
    strings[i] = skey[i];
    weights[i] = make_double2(sp_to_double(x.x, T), sp_to_double(x.y, T));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *out_count = E;
}

unsigned grid_for(unsigned long long items) {
  unsigned long long b = (items + 255) / 256;
  if (b < 1) b = 1;
  return (unsigned)(b > 4096 ? 4096 : b);
}

}  // namespace

// Workspace: counters | entries (keys, values) | hash table (2x entries,
// power of two) | sort buffer (power of two >= entries).
struct SparseLayout {
  size_t ctr, emax, keys, vals, tkeys, tvals, skey, sidx, total;
  unsigned long long entries, slots, sortn;
};

static SparseLayout sparse_layout(unsigned long long max_entries) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  SparseLayout L;
  L.entries = max_entries < 1 ? 1 : max_entries;
  L.slots = 1;
  while (L.slots < 2 * L.entries) L.slots <<= 1;
  L.sortn = 1;
  while (L.sortn < L.entries) L.sortn <<= 1;
  size_t off = 0;
  L.ctr = off; off += al(kSpCounters * sizeof(unsigned long long));
  L.emax = off; off += al(sizeof(int) << 15);     // one per X-mask, n <= 15
  L.keys = off; off += al(L.entries * 4);
  L.vals = off; off += al(L.entries * 16);
  L.tkeys = off; off += al(L.slots * 4);
  L.tvals = off; off += al(L.slots * 16);
  L.skey = off; off += al(L.sortn * 8);
  L.sidx = off; off += al(L.sortn * 4);
  L.total = off;
  return L;
}

size_t sparse_workspace_bytes(unsigned long long max_entries) { return sparse_layout(max_entries).total; }

cudaError_t launch_sparse(const int* rows, const int* cols, const void* vals, unsigned long long m, int n,
                          unsigned long long max_entries, unsigned long long* strings, void* weights,
                          unsigned long long capacity, unsigned long long* count, void* ws, unsigned* status,
                          cudaStream_t s) {
  const SparseLayout L = sparse_layout(max_entries);
  char* w = static_cast<char*>(ws);
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(w + L.ctr);   // see kSpCounters
  int* emax = reinterpret_cast<int*>(w + L.emax);
  uint32_t* keys = reinterpret_cast<uint32_t*>(w + L.keys);
  longlong2* v = reinterpret_cast<longlong2*>(w + L.vals);
  uint32_t* tkeys = reinterpret_cast<uint32_t*>(w + L.tkeys);
  unsigned long long* tv = reinterpret_cast<unsigned long long*>(w + L.tvals);
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(w + L.skey);
  uint32_t* sidx = reinterpret_cast<uint32_t*>(w + L.sidx);
  const unsigned long long cap = L.entries;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w, 0, L.keys, s)) != cudaSuccess) return e;        // counters, X-mask maxima
  if ((e = cudaMemsetAsync(tkeys, 0xFF, L.slots * 4, s)) != cudaSuccess) return e;   // the table starts empty;
  if ((e = cudaMemsetAsync(tv, 0, L.slots * 16, s)) != cudaSuccess) return e;        // each level leaves it so
  const unsigned long long m0 = m < cap ? m : cap;
  k_sp_start<<<1, 1, 0, s>>>(ctr, m, cap);
  if (m0 > 0) {
    k_sp_emax<<<grid_for(m0), 256, 0, s>>>(rows, cols, static_cast<const double2*>(vals), m0, n, emax);
    k_sp_init<<<(unsigned)((m0 + 255) / 256), 256, 0, s>>>(rows, cols, static_cast<const double2*>(vals), m0, n, emax,
                                                         keys, v);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const uint32_t mask = (uint32_t)(L.slots - 1);
  for (int beta = 0; beta < n; ++beta) {
    k_sp_level<<<grid_for(cap), 256, 0, s>>>(keys, v, ctr + 1 + beta, cap, n, beta, tkeys, tv, mask, ctr);
    k_sp_compact<<<grid_for(L.slots), 256, 0, s>>>(tkeys, tv, (uint32_t)L.slots, keys, v, ctr + 2 + beta, cap, ctr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const unsigned long long* fin = ctr + 1 + n;
  k_sp_keys<<<grid_for(L.sortn), 256, 0, s>>>(keys, fin, cap, n, skey, sidx);
  const unsigned chunks = (unsigned)((L.sortn + kSpChunk - 1) / kSpChunk);
  k_sp_local<<<chunks, kSpLocalThreads, 0, s>>>(skey, sidx, fin, cap, 2, kSpChunk);
  for (unsigned long long k = 2ull * kSpChunk; k <= L.sortn; k <<= 1) {
    for (unsigned long long j = k >> 1; j >= (unsigned long long)kSpChunk; j >>= 1)
      k_sp_bitonic<<<grid_for(L.sortn), 256, 0, s>>>(skey, sidx, fin, cap, j, k);
    k_sp_local<<<chunks, kSpLocalThreads, 0, s>>>(skey, sidx, fin, cap, k, k);
  }
  k_sp_emit<<<grid_for(cap), 256, 0, s>>>(keys, v, fin, cap, skey, sidx, n, emax, capacity, strings,
                                          static_cast<double2*>(weights), count);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (status) k_sp_status<<<1, 1, 0, s>>>(ctr, status);
  return cudaGetLastError();
}

}  // namespace tpd
