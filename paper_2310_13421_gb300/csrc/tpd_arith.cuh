// Element arithmetic for the Pauli butterfly (Eq. 4) and its inverse.
//
// Per qubit level the decomposition maps the quad (a00, a01, a10, a11) of a
// 2x2 block (row bit, column bit) to
//     I = a00 + a11,  X = a01 + a10,  Y = i (a01 - a10),  Z = a00 - a11
// and leaves them at the same four positions; the factor 1/2 of Eq. 4 is
// applied once per pass as 2^-K, which is exact.  The composition maps
//     a00 = I + Z,  a01 = X - iY,  a10 = X + iY,  a11 = I - Z.
//
// Five arithmetics share this interface:
//   FixedArith  complex128 storage; a pass loads each tile onto a common
//               binary point in int64 (block fixed point), sums exactly, and
//               rounds once to double (RNE) when it stores.  Only integer
//               instructions: on GB300 the fp64 pipe issues ~2 ops/clk/SM,
//               far below the HBM rate of this kernel.
//   F64Arith    complex128, IEEE double adds (rounded every level).
//   F32Arith    complex64, IEEE float adds.
//   F32CArith   complex64, float sums with TwoSum error terms carried through
//               the pass (cascaded summation, Ogita-Rump-Oishi 2005), one
//               rounding fl(hi + lo) per pass.
//   Fixed32Arith complex64 storage, every pass on its own tile binary point in
//               int64 (exact sums), rounded to float (RNE) when it stores:
//               one rounding per pass, integer instructions only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tpd {

// ---------------------------------------------------------------- per-tile output scaling
struct OutScale {
  int pow2;        // multiply by 2^pow2 (exact)
  double extra;    // remaining non-power-of-two factor (1.0 normally)
};

__device__ __forceinline__ uint32_t shfl_x(uint32_t v, int mask) {
  return __shfl_xor_sync(0xffffffffu, v, mask);
}

// ================================================================ fixed point
struct FixedArith {
  using Store = double2;
  struct __align__(16) V { long long re, im; };   // 16-byte aligned: one 128-bit shared access
  static constexpr bool kFixed = true;
  static constexpr bool kFixed32 = false;
  static constexpr int kStoreBytes = 16;

  __device__ static __forceinline__ V add(V a, V b) { return {a.re + b.re, a.im + b.im}; }
  __device__ static __forceinline__ V sub(V a, V b) { return {a.re - b.re, a.im - b.im}; }
  __device__ static __forceinline__ V mul_i(V d) { return {-d.im, d.re}; }       //  i d
  __device__ static __forceinline__ V mul_mi(V d) { return {d.im, -d.re}; }      // -i d
  __device__ static __forceinline__ V neg(V d) { return {-d.re, -d.im}; }
  __device__ static __forceinline__ V shfl(V v, int mask) {
    V o;
    o.re = (long long)(((unsigned long long)shfl_x((uint32_t)(v.re >> 32), mask) << 32) |
                       shfl_x((uint32_t)v.re, mask));
    o.im = (long long)(((unsigned long long)shfl_x((uint32_t)(v.im >> 32), mask) << 32) |
                       shfl_x((uint32_t)v.im, mask));
    return o;
  }

  // x * 2^S truncated toward zero, S = 1084 - K - Emax_eff (see from_double).
  // shift_base = 9 - K - Emax_eff, so that the element with the tile's
  // largest exponent lands below 2^(62-K) and 2^K of them sum below 2^62.
  __device__ static __forceinline__ long long to_fixed(double x, int shift_base) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int e = (int)(bits >> 52) & 0x7FF;
    const unsigned long long m =
        (bits & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
    const int sh = max(e, 1) + shift_base;   // <= 9 - K <= 8
    const unsigned rs = (unsigned)(11 - sh); // >= 3
    unsigned long long mag;
    const unsigned long long ml = m << 11;   // m < 2^53
    // PTX clamps shift amounts above 64 to 64 (result 0): no undefined shifts.
    asm("shr.b64 %0, %1, %2;" : "=l"(mag) : "l"(ml), "r"(rs));
    const unsigned long long s = (unsigned long long)((long long)bits >> 63);
    return (long long)((mag ^ s) - s);
  }

  // The same value through the fp64 conversion unit: scale by 2^S with an
  // exact exponent shift, then convert truncating toward zero.  Subnormal x
  // or a scaled exponent outside the normal range takes the integer path.
  // Used for one of the two components so that the integer pipe and the
  // otherwise idle fp64 pipe share the work.
  __device__ static __forceinline__ long long to_fixed_cvt(double x, int shift_base) {
    const long long bits = __double_as_longlong(x);
    const int e = (int)(bits >> 52) & 0x7FF;
    const int S = shift_base + 1075;          // = 1084 - K - Emax_eff
    if (e >= 1 && e + S >= 1 && e + S <= 2046)
      return __double2ll_rz(__longlong_as_double(bits + ((long long)S << 52)));
    return to_fixed(x, shift_base);
  }

  // to_fixed through the fp64 conversion unit, for elements of a class whose
  // largest exponent field is E (shift_base = 9 - K - max(E, 1), so e + S
  // <= 1084 - K stays in the normal range for every element of the class):
  // scale by 2^S with an exact exponent shift, then convert truncating
  // toward zero.  A scaled exponent below the normal range means
  // |x| 2^S < 1: the result is 0.  Zeros are 0; subnormal x (rare) take the
  // integer path out of line.
  __device__ static __forceinline__ long long to_fixed_cvt_class(double x, int shift_base) {
    const long long bits = __double_as_longlong(x);
    const int e = (int)(bits >> 52) & 0x7FF;
    const int S = shift_base + 1075;          // = 1084 - K - max(E, 1)
    if (e == 0) return ((unsigned long long)bits << 1) == 0 ? 0ll : to_fixed_rare(x, shift_base);
    return e + S >= 1 ? __double2ll_rz(__longlong_as_double(bits + ((long long)S << 52))) : 0ll;
  }
  static __device__ __noinline__ long long to_fixed_rare(double x, int shift_base) { return to_fixed(x, shift_base); }

  // Magnitude bits of a * 2^(be - 1086) (a has its leading one at bit 63)
  // rounded to nearest even, when that falls outside the normal range:
  // overflow to Inf or a subnormal result.  Out of line: never taken for
  // data in the normal range.
  __device__ static __noinline__ unsigned long long rare_bits(unsigned long long a, int be) {
    if (be > 2046) return 0x7FF0000000000000ull;
    const int rsh = 12 - be;                    // >= 12: subnormal, mantissa = a >> rsh
    if (rsh > 64) return 0;
    if (rsh == 64) return (a > 0x8000000000000000ull) ? 1ull : 0ull;
    unsigned long long mant = a >> rsh;
    const unsigned long long rem = a & ((1ull << rsh) - 1);
    const unsigned long long half = 1ull << (rsh - 1);
    mant += (unsigned long long)((rem > half) | ((rem == half) & (mant & 1ull)));
    return mant;                                // reaching 2^52 gives the smallest normal
  }

  // v * 2^-T rounded to nearest even (integer instructions only).
  __device__ static __forceinline__ double to_double_int(long long v, int T) {
    if (v == 0) return 0.0;
    const unsigned long long s = (unsigned long long)(v >> 63);
    unsigned long long a = ((unsigned long long)v ^ s) - s;
    const int lz = __clzll((long long)a);
    a <<= lz;                                   // leading one at bit 63
    const int be = 1086 - lz - T;               // biased exponent of that bit
    unsigned long long bits;
    if (be >= 1 && be <= 2046) {
      unsigned long long mant = a >> 11;        // 53 bits
      const unsigned rem = (unsigned)a & 0x7FFu;
      mant += (unsigned long long)((rem > 0x400u) | ((rem == 0x400u) & (unsigned)mant));
      bits = ((unsigned long long)(be - 1) << 52) + mant;   // a carry out of mant bumps the exponent
      if ((bits >> 52) >= 2047) bits = 0x7FF0000000000000ull;
    } else {
      bits = rare_bits(a, be);
    }
    return __longlong_as_double((long long)(bits | (s & 0x8000000000000000ull)));
  }

  // True when every nonzero |v| < 2^62 scaled by 2^-T lands in the normal
  // range (also after rounding up): then to_double_fast applies to the tile.
  __device__ static __forceinline__ bool fast_range(int T) { return T <= 1022 && T >= -961; }

  // v * 2^-T rounded to nearest even for |v| < 2^62 in the normal range
  // (fast_range(T)), in 32-bit integer instructions: normalise with a
  // funnel shift, round with a carry trick, assemble the exponent.
  __device__ static __forceinline__ double to_double_fast(long long v, int T) {
    const unsigned long long s64 = (unsigned long long)(v >> 63);
    const unsigned long long a = ((unsigned long long)v ^ s64) - s64;
    const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
    const bool big = ah != 0u;
    const uint32_t h = big ? ah : al;               // the word holding the leading one
    const uint32_t l = big ? al : 0u;
    const int lz = __clz((int)h);                   // 0..31 for a != 0
    const uint32_t mh = __funnelshift_l(l, h, lz);  // (h:l) << lz, leading one at bit 31
    const uint32_t ml = l << (lz & 31);
    uint32_t mant_hi = mh >> 11;                    // 21 bits, implicit one at bit 20
    uint32_t mant_lo = __funnelshift_r(ml, mh, 11); // next 32 bits
    const uint32_t rem = ml & 0x7FFu;
    const uint32_t up = (rem + 0x3FFu + (mant_lo & 1u)) >> 11;   // RNE: 1 iff rem > half or tie with odd lsb
    const unsigned long long mant = (((unsigned long long)mant_hi << 32) | mant_lo) + up;
    const int be = 1086 - (lz + (big ? 0 : 32)) - T;
    const uint32_t hi = ((uint32_t)(be - 1) << 20) + (uint32_t)(mant >> 32);   // a carry bumps the exponent
    const unsigned long long bits =
        ((unsigned long long)(hi | ((uint32_t)s64 & 0x80000000u)) << 32) | (uint32_t)mant;
    return a == 0 ? 0.0 : __longlong_as_double((long long)bits);
  }

  // to_double_fast through the fp64 conversion unit: round to nearest even,
  // then an exact exponent shift (fast_range(T): every nonzero |v| < 2^62
  // lands in the normal range).
  __device__ static __forceinline__ double to_double_cvt_fast(long long v, int T) {
    const long long b = __double_as_longlong(__ll2double_rn(v)) - ((long long)T << 52);
    return __longlong_as_double(v == 0 ? 0ll : b);
  }

  // v * 2^-T: the int64 -> double conversion (round to nearest even) followed
  // by an exact exponent shift; out-of-range exponents take the integer path.
  __device__ static __forceinline__ double to_double_cvt(long long v, int T) {
    const double d = __ll2double_rn(v);
    const long long b = __double_as_longlong(d);
    const int e = (int)(b >> 52) & 0x7FF;       // >= 1023 for v != 0
    if (v != 0 && e - T >= 1 && e - T <= 2046) return __longlong_as_double(b - ((long long)T << 52));
    return to_double_int(v, T);
  }

  // Both components rounded with integer instructions (any T): the rare
  // case of the block fixed point's stores, out of line.
  static __device__ __noinline__ double2 to_double2_rare(long long re, long long im, int T, double mul) {
    double2 o = make_double2(to_double_int(re, T), to_double_int(im, T));
    if (mul != 1.0) { o.x *= mul; o.y *= mul; }
    return o;
  }

  __device__ static __forceinline__ double to_double(long long v, int T) {
#ifdef TPD_TO_DOUBLE_CVT
    return to_double_cvt(v, T);
#else
    return to_double_int(v, T);
#endif
  }
};

// ================================================================ IEEE double
struct F64Arith {
  using Store = double2;
  using V = double2;
  static constexpr bool kFixed = false;
  static constexpr bool kFixed32 = false;
  static constexpr int kStoreBytes = 16;
  __device__ static __forceinline__ V add(V a, V b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
  __device__ static __forceinline__ V sub(V a, V b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
  __device__ static __forceinline__ V mul_i(V d) { return make_double2(-d.y, d.x); }
  __device__ static __forceinline__ V mul_mi(V d) { return make_double2(d.y, -d.x); }
  __device__ static __forceinline__ V neg(V d) { return make_double2(-d.x, -d.y); }
  __device__ static __forceinline__ V shfl(V v, int mask) {
    V o;
    o.x = __hiloint2double((int)shfl_x((uint32_t)__double2hiint(v.x), mask),
                           (int)shfl_x((uint32_t)__double2loint(v.x), mask));
    o.y = __hiloint2double((int)shfl_x((uint32_t)__double2hiint(v.y), mask),
                           (int)shfl_x((uint32_t)__double2loint(v.y), mask));
    return o;
  }
  __device__ static __forceinline__ V load(Store s) { return s; }

  // x * 2^-sh, 1 <= sh <= 11, with integer instructions and bit for bit the
  // fp64 product: a normal result moves the exponent field; a subnormal or
  // zero result is the magnitude in units of 2^-1074 shifted right with
  // round to nearest even; Inf and NaN pass unchanged.  Keeps the pass's
  // 2^-K off the fp64 pipe, which bounds this arithmetic on GB300.
  __device__ static __forceinline__ double mul_pow2_neg(double x, int sh) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long sgn = (unsigned long long)b & 0x8000000000000000ull;
    const unsigned long long m = (unsigned long long)b & 0x000FFFFFFFFFFFFFull;
    const unsigned long long v = e == 0 ? m : (m | (1ull << 52)) << min(max(e - 1, 0), 10);
    unsigned long long q = v >> sh;
    const unsigned long long rem = v & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q += (unsigned long long)((rem > half) | ((rem == half) & (q & 1ull)));
    const long long sub = (long long)(sgn | q);
    return __longlong_as_double(e > sh && e < 0x7FF ? b - ((long long)sh << 52) : (e == 0x7FF ? b : sub));
  }
  __device__ static __forceinline__ Store store(V v, const OutScale& sc, double mul) {
    if (mul == 1.0) return v;
    const long long mb = __double_as_longlong(mul);
    const int sh = 1023 - (int)((mb >> 52) & 0x7FF);
    if (mb > 0 && (mb & 0x000FFFFFFFFFFFFFll) == 0 && sh >= 1 && sh <= 11)   // mul = 2^-sh
      return make_double2(mul_pow2_neg(v.x, sh), mul_pow2_neg(v.y, sh));
    return make_double2(__dmul_rn(v.x, mul), __dmul_rn(v.y, mul));
  }
  __device__ static __forceinline__ bool nonzero(Store o) {   // +-0 is zero, NaN is not
    return (((uint32_t)__double2hiint(o.x) << 1) | (uint32_t)__double2loint(o.x) |
            ((uint32_t)__double2hiint(o.y) << 1) | (uint32_t)__double2loint(o.y)) != 0;
  }
};

// ================================================================ IEEE float
struct F32Arith {
  using Store = float2;
  using V = float2;
  static constexpr bool kFixed = false;
  static constexpr bool kFixed32 = false;
  static constexpr int kStoreBytes = 8;
  __device__ static __forceinline__ V add(V a, V b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
  __device__ static __forceinline__ V sub(V a, V b) { return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
  __device__ static __forceinline__ V mul_i(V d) { return make_float2(-d.y, d.x); }
  __device__ static __forceinline__ V mul_mi(V d) { return make_float2(d.y, -d.x); }
  __device__ static __forceinline__ V neg(V d) { return make_float2(-d.x, -d.y); }
  __device__ static __forceinline__ V shfl(V v, int mask) {
    return make_float2(__uint_as_float(shfl_x(__float_as_uint(v.x), mask)),
                       __uint_as_float(shfl_x(__float_as_uint(v.y), mask)));
  }
  __device__ static __forceinline__ V load(Store s) { return s; }
  __device__ static __forceinline__ Store store(V v, const OutScale& sc, double mul) {
    const float m = (float)mul;
    if (m == 1.0f) return v;
    return make_float2(__fmul_rn(v.x, m), __fmul_rn(v.y, m));
  }
  __device__ static __forceinline__ bool nonzero(Store o) {
    return ((__float_as_uint(o.x) | __float_as_uint(o.y)) << 1) != 0;
  }
};

// ================================================================ compensated float
struct F32CArith {
  using Store = float2;
  struct __align__(16) V { float re, im, rl, il; };   // value = (re + rl) + i (im + il)
  static constexpr bool kFixed = false;
  static constexpr bool kFixed32 = false;
  static constexpr int kStoreBytes = 8;

  // Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b).
  __device__ static __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
  }
#ifdef TPD_F32C_SCALAR
  __device__ static __forceinline__ V add(V a, V b) {
    V o; float e;
    two_sum(a.re, b.re, o.re, e); o.rl = __fadd_rn(__fadd_rn(a.rl, b.rl), e);
    two_sum(a.im, b.im, o.im, e); o.il = __fadd_rn(__fadd_rn(a.il, b.il), e);
    return o;
  }
  __device__ static __forceinline__ V sub(V a, V b) {
    V o; float e;
    two_sum(a.re, -b.re, o.re, e); o.rl = __fadd_rn(__fsub_rn(a.rl, b.rl), e);
    two_sum(a.im, -b.im, o.im, e); o.il = __fadd_rn(__fsub_rn(a.il, b.il), e);
    return o;
  }
#else
  // The same TwoSum on the (re, im) pair at once with packed fp32x2
  // instructions (sm_100 family): half the instructions of the scalar form,
  // identical roundings -- y - x is fma(x, -1, y), rounded once.
  __device__ static __forceinline__ float2 sub2(float2 y, float2 x) {
    return __ffma2_rn(x, make_float2(-1.0f, -1.0f), y);
  }
  __device__ static __forceinline__ V add2(float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 s = __fadd2_rn(ah, bh);
    const float2 bb = sub2(s, ah);
    const float2 aa = sub2(s, bb);
    const float2 e = __fadd2_rn(sub2(ah, aa), sub2(bh, bb));
    const float2 l = __fadd2_rn(__fadd2_rn(al, bl), e);
    return {s.x, s.y, l.x, l.y};
  }
  // TwoSum of a + (-b) without negating b: s = a - b; the error of adding -b,
  // (a - aa) + (-b - bb), is (a - aa) - (b + bb) (rounding to nearest is
  // symmetric), so every rounding is the scalar form's.
  __device__ static __forceinline__ V sub2(float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 s = sub2(ah, bh);
    const float2 bb = sub2(s, ah);
    const float2 aa = sub2(s, bb);
    const float2 e = sub2(sub2(ah, aa), __fadd2_rn(bh, bb));
    const float2 l = __fadd2_rn(sub2(al, bl), e);
    return {s.x, s.y, l.x, l.y};
  }
  __device__ static __forceinline__ V add(V a, V b) {
    return add2(make_float2(a.re, a.im), make_float2(a.rl, a.il), make_float2(b.re, b.im),
                make_float2(b.rl, b.il));
  }
  __device__ static __forceinline__ V sub(V a, V b) {
    return sub2(make_float2(a.re, a.im), make_float2(a.rl, a.il), make_float2(b.re, b.im),
                make_float2(b.rl, b.il));
  }
  // i (a - b) = (b.im - a.im) + i (a.re - b.re), as one packed subtraction
  // (the TwoSum error of the swapped operands is the exact negative, so the
  // bits are those of mul_i(sub(a, b)), up to the sign of an exact zero)
  __device__ static __forceinline__ V isub(V a, V b) {
    return sub2(make_float2(b.im, a.re), make_float2(b.il, a.rl), make_float2(a.im, b.re),
                make_float2(a.il, b.rl));
  }
#endif
  __device__ static __forceinline__ V mul_i(V d) { return {-d.im, d.re, -d.il, d.rl}; }
  __device__ static __forceinline__ V mul_mi(V d) { return {d.im, -d.re, d.il, -d.rl}; }
  __device__ static __forceinline__ V neg(V d) { return {-d.re, -d.im, -d.rl, -d.il}; }
  __device__ static __forceinline__ V shfl(V v, int mask) {
    return {__uint_as_float(shfl_x(__float_as_uint(v.re), mask)),
            __uint_as_float(shfl_x(__float_as_uint(v.im), mask)),
            __uint_as_float(shfl_x(__float_as_uint(v.rl), mask)),
            __uint_as_float(shfl_x(__float_as_uint(v.il), mask))};
  }
  __device__ static __forceinline__ V load(Store s) { return {s.x, s.y, 0.0f, 0.0f}; }
  __device__ static __forceinline__ Store store(V v, const OutScale& sc, double mul) {
    float re = __fadd_rn(v.re, v.rl), im = __fadd_rn(v.im, v.il);
    const float m = (float)mul;
    if (m != 1.0f) { re = __fmul_rn(re, m); im = __fmul_rn(im, m); }
    return make_float2(re, im);
  }
  __device__ static __forceinline__ bool nonzero(Store o) {
    return ((__float_as_uint(o.x) | __float_as_uint(o.y)) << 1) != 0;
  }
};

// ================================================================ fixed point, float storage
//
// A tile of floats (binary exponent field E <= 254 of its largest component)
// goes onto the binary point S = 188 - K - max(E, 1): x * 2^S is exact for
// every component within 2^(38-K) of the largest (smaller ones are truncated
// toward zero, an error below 2^-(62-K) of the largest), the largest lands
// below 2^(62-K), and the 2^K-term sums of the pass stay below 2^62.
struct Fixed32Arith {
  using Store = float2;
  using V = FixedArith::V;
  static constexpr bool kFixed = false;
  static constexpr bool kFixed32 = true;
  static constexpr int kStoreBytes = 8;
  __device__ static __forceinline__ V add(V a, V b) { return FixedArith::add(a, b); }
  __device__ static __forceinline__ V sub(V a, V b) { return FixedArith::sub(a, b); }
  __device__ static __forceinline__ V mul_i(V d) { return FixedArith::mul_i(d); }
  __device__ static __forceinline__ V mul_mi(V d) { return FixedArith::mul_mi(d); }
  __device__ static __forceinline__ V neg(V d) { return FixedArith::neg(d); }
  __device__ static __forceinline__ V shfl(V v, int mask) { return FixedArith::shfl(v, mask); }

  // x * 2^S truncated toward zero; rs_base = max(E_tile, 1) + K.
  __device__ static __forceinline__ long long to_fixed(float x, int rs_base) {
    const uint32_t bits = __float_as_uint(x);
    const int e = (int)(bits >> 23) & 0xFF;
    const uint32_t m = (bits & 0x007FFFFFu) | ((uint32_t)(e != 0) << 23);
    const unsigned rs = (unsigned)(rs_base - max(e, 1));   // >= K >= 1
    unsigned long long mag;
    const unsigned long long ml = (unsigned long long)m << 38;   // m < 2^24
    asm("shr.b64 %0, %1, %2;" : "=l"(mag) : "l"(ml), "r"(rs));   // clamps above 64: 0
    const unsigned long long sg = (unsigned long long)(long long)((int)bits >> 31);
    return (long long)((mag ^ sg) - sg);
  }

  // True when every nonzero |v| < 2^62 scaled by 2^-T is a normal float
  // (also after rounding up): then to_float_cvt_fast applies to the tile.
  __device__ static __forceinline__ bool fast_range(int T) { return T <= 126 && T >= -65; }

  // to_float for fast_range(T) through the conversion unit: round to nearest
  // even, then an exact exponent shift.
  __device__ static __forceinline__ float to_float_cvt_fast(long long v, int T) {
    const uint32_t b = __float_as_uint(__ll2float_rn(v)) - ((uint32_t)T << 23);
    return __uint_as_float(v == 0 ? 0u : b);
  }

  // v * 2^-T rounded to the nearest float, ties to even (integer instructions;
  // subnormal results and overflow to Inf included).
  __device__ static __forceinline__ float to_float(long long v, int T) {
    if (v == 0) return 0.0f;
    const unsigned long long s = (unsigned long long)(v >> 63);
    unsigned long long a = ((unsigned long long)v ^ s) - s;
    const int lz = __clzll((long long)a);
    a <<= lz;                                   // leading one at bit 63
    const int be = 190 - lz - T;                // biased exponent of that bit
    uint32_t bits;
    if (be >= 1) {
      const uint32_t hi = (uint32_t)(a >> 32);
      const uint32_t mant = hi >> 8;            // 24 bits, implicit one at bit 23
      const uint32_t r8 = hi & 0xFFu;           // the next 8 bits ...
      const bool sticky = (uint32_t)a != 0u;    // ... and the rest
      const uint32_t up = (r8 > 0x80u) | ((r8 == 0x80u) & (sticky | (mant & 1u)));
      bits = be > 254 ? 0x7F800000u : ((uint32_t)(be - 1) << 23) + mant + up;   // a carry bumps the exponent
      if (bits > 0x7F800000u) bits = 0x7F800000u;
    } else {
      const int rsh = 41 - be;                  // >= 41: subnormal mantissa = a >> rsh
      if (rsh > 64) {
        bits = 0u;
      } else if (rsh == 64) {
        bits = a > 0x8000000000000000ull ? 1u : 0u;
      } else {
        const unsigned long long mant = a >> rsh;
        const unsigned long long rem = a & ((1ull << rsh) - 1);
        const unsigned long long half = 1ull << (rsh - 1);
        bits = (uint32_t)(mant + ((rem > half) | ((rem == half) & (mant & 1ull))));
      }
    }
    return __uint_as_float(bits | ((uint32_t)s & 0x80000000u));
  }
};

}  // namespace tpd
