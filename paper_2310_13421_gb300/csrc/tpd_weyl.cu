// Decomposition in the Weyl (clock-and-shift) basis of n qudits of dimension
// d: the tensorized basis Sec. V names as the natural next candidate for the
// method.  With omega = exp(2 pi i / d), X|j> = |j+1 mod d>, Z|j> = omega^j |j>
// and W_{a,b} = X^a Z^b (tensor products over the qudits), the weights of
// A in Mat(d^n) are c_{a,b} = d^-n tr(W_{a,b}^* A).
//
// The same recursion as Eqs. 3-5: partitioning A into d x d blocks A_{rc}
// (qudit 1's digits), A = sum_{a,b} W_{a,b} (x) Omega_{a,b} with the
// cumulative matrix weights
//     Omega_{a,b} = d^-1 sum_c omega^(-b c) A_{c+a, c}
// (the d x d analogue of Eq. 4: for each shift a, a length-d DFT along the
// block's a-th cyclic diagonal), and the levels commute.  On the GPU every
// level is applied to all d x d blocks at once, in place: one launch per
// qudit, each thread one block of d^2 elements in registers.  Omega_{a,b}
// goes to the block position (row digit b, column digit a + b mod d), which
// for d = 2 is where the Pauli decomposition puts I, X, Y, Z (with
// W_{1,1} = XZ = -iY).  The composition inverts each level:
// A_{c+a, c} = sum_b omega^(b c) Omega_{a,b}.
//
// Arithmetic.  complex64: IEEE fp32, rounded every level.  complex128: by
// default (d = 2, 3, 4) a block fixed point, as for the Pauli basis: the d
// elements one DFT combines (a cyclic diagonal of a block, a "class") go onto
// their own binary point in int64, set by the largest exponent among their
// components with headroom for the sums, the DFT runs in int64 -- exactly
// for d = 2 and 4 (twiddles +-1, +-i); for d = 3 with the outputs computed
// doubled, so that nothing is halved, and sqrt(3) multiplied once, rounded to
// the nearest point of the class's grid -- and each output is rounded to
// double once (RNE), the decomposition's 1/d folded in as an exponent (d = 2,
// 4) or as the nearest integer of a third on the class grid (d = 3).  The
// fp64 pipe of GB300 issues ~2 operations per clock per SM, far below what a
// level at HBM speed needs; integer instructions are not.  Classes meeting
// Inf or NaN, d = 5, and TPD_PREC_PLAIN run IEEE fp64 rounded every level
// (the paper's arithmetic carried over).  d = 3 uses the 3-point DFT written
// out (4 real additions-or-multiplications per element and level instead of
// 12): with s = x1 + x2, u = x1 - x2, m = x0 - s/2 and h = sqrt(3)/2,
//     y0 = x0 + s,   y1 = m - i h u,   y2 = m + i h u     (omega^-bc)
// and the conjugate signs for the composition.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <type_traits>

#include "tpd.h"
#include "tpd_arith.cuh"

namespace tpd {
namespace {

template <class T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <class T>
struct Cx {
  T re, im;
};

template <class T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
// a * (wr + i wi), written without contraction into fused multiply-adds
template <class T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, T wr, T wi) {
  if constexpr (sizeof(T) == 8)
    return {__dsub_rn(__dmul_rn(a.re, wr), __dmul_rn(a.im, wi)), __dadd_rn(__dmul_rn(a.re, wi), __dmul_rn(a.im, wr))};
  else
    return {__fsub_rn(__fmul_rn(a.re, wr), __fmul_rn(a.im, wi)), __fadd_rn(__fmul_rn(a.re, wi), __fmul_rn(a.im, wr))};
}

// Division of x < 2^32 by a divisor 0 < v < 2^32 fixed per launch: with
// m = ceil(2^64 / v), floor(x m / 2^64) = floor(x / v) (the excess x (m -
// 2^64 / v) / 2^64 < 2^-32 is below the gap 1 / v to the next integer).
struct Div32 {
  unsigned long long m;
  uint32_t v;
};
inline Div32 make_div32(uint32_t v) {
  Div32 d;
  d.v = v;
  d.m = v == 1 ? 0ull : (~0ull / v) + 1ull;    // ceil(2^64 / v) for every v > 1
  return d;
}
__device__ __forceinline__ uint32_t div32(uint32_t x, const Div32& d) {
  return d.v == 1 ? x : (uint32_t)__umul64hi((unsigned long long)x, d.m);
}

// The block of thread item q (q < nblk = (N/D)^2 < 2^30): its first element's
// index and the stride between its rows (digit k of row and column 0).
template <int D>
__device__ __forceinline__ void weyl_block(uint32_t q, long long N, uint32_t s, const Div32& dM, const Div32& ds,
                                           long long& base, long long& rs) {
  const uint32_t qr = div32(q, dM), qc = q - qr * dM.v;
  const uint32_t hr = div32(qr, ds), hc = div32(qc, ds);
  const long long R = (long long)hr * s * D + (qr - hr * s);   // digit k of the row set to 0
  const long long Cc = (long long)hc * s * D + (qc - hc * s);  // and of the column
  base = R * N + Cc;
  rs = (long long)s * N;
}

template <class T>
struct Twiddles {
  T re[8], im[8];     // omega^k, k < d
  T h;                // sqrt(3) / 2 (d = 3)
  T scale;            // factor applied to every output of this launch
};

// The d-point DFT of one class in the arithmetic T (y_b = sum_c omega^-bc x_c
// for the decomposition, omega^+bc for the composition).
template <class T, int D, bool kDec>
__device__ __forceinline__ void dft_ieee(const Cx<T> (&x)[D], Cx<T> (&y)[D], const Twiddles<T>& tw) {
  if constexpr (D == 3) {
    const Cx<T> sm = cadd(x[1], x[2]), u = csub(x[1], x[2]);
    const Cx<T> m = csub(x[0], Cx<T>{sm.re * T(0.5), sm.im * T(0.5)});
    const Cx<T> hu = {u.re * tw.h, u.im * tw.h};
    y[0] = cadd(x[0], sm);
    // -i h u = (h u.im, -h u.re); the composition takes +i h u for y1
    const Cx<T> mihu = {hu.im, -hu.re};
    y[1] = kDec ? cadd(m, mihu) : csub(m, mihu);
    y[2] = kDec ? csub(m, mihu) : cadd(m, mihu);
  } else {
#pragma unroll
    for (int b = 0; b < D; ++b) {
      Cx<T> acc = x[0];
#pragma unroll
      for (int c = 1; c < D; ++c) {
        const int k = kDec ? (D - (b * c) % D) % D : (b * c) % D;
        acc = cadd(acc, cmul(x[c], tw.re[k], tw.im[k]));
      }
      y[b] = acc;
    }
  }
}

// One qudit level on every d x d block: digit stride s (d^k for qudit n - k),
// N = d^n, nblk = (N / D)^2 blocks.
template <class T, int D, bool kDec>
__global__ void __launch_bounds__(256) k_weyl_level(typename C2<T>::t* __restrict__ mat, long long N, long long s,
                                                    long long nblk, const Twiddles<T> tw) {
  using S = typename C2<T>::t;
  const long long M = N / D;                 // other-digit combinations per row / column
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nblk;
       q += (long long)gridDim.x * blockDim.x) {
    const long long qr = q / M, qc = q - qr * M;
    const long long R = (qr / s) * s * D + qr % s;   // digit k of the row set to 0
    const long long Cc = (qc / s) * s * D + qc % s;  // and of the column
    const long long base = R * N + Cc, rs = s * N;
    Cx<T> in[D][D], out[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const S v = mat[base + r * rs + c * s];
        in[r][c] = {v.x, v.y};
      }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      // decomposition: x_c = A_{c+a, c} -> Omega_{a,b} at (b, a+b);
      // composition: Omega_{a,b} at (b, a+b) -> A_{c+a, c}
      Cx<T> x[D], y[D];
#pragma unroll
      for (int c = 0; c < D; ++c) x[c] = kDec ? in[(c + a) % D][c] : in[c][(a + c) % D];
      dft_ieee<T, D, kDec>(x, y, tw);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        if (kDec) out[b][(a + b) % D] = y[b];
        else out[(b + a) % D][b] = y[b];
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        S v;
        v.x = out[r][c].re * tw.scale;
        v.y = out[r][c].im * tw.scale;
        mat[base + r * rs + c * s] = v;
      }
  }
}

// round(sqrt(3) * 2^62) and (2^64 + 2) / 3
constexpr long long kSqrt3Q62 = 7987674492471257551ll;
constexpr long long kThirdQ64 = 0x5555555555555556ll;

// round(u * sqrt(3)) for |u| < 2^61 (the 128-bit product, rounded half up)
__device__ __forceinline__ long long mul_sqrt3(long long u) {
  const long long hi = __mul64hi(u, kSqrt3Q62);
  const unsigned long long lo = (unsigned long long)u * (unsigned long long)kSqrt3Q62;
  return (long long)(((unsigned long long)hi << 2) | (lo >> 62)) + (long long)((lo >> 61) & 1ull);
}

// the nearest integer to y / 3 for |y| < 2^62: q = floor(y / 3 + delta) with
// |delta| < 1/6 is floor(y / 3) or, for y divisible by 3 and negative, one
// less; the remainder y - 3 q in [0, 3] then says whether to round up
__device__ __forceinline__ long long div3_rn(long long y) {
  const long long q = __mul64hi(y, kThirdQ64);
  const long long r = y - 3 * q;
  return q + (r >= 2 ? 1 : 0);
}

__device__ __forceinline__ uint32_t exp_field(double2 v) {
  return max((uint32_t)__double2hiint(v.x) & 0x7fffffffu, (uint32_t)__double2hiint(v.y) & 0x7fffffffu) >> 20;
}

// One qudit level in the complex128 block fixed point (d = 2, 3, 4; see the
// top of this file).  out_pow2 / out_mul: the factor of this level's outputs
// (the composition's scale, on its last level) beyond the 1/d of the
// decomposition.
template <int D, bool kDec>
__global__ void __launch_bounds__(256) k_weyl_level_fx(double2* __restrict__ mat, long long N, uint32_t s,
                                                       uint32_t nblk, const Div32 dM, const Div32 ds,
                                                       const Twiddles<double> tw, int out_pow2, double out_mul) {
  static_assert(D >= 2 && D <= 4, "fixed point for d = 2, 3, 4");
  using I = long long;
  constexpr int G = D == 2 ? 1 : (D == 4 ? 2 : 3);   // headroom: |outputs (d = 3: doubled)| < 2^G max
  constexpr int kLogD = D == 2 ? 1 : (D == 4 ? 2 : 0);
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nblk; q += gridDim.x * blockDim.x) {
    long long base, rs;
    weyl_block<D>(q, N, s, dM, ds, base, rs);
    double2 in[D][D], out[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) in[r][c] = mat[base + r * rs + c * s];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double2 x[D];
      uint32_t E = 0;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        x[c] = kDec ? in[(c + a) % D][c] : in[c][(a + c) % D];
        E = max(E, exp_field(x[c]));
      }
      double2 y[D];
      if (E == 2047u) {
        // Inf or NaN in the class: IEEE fp64, as the plain path
        Cx<double> xc[D], yc[D];
#pragma unroll
        for (int c = 0; c < D; ++c) xc[c] = {x[c].x, x[c].y};
        dft_ieee<double, D, kDec>(xc, yc, tw);
#pragma unroll
        for (int b = 0; b < D; ++b) y[b] = make_double2(yc[b].re * tw.scale, yc[b].im * tw.scale);
      } else {
        // onto the class's binary point: x * 2^S, S = 1084 - G - max(E, 1)
        const int sb = 9 - G - max((int)E, 1);
        I xr[D], xi[D], yr[D], yi[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
          xr[c] = FixedArith::to_fixed(x[c].x, sb);
          xi[c] = FixedArith::to_fixed(x[c].y, sb);
        }
        int T = sb + 1075;                    // value = sum * 2^-T
        if constexpr (D == 2) {
          yr[0] = xr[0] + xr[1]; yi[0] = xi[0] + xi[1];
          yr[1] = xr[0] - xr[1]; yi[1] = xi[0] - xi[1];
        } else if constexpr (D == 4) {
          const I t0r = xr[0] + xr[2], t0i = xi[0] + xi[2], t1r = xr[0] - xr[2], t1i = xi[0] - xi[2];
          const I t2r = xr[1] + xr[3], t2i = xi[1] + xi[3], t3r = xr[1] - xr[3], t3i = xi[1] - xi[3];
          yr[0] = t0r + t2r; yi[0] = t0i + t2i;
          yr[2] = t0r - t2r; yi[2] = t0i - t2i;
          // decomposition: y1 = t1 - i t3, y3 = t1 + i t3; composition: conjugate twiddles
          const I pr = t1r + t3i, pi = t1i - t3r, mr = t1r - t3i, mi = t1i + t3r;
          yr[1] = kDec ? pr : mr; yi[1] = kDec ? pi : mi;
          yr[3] = kDec ? mr : pr; yi[3] = kDec ? mi : pi;
        } else {
          // doubled: 2 y0 = 2 (x0 + s), 2 m = 2 x0 - s, 2 h u = sqrt(3) u
          const I sr = xr[1] + xr[2], si = xi[1] + xi[2], ur = xr[1] - xr[2], ui = xi[1] - xi[2];
          yr[0] = (xr[0] + sr) * 2; yi[0] = (xi[0] + si) * 2;
          const I mr = 2 * xr[0] - sr, mi = 2 * xi[0] - si;
          const I hr = mul_sqrt3(ur), hi = mul_sqrt3(ui);
          // decomposition: 2 y1 = 2m - i (2hu), 2 y2 = 2m + i (2hu); composition: conjugate
          const I ar = mr + hi, ai = mi - hr, br = mr - hi, bi = mi + hr;
          yr[1] = kDec ? ar : br; yi[1] = kDec ? ai : bi;
          yr[2] = kDec ? br : ar; yi[2] = kDec ? bi : ai;
          T += 1;
          if constexpr (kDec) {               // the 1/3 of the level, on the class grid
#pragma unroll
            for (int b = 0; b < D; ++b) { yr[b] = div3_rn(yr[b]); yi[b] = div3_rn(yi[b]); }
          }
        }
        if constexpr (kDec) T += kLogD;       // the 1/d of the level (d = 2, 4)
        T -= out_pow2;
        // |sums| < 2^62: in the normal range after scaling (the usual case),
        // real parts through the fp64 conversion unit and imaginary parts
        // through integer instructions (identical roundings); else both the
        // general way
        if (FixedArith::fast_range(T)) {
#pragma unroll
          for (int b = 0; b < D; ++b)
            y[b] = make_double2(FixedArith::to_double_cvt_fast(yr[b], T), FixedArith::to_double_fast(yi[b], T));
        } else {
#pragma unroll
          for (int b = 0; b < D; ++b)
            y[b] = make_double2(FixedArith::to_double_int(yr[b], T), FixedArith::to_double_int(yi[b], T));
        }
        if (out_mul != 1.0) {
#pragma unroll
          for (int b = 0; b < D; ++b) { y[b].x *= out_mul; y[b].y *= out_mul; }
        }
      }
#pragma unroll
      for (int b = 0; b < D; ++b) {
        if (kDec) out[b][(a + b) % D] = y[b];
        else out[(b + a) % D][b] = y[b];
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) mat[base + r * rs + c * s] = out[r][c];
  }
}

// A cosine or sine within a few ulps of 0, +-1/2 or +-1 is that value
// exactly, so quarter and sixth turns carry no rounding.
double exact_if_near_half_integer(double v) {
  const double h = std::nearbyint(2.0 * v) * 0.5;
  return std::fabs(v - h) <= 4e-16 ? h : v;
}

template <class T>
Twiddles<T> twiddles(int d, double scale) {
  Twiddles<T> t{};
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < d; ++k) {
    t.re[k] = (T)exact_if_near_half_integer(std::cos(2.0 * pi * k / d));
    t.im[k] = (T)exact_if_near_half_integer(std::sin(2.0 * pi * k / d));
  }
  t.h = (T)(std::sqrt(3.0) * 0.5);
  t.scale = (T)scale;
  return t;
}

// exponent of an exact power of two, else 0 with *resid = v
int split_pow2(double v, double* resid) {
  int e = 0;
  const double m = std::frexp(v, &e);
  if (m == 0.5 || m == -0.5) {
    *resid = m < 0 ? -1.0 : 1.0;
    return e - 1;
  }
  *resid = v;
  return 0;
}

template <class T, bool kDec>
cudaError_t launch_levels(void* mat, int n, int d, double last_scale, bool fixed, cudaStream_t st) {
  long long N = 1;
  for (int k = 0; k < n; ++k) N *= d;
  const long long nblk = (N / d) * (N / d);   // < 2^30: N <= 65536
  const Div32 dM = make_div32((uint32_t)(N / d));
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  long long grid = (nblk + 255) / 256;
  if (grid > 16ll * nsm) grid = 16ll * nsm;
  if (grid < 1) grid = 1;
  using S = typename C2<T>::t;
  long long s = 1;
  for (int k = 0; k < n; ++k, s *= d) {
    const Div32 ds = make_div32((uint32_t)s);
    // the decomposition's 1/d per level; the composition's scale on its last level
    const double sc = kDec ? 1.0 / d : (k == n - 1 ? last_scale : 1.0);
    const Twiddles<T> tw = twiddles<T>(d, sc);
    S* m = static_cast<S*>(mat);
    if constexpr (std::is_same<T, double>::value) {
      if (fixed && d <= 4) {
        double resid = 1.0;
        const int p2 = kDec ? 0 : split_pow2(sc, &resid);
        double2* md = m;
        const Twiddles<double>& twd = tw;
        switch (d) {
          case 2:
            k_weyl_level_fx<2, kDec><<<(unsigned)grid, 256, 0, st>>>(md, N, (uint32_t)s, (uint32_t)nblk, dM, ds, twd,
                                                                     p2, resid);
            break;
          case 3:
            k_weyl_level_fx<3, kDec><<<(unsigned)grid, 256, 0, st>>>(md, N, (uint32_t)s, (uint32_t)nblk, dM, ds, twd,
                                                                     p2, resid);
            break;
          default:
            k_weyl_level_fx<4, kDec><<<(unsigned)grid, 256, 0, st>>>(md, N, (uint32_t)s, (uint32_t)nblk, dM, ds, twd,
                                                                     p2, resid);
            break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        continue;
      }
    }
    switch (d) {
      case 2: k_weyl_level<T, 2, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, tw); break;
      case 3: k_weyl_level<T, 3, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, tw); break;
      case 4: k_weyl_level<T, 4, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, tw); break;
      default: k_weyl_level<T, 5, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, tw); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

tpd_status weyl_run(bool dec, void* A, int n, int d, int dtype, double scale, const tpd_options* opt, void* stream) {
  if (A == nullptr || d < 2 || d > 5 || n < 1 || (dtype != TPD_C128 && dtype != TPD_C64)) return TPD_ERR_INVALID_ARG;
  // arithmetic: complex128 block fixed point (d <= 4) unless PLAIN is asked
  // for; complex64 fp32; FIXED for d = 5 or complex64 and COMPENSATED are
  // not offered
  const int prec = opt ? opt->precision : TPD_PREC_DEFAULT;
  if (prec != TPD_PREC_DEFAULT && prec != TPD_PREC_PLAIN && prec != TPD_PREC_FIXED) return TPD_ERR_INVALID_ARG;
  if (prec == TPD_PREC_FIXED && (dtype != TPD_C128 || d > 4)) return TPD_ERR_INVALID_ARG;
  const bool fixed = dtype == TPD_C128 && d <= 4 && prec != TPD_PREC_PLAIN;
  long long N = 1;
  for (int k = 0; k < n; ++k) {
    N *= d;
    if (N > 65536) return TPD_ERR_INVALID_ARG;
  }
  if (!dec && (!std::isfinite(scale) || scale == 0.0)) return TPD_ERR_INVALID_ARG;
  const size_t align = dtype == TPD_C128 ? 16 : 8;
  if (reinterpret_cast<uintptr_t>(A) % align) return TPD_ERR_MISALIGNED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dtype == TPD_C128)
    e = dec ? launch_levels<double, true>(A, n, d, 1.0, fixed, st)
            : launch_levels<double, false>(A, n, d, scale, fixed, st);
  else
    e = dec ? launch_levels<float, true>(A, n, d, 1.0, false, st)
            : launch_levels<float, false>(A, n, d, scale, false, st);
  return e == cudaSuccess ? TPD_OK : TPD_ERR_CUDA;
}

}  // namespace
}  // namespace tpd

extern "C" {

tpd_status tpd_weyl_decompose(void* A, int n, int d, int dtype, const tpd_options* opt, void* stream) {
  return tpd::weyl_run(true, A, n, d, dtype, 1.0, opt, stream);
}

tpd_status tpd_weyl_compose(void* C, int n, int d, int dtype, double scale, const tpd_options* opt,
                            void* stream) {
  return tpd::weyl_run(false, C, n, d, dtype, scale, opt, stream);
}

}  // extern "C"
