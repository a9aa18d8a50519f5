// Decomposition in the generalized Gell-Mann basis of n qudits of dimension
// d: the other tensorized basis Sec. V names as a natural candidate for the
// method.  For one qudit the d^2 Hermitian elements carry a label (r, c) of
// the d x d grid: the identity at (0, 0); the diagonal
// D_l = sqrt(2 / (l (l+1))) (sum_{m<l} E_mm - l E_ll) at (l, l), l >= 1;
// the symmetric S_jk = E_jk + E_kj at (j, k) and the antisymmetric
// A_jk = -i E_jk + i E_kj at (k, j), j < k.  Their squares have trace d
// (identity) or 2 (every other element), and they are orthogonal.  For
// n qudits an element is the tensor product over the digit pairs of its
// label, with N_(r,c) the product of those traces, and
//     A = sum g_(r,c) G_(r,c),     g_(r,c) = tr(G_(r,c) A) / N_(r,c).
// For d = 2 the elements are I, X, Y, Z at the positions where Eq. 4 puts
// their weights: the Pauli decomposition itself.
//
// The recursion of Eqs. 3-5 carries over: tr((G (x) G') A) contracts qudit 1
// with G and the rest with G', so the coefficients are d x d blocks of
// cumulative weights computed level by level, one qudit at a time, in any
// order.  One level maps each d x d block x (the qudit's row and column
// digits, all other digits fixed) in place to
//     (j, k), j < k:  (x_jk + x_kj) / 2           (symmetric)
//     (k, j), j < k:  i (x_jk - x_kj) / 2         (antisymmetric)
//     (l, l), l >= 1: c_l / 2 (sum_{m<l} x_mm - l x_ll),   c_l = sqrt(2 / (l (l+1)))
//     (0, 0):         (1 / d) sum_m x_mm
// (for d = 2 exactly Eq. 4), and the composition inverts it:
//     x_jk = y_jk - i y_kj,  x_kj = y_jk + i y_kj,
//     x_mm = y_00 + sum_{l>m} c_l y_ll - m c_m y_mm.
// On the GPU every level is applied to all blocks at once: one launch per
// qudit, each thread one block of d^2 elements held in registers, a
// grid-stride loop.  Arithmetic: IEEE fp64 (complex128) or fp32 (complex64),
// rounded every level, without contraction into fused multiply-adds, so real
// and imaginary parts see the same operations: conjugate blocks of a
// Hermitian input stay exact conjugates level by level, and its
// coefficients come out exactly real.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "tpd.h"

namespace tpd {
namespace {

constexpr int kGmMaxD = 5;

template <class T> struct GmVec;
template <> struct GmVec<double> { using t = double2; };
template <> struct GmVec<float> { using t = float2; };

// single roundings, never contracted into an fma
__device__ __forceinline__ double gadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double gsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double gmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float gadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float gsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float gmul(float a, float b) { return __fmul_rn(a, b); }

// x / 2 and 2 x.  For complex128 with integer instructions, bit for bit the
// fp64 product for every input (normal: the exponent field moves by one;
// zero and subnormal: the magnitude bits halved to nearest even, or doubled;
// 2 x beyond the largest double: Inf; Inf and NaN pass unchanged), so the
// fp64 pipe -- which bounds these kernels on GB300 -- only carries the adds,
// subtractions and the irrational diagonal factors.  complex64: the fp32
// multiply (not the bound there).
__device__ __forceinline__ double ghalf(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long sgn = b & (long long)0x8000000000000000ull, v = b & 0x7FFFFFFFFFFFFFFFll;
  const long long sub = sgn | ((v >> 1) + ((v & (v >> 1)) & 1));         // e <= 1: v / 2, ties to even
  return __longlong_as_double(e >= 2 && e < 0x7FF ? b - (1ll << 52) : (e < 2 ? sub : b));
}
__device__ __forceinline__ double gtwice(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long sgn = b & (long long)0x8000000000000000ull, v = b & 0x7FFFFFFFFFFFFFFFll;
  return __longlong_as_double(e == 0 ? (sgn | (v << 1))
                                     : e < 0x7FE ? b + (1ll << 52) : (e == 0x7FE ? (sgn | 0x7FF0000000000000ll) : b));
}
__device__ __forceinline__ float ghalf(float x) { return __fmul_rn(x, 0.5f); }
__device__ __forceinline__ float gtwice(float x) { return __fmul_rn(x, 2.0f); }

template <class T>
struct GmConst {
  T hc[kGmMaxD];   // c_l / 2: the decomposition's diagonal factors (l >= 1)
  T c[kGmMaxD];    // c_l: the composition's diagonal factors
  T lc[kGmMaxD];   // l c_l
  T l[kGmMaxD];    // l (as T)
  T inv_d;         // 1 / d (the identity's coefficient)
  T scale;         // factor on every output of this launch (the composition's last level)
  int scaled;      // scale != 1
};

// One qudit level on every d x d block: digit stride s (d^k), N = d^n,
// nblk = (N / D)^2 blocks (< 2^30 for N <= 65536).
template <class T, int D, bool kDec>
__global__ void __launch_bounds__(256) k_gellmann_level(typename GmVec<T>::t* __restrict__ mat, uint32_t N,
                                                        uint32_t s, uint32_t nblk, const GmConst<T> k) {
  using S = typename GmVec<T>::t;
  const uint32_t M = N / D;                      // combinations of the other digits per row / column
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nblk; q += gridDim.x * blockDim.x) {
    const uint32_t qr = q / M, qc = q - qr * M;
    const uint32_t R = (qr / s) * s * D + qr % s;      // row with this qudit's digit 0
    const uint32_t C = (qc / s) * s * D + qc % s;      // column likewise
    const long long base = (long long)R * N + C, rs = (long long)s * N;
    S x[D][D], y[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) x[r][c] = mat[base + r * rs + (long long)c * s];

    // off-diagonal pairs
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int i = j + 1; i < D; ++i) {
        const S a = x[j][i], b = x[i][j];
        if constexpr (kDec) {
          y[j][i] = {ghalf(gadd(a.x, b.x)), ghalf(gadd(a.y, b.y))};
          const T tr = ghalf(gsub(a.x, b.x)), ti = ghalf(gsub(a.y, b.y));
          y[i][j] = {-ti, tr};                                   // i (a - b) / 2
        } else {
          y[j][i] = {gadd(a.x, b.y), gsub(a.y, b.x)};            // a - i b
          y[i][j] = {gsub(a.x, b.y), gadd(a.y, b.x)};            // a + i b
        }
      }

    // diagonal
    if constexpr (kDec) {
      S P = x[0][0];                                             // running sum_{m<l} x_mm
#pragma unroll
      for (int l = 1; l < D; ++l) {
        const S xl = x[l][l];
        S lx = xl;                                               // l x_ll
        if (l == 2) lx = S{gtwice(xl.x), gtwice(xl.y)};
        if (l >= 3) lx = S{gmul(k.l[l], xl.x), gmul(k.l[l], xl.y)};
        if (l == 1)                                              // c_1 / 2 = 1/2 exactly
          y[l][l] = {ghalf(gsub(P.x, lx.x)), ghalf(gsub(P.y, lx.y))};
        else
          y[l][l] = {gmul(k.hc[l], gsub(P.x, lx.x)), gmul(k.hc[l], gsub(P.y, lx.y))};
        P = {gadd(P.x, xl.x), gadd(P.y, xl.y)};
      }
      if constexpr (D == 2) y[0][0] = {ghalf(P.x), ghalf(P.y)};
      else y[0][0] = {gmul(P.x, k.inv_d), gmul(P.y, k.inv_d)};
    } else {
      const S y0 = x[0][0];
      S Q = {T(0), T(0)};                                        // running sum_{l>m} c_l y_ll
#pragma unroll
      for (int m = D - 1; m >= 1; --m) {
        const S ym = x[m][m];
        // c_1 = 1 and 1 c_1 = 1 exactly: no multiply for m = 1
        const S cy = m == 1 ? ym : S{gmul(k.c[m], ym.x), gmul(k.c[m], ym.y)};
        const S lcy = m == 1 ? ym : S{gmul(k.lc[m], ym.x), gmul(k.lc[m], ym.y)};
        y[m][m] = {gadd(y0.x, gsub(Q.x, lcy.x)), gadd(y0.y, gsub(Q.y, lcy.y))};
        Q = {gadd(Q.x, cy.x), gadd(Q.y, cy.y)};
      }
      y[0][0] = {gadd(y0.x, Q.x), gadd(y0.y, Q.y)};
    }

    if (k.scaled) {
#pragma unroll
      for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) y[r][c] = {gmul(y[r][c].x, k.scale), gmul(y[r][c].y, k.scale)};
    }
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) mat[base + r * rs + (long long)c * s] = y[r][c];
  }
}

template <class T>
GmConst<T> gm_const(int d, double scale) {
  GmConst<T> k{};
  for (int l = 1; l < d; ++l) {
    const double c = std::sqrt(2.0 / ((double)l * (double)(l + 1)));
    k.c[l] = (T)c;
    k.hc[l] = (T)(0.5 * c);
    k.lc[l] = (T)((double)l * c);
    k.l[l] = (T)l;
  }
  k.inv_d = (T)(1.0 / d);
  k.scale = (T)scale;
  k.scaled = scale != 1.0;
  return k;
}

template <class T, bool kDec>
cudaError_t gm_levels(void* mat, int n, int d, double last_scale, cudaStream_t st) {
  uint32_t N = 1;
  for (int k = 0; k < n; ++k) N *= (uint32_t)d;
  const uint32_t nblk = (N / d) * (N / d);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  long long grid = ((long long)nblk + 255) / 256;
  if (grid > 16ll * nsm) grid = 16ll * nsm;
  if (grid < 1) grid = 1;
  auto* m = static_cast<typename GmVec<T>::t*>(mat);
  uint32_t s = 1;
  for (int k = 0; k < n; ++k, s *= (uint32_t)d) {
    const GmConst<T> kc = gm_const<T>(d, !kDec && k == n - 1 ? last_scale : 1.0);
    switch (d) {
      case 2: k_gellmann_level<T, 2, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, kc); break;
      case 3: k_gellmann_level<T, 3, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, kc); break;
      case 4: k_gellmann_level<T, 4, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, kc); break;
      default: k_gellmann_level<T, 5, kDec><<<(unsigned)grid, 256, 0, st>>>(m, N, s, nblk, kc); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

tpd_status gellmann_run(bool dec, void* A, int n, int d, int dtype, double scale, const tpd_options* opt,
                        void* stream) {
  if (A == nullptr || d < 2 || d > kGmMaxD || n < 1 || (dtype != TPD_C128 && dtype != TPD_C64))
    return TPD_ERR_INVALID_ARG;
  const int prec = opt ? opt->precision : TPD_PREC_DEFAULT;
  if (prec != TPD_PREC_DEFAULT && prec != TPD_PREC_PLAIN) return TPD_ERR_INVALID_ARG;
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
    e = dec ? gm_levels<double, true>(A, n, d, 1.0, st) : gm_levels<double, false>(A, n, d, scale, st);
  else
    e = dec ? gm_levels<float, true>(A, n, d, 1.0, st) : gm_levels<float, false>(A, n, d, scale, st);
  return e == cudaSuccess ? TPD_OK : TPD_ERR_CUDA;
}

}  // namespace
}  // namespace tpd

extern "C" {

tpd_status tpd_gellmann_decompose(void* A, int n, int d, int dtype, const tpd_options* opt, void* stream) {
  return tpd::gellmann_run(true, A, n, d, dtype, 1.0, opt, stream);
}

tpd_status tpd_gellmann_compose(void* C, int n, int d, int dtype, double scale, const tpd_options* opt,
                                void* stream) {
  return tpd::gellmann_run(false, C, n, d, dtype, scale, opt, stream);
}

}  // extern "C"
