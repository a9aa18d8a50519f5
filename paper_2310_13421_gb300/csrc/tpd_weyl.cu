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
// Arithmetic: complex128 in IEEE fp64, complex64 in fp32, rounded every level
// (the paper's arithmetic carried over).  d = 3 uses the 3-point DFT written
// out (4 real additions-or-multiplications per element and level instead of
// 12): with s = x1 + x2, u = x1 - x2, m = x0 - s/2 and h = sqrt(3)/2,
//     y0 = x0 + s,   y1 = m - i h u,   y2 = m + i h u     (omega^-bc)
// and the conjugate signs for the composition.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "tpd.h"

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

template <class T>
struct Twiddles {
  T re[8], im[8];     // omega^k, k < d
  T h;                // sqrt(3) / 2 (d = 3)
  T scale;            // factor applied to every output of this launch
};

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

template <class T, bool kDec>
cudaError_t launch_levels(void* mat, int n, int d, double last_scale, cudaStream_t st) {
  long long N = 1;
  for (int k = 0; k < n; ++k) N *= d;
  const long long nblk = (N / d) * (N / d);
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
    // the decomposition's 1/d per level; the composition's scale on its last level
    const double sc = kDec ? 1.0 / d : (k == n - 1 ? last_scale : 1.0);
    const Twiddles<T> tw = twiddles<T>(d, sc);
    S* m = static_cast<S*>(mat);
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

tpd_status weyl_run(bool dec, void* A, int n, int d, int dtype, double scale, void* stream) {
  if (A == nullptr || d < 2 || d > 5 || n < 1 || (dtype != TPD_C128 && dtype != TPD_C64)) return TPD_ERR_INVALID_ARG;
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
    e = dec ? launch_levels<double, true>(A, n, d, 1.0, st) : launch_levels<double, false>(A, n, d, scale, st);
  else
    e = dec ? launch_levels<float, true>(A, n, d, 1.0, st) : launch_levels<float, false>(A, n, d, scale, st);
  return e == cudaSuccess ? TPD_OK : TPD_ERR_CUDA;
}

}  // namespace
}  // namespace tpd

extern "C" {

tpd_status tpd_weyl_decompose(void* A, int n, int d, int dtype, void* stream) {
  return tpd::weyl_run(true, A, n, d, dtype, 1.0, stream);
}

tpd_status tpd_weyl_compose(void* C, int n, int d, int dtype, double scale, void* stream) {
  return tpd::weyl_run(false, C, n, d, dtype, scale, stream);
}

}  // extern "C"
