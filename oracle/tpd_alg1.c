/*
 * The paper's recursive Tensorized Pauli Decomposition (Alg. 1, Sec. III) on
 * the CPU, as the paper states it: split the matrix into the four blocks of
 * Eq. 3, form the cumulative matrix weights of Eq. 4
 *
 *     Omega_I = (A11 + A22)/2,  Omega_X = (A12 + A21)/2,
 *     Omega_Y = i (A12 - A21)/2,  Omega_Z = (A11 - A22)/2,
 *
 * one after the other, and recurse on each one that is not zero (exact test:
 * every real and imaginary part == 0); a 1x1 CMW is the weight of the string
 * built so far (Eq. 5).
 *
 * TEST INFRASTRUCTURE ONLY: the algorithmic CPU baseline of the benchmark and
 * an independent check of the definitional functions in tpd_oracle.c (it
 * shares nothing with them).  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load or run it.
 *
 * Output: all 4^n weights in STRING order (t_1 most significant), strings
 * below a zero CMW left at 0.  Single-threaded, fp64, no FMA.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx1;

static int all_zero(const cplx1* C, uint64_t count) {
  for (uint64_t k = 0; k < count; ++k)
    if (!(C[k].re == 0.0 && C[k].im == 0.0)) return 0;   /* NaN counts as nonzero */
  return 1;
}

/* A: 2^m x 2^m CMW of the strings with prefix `prefix` (base 4, n - m digits). */
static void tpd_rec(const cplx1* A, int m, uint64_t prefix, cplx1* out, cplx1* scratch) {
  if (m == 0) {
    out[prefix] = A[0];
    return;
  }
  const uint64_t M = 1ull << m, H = M >> 1;
  cplx1* C = scratch;
  for (int t = 0; t < 4; ++t) {
    for (uint64_t i = 0; i < H; ++i)
      for (uint64_t j = 0; j < H; ++j) {
        const cplx1 a11 = A[i * M + j], a12 = A[i * M + j + H];
        const cplx1 a21 = A[(i + H) * M + j], a22 = A[(i + H) * M + j + H];
        cplx1 c;
        switch (t) {
          case 0: c.re = (a11.re + a22.re) * 0.5; c.im = (a11.im + a22.im) * 0.5; break;
          case 1: c.re = (a12.re + a21.re) * 0.5; c.im = (a12.im + a21.im) * 0.5; break;
          case 2: c.re = -((a12.im - a21.im) * 0.5); c.im = (a12.re - a21.re) * 0.5; break;
          default: c.re = (a11.re - a22.re) * 0.5; c.im = (a11.im - a22.im) * 0.5; break;
        }
        C[i * H + j] = c;
      }
    if (!all_zero(C, H * H)) tpd_rec(C, m - 1, prefix * 4 + (uint64_t)t, out, scratch + H * H);
  }
}

/* A_: N x N complex128 (re, im interleaved); out_: 4^n complex128, string order. */
int oracle_tpd_alg1(const double* A_, int n, double* out_) {
  if (n < 0 || n > 16) return 1;
  const uint64_t N = 1ull << n;
  cplx1* out = (cplx1*)out_;
  memset(out, 0, sizeof(cplx1) * N * N);
  uint64_t scratch_elems = 0;
  for (int m = 1; m <= n; ++m) scratch_elems += 1ull << (2 * (m - 1));
  cplx1* scratch = (cplx1*)malloc(sizeof(cplx1) * (scratch_elems ? scratch_elems : 1));
  if (!scratch) return 2;
  tpd_rec((const cplx1*)A_, n, 0, out, scratch);
  free(scratch);
  return 0;
}
