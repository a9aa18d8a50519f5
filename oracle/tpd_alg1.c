/*
 * The paper's Tensorized Pauli Decomposition on the CPU, in its two forms.
 *
 * oracle_tpd_alg1: the recursive form (Alg. 1, Sec. III), as the paper states
 * it: split the matrix into the four blocks of Eq. 3, form the cumulative
 * matrix weights of Eq. 4
 *
 *     Omega_I = (A11 + A22)/2,  Omega_X = (A12 + A21)/2,
 *     Omega_Y = i (A12 - A21)/2,  Omega_Z = (A11 - A22)/2,
 *
 * one after the other, and recurse on each one that is not zero (exact test:
 * every real and imaginary part == 0); a 1x1 CMW is the weight of the string
 * built so far (Eq. 5).
 *
 * oracle_tpd_alg2: the iterative form (Alg. 2): level by level, every CMW of
 * the current level is split into its four children at once.  Stored in
 * place in one N x N array (the children of a block take its four
 * quadrants, the layout the GPU path also uses), with OpenMP over the
 * blocks of a level; a quadrant quad that is all zero stays zero (the
 * pruning of zero CMWs costs nothing in place).  The result is reordered to
 * string order at the end.
 *
 * TEST INFRASTRUCTURE ONLY: the algorithmic CPU baselines of the benchmark
 * and independent checks of the definitional functions in tpd_oracle.c (they
 * share nothing with them).  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may load or run them.
 *
 * Output: all 4^n weights in STRING order (t_1 most significant), strings
 * below a zero CMW left at 0.  fp64, no FMA.
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

/* One level of Alg. 2 on the whole array: for qubit j (row / column bit
 * beta = n - j of the index), every 2x2 quad (r_beta, c_beta) of every CMW
 * becomes (I, X, Y, Z) = ((a00+a11)/2, (a01+a10)/2, i(a01-a10)/2, (a00-a11)/2)
 * at the quad's four positions (Eq. 4 applied to all CMWs of the level). */
static void alg2_level(cplx1* W, int n, int beta) {
  const int64_t N = (int64_t)1 << n;
  const int64_t quads = (int64_t)1 << (2 * n - 2);
  const int64_t lo = ((int64_t)1 << beta) - 1;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < quads; ++q) {
    /* q = (the n-1 other row bits, the n-1 other column bits); insert a zero
       at bit beta of each to get the quad's a00 position */
    const int64_t cq = q & ((N >> 1) - 1), rq = q >> (n - 1);
    const int64_t c = (cq & lo) | ((cq & ~lo) << 1);
    const int64_t r = (rq & lo) | ((rq & ~lo) << 1);
    const int64_t i00 = r * N + c, i01 = i00 + ((int64_t)1 << beta);
    const int64_t i10 = i00 + (((int64_t)1 << beta) * N), i11 = i10 + ((int64_t)1 << beta);
    const cplx1 a00 = W[i00], a01 = W[i01], a10 = W[i10], a11 = W[i11];
    if (a00.re == 0.0 && a00.im == 0.0 && a01.re == 0.0 && a01.im == 0.0 && a10.re == 0.0 && a10.im == 0.0 &&
        a11.re == 0.0 && a11.im == 0.0)
      continue;                                      /* a zero quad of a CMW: its children stay zero */
    W[i00].re = (a00.re + a11.re) * 0.5; W[i00].im = (a00.im + a11.im) * 0.5;
    W[i01].re = (a01.re + a10.re) * 0.5; W[i01].im = (a01.im + a10.im) * 0.5;
    W[i10].re = -((a01.im - a10.im) * 0.5); W[i10].im = (a01.re - a10.re) * 0.5;
    W[i11].re = (a00.re - a11.re) * 0.5; W[i11].im = (a00.im - a11.im) * 0.5;
  }
}

/* A_: N x N complex128, overwritten (the in-place working array);
 * out_: 4^n complex128, string order. */
int oracle_tpd_alg2(double* A_, int n, double* out_) {
  if (n < 1 || n > 16) return 1;
  cplx1* W = (cplx1*)A_;
  cplx1* out = (cplx1*)out_;
  const int64_t N = (int64_t)1 << n;
  for (int j = 1; j <= n; ++j) alg2_level(W, n, n - j);       /* qubit 1 (the top bit) first */
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < N * N; ++s) {                         /* string s: digit b = (r_b, c_b) */
    int64_t r = 0, c = 0;
    for (int b = 0; b < n; ++b) {
      c |= ((s >> (2 * b)) & 1) << b;
      r |= ((s >> (2 * b + 1)) & 1) << b;
    }
    out[s] = W[r * N + c];
  }
  return 0;
}
