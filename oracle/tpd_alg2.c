/*
 * The paper's Tensorized Pauli Decomposition on the CPU, in its iterative
 * form (Alg. 2, Sec. III): level by level, every cumulative matrix weight
 * (CMW) of the current level is split into the four CMWs of Eq. 4,
 *
 *     Omega_I = (A11 + A22)/2,  Omega_X = (A12 + A21)/2,
 *     Omega_Y = i (A12 - A21)/2,  Omega_Z = (A11 - A22)/2,
 *
 * over all n qubits (Eq. 5: after the last level every CMW is a 1x1 weight).
 * The CMWs of a level are kept in place in one N x N array: the children of
 * a block take its four quadrants (the layout the GPU path also uses), so a
 * level is a sweep over all 2x2 quads (r_beta, c_beta) of one qubit's row and
 * column bit.  A quad that is all zero belongs to a zero CMW and stays zero:
 * the paper's pruning of zero CMWs costs nothing in place.  OpenMP over the
 * quads of a level; the result is reordered to string order at the end.
 *
 * TEST INFRASTRUCTURE ONLY: the algorithmic CPU baseline of the benchmark and
 * an independent check of the definitional functions in tpd_oracle.c (it
 * shares nothing with them).  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load or run it.
 *
 * Output: all 4^n weights in STRING order (t_1 most significant).  fp64, no
 * FMA.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx2;

/* One level on the whole array: for qubit j (row / column bit beta = n - j of
 * the index), every 2x2 quad (r_beta, c_beta) of every CMW becomes
 * (I, X, Y, Z) = ((a00+a11)/2, (a01+a10)/2, i(a01-a10)/2, (a00-a11)/2) at the
 * quad's four positions (Eq. 4 applied to all CMWs of the level). */
static void alg2_level(cplx2* W, int n, int beta, int nthreads) {
  const int64_t N = (int64_t)1 << n;
  const int64_t quads = (int64_t)1 << (2 * n - 2);
  const int64_t lo = ((int64_t)1 << beta) - 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int64_t q = 0; q < quads; ++q) {
    /* q = (the n-1 other row bits, the n-1 other column bits); insert a zero
       at bit beta of each to get the quad's a00 position */
    const int64_t cq = q & ((N >> 1) - 1), rq = q >> (n - 1);
    const int64_t c = (cq & lo) | ((cq & ~lo) << 1);
    const int64_t r = (rq & lo) | ((rq & ~lo) << 1);
    const int64_t i00 = r * N + c, i01 = i00 + ((int64_t)1 << beta);
    const int64_t i10 = i00 + (((int64_t)1 << beta) * N), i11 = i10 + ((int64_t)1 << beta);
    const cplx2 a00 = W[i00], a01 = W[i01], a10 = W[i10], a11 = W[i11];
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
 * out_: 4^n complex128, string order; nthreads: OpenMP threads (<= 0: all). */
int oracle_tpd_alg2(double* A_, int n, double* out_, int nthreads) {
  if (n < 1 || n > 16) return 1;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
  cplx2* W = (cplx2*)A_;
  cplx2* out = (cplx2*)out_;
  const int64_t N = (int64_t)1 << n;
  for (int j = 1; j <= n; ++j) alg2_level(W, n, n - j, nthreads);   /* qubit 1 (the top bit) first */
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int64_t s = 0; s < N * N; ++s) {                               /* string s: digit b = (r_b, c_b) */
    int64_t r = 0, c = 0;
    for (int b = 0; b < n; ++b) {
      c |= ((s >> (2 * b)) & 1) << b;
      r |= ((s >> (2 * b + 1)) & 1) << b;
    }
    out[s] = W[r * N + c];
  }
  return 0;
}
