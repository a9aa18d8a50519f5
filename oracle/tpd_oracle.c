/*
 * Plain CPU oracle for the Pauli decomposition of arXiv:2310.13421.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load or run this file.  It shares
 * no code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * What it computes (Sec. II.A, Eq. 2): for A in Mat(2^n) and every quaternary
 * string t in Q^n,
 *
 *     w_t = 2^-n tr(sigma^t A),   sigma^t = sigma^{t_1} (x) ... (x) sigma^{t_n}   (Eq. 1)
 *
 * with sigma^0..3 = I, X, Y, Z (Sec. II.A).  The tensor factor t_1 acts on the
 * most significant bit of the row / column index: Eq. 3 splits A into the
 * quadrants A11, A12, A21, A22 by that bit.  Qubit j <-> index bit beta = n-j.
 *
 * Evaluation without matrix products.  A Pauli string has one nonzero per row
 * (the fact the Pauli Composer rests on, Sec. II.B).  Per factor, row bit r_b
 * of sigma^t has its entry at column r_b xor x_b with value 1 (I, X),
 * (-1)^{r_b} (Z) or -i (-1)^{r_b} (Y), where x_b = [t_b in {X,Y}] and
 * z_b = [t_b in {Y,Z}].  Hence sigma^t[r][r^x] = (-i)^{#Y} (-1)^{popc(z&r)} and
 *
 *     tr(sigma^t A) = sum_r sigma^t[r][r^x] A[r^x][r]
 *                   = (-i)^{#Y} sum_r (-1)^{popc(z&r)} A[r^x][r].          (*)
 *
 * Nothing else: no butterfly, no CMW (Eq. 4) and no blocking.  The sum over r
 * runs in increasing r, in double, with a branch for the sign (no FMA).
 *
 * Layouts.  A is row-major N x N complex128 (re, im interleaved), N = 2^n.
 * Coefficients are in STRING order: s = sum_j t_j 4^{n-j}, i.e. base 4 with
 * t_1 most significant; in terms of index bits, t at bit beta is
 * (s >> 2 beta) & 3.
 *
 * Functions:
 *   oracle_coeffs          all 4^n w_t by (*)                        O(8^n)
 *   oracle_coeffs_at       w_t for a list of strings by (*)          O(count 2^n)
 *   oracle_coeffs_xrows    all z for given x by (*) with the inner
 *                          sum over r done by a Walsh-Hadamard transform,
 *                          a textbook routine for sum_r (-1)^{popc(z&r)} v[r]
 *                                                                    O(count n 2^n)
 *   oracle_coeffs_xdiags   the same from the gathered entries A[r^x][r]
 *   oracle_coeffs_fwht     the same for every x                      O(n 4^n)
 *   oracle_compose         A = sum_t w_t sigma^t (Eq. 2, left side)  O(8^n)
 *   oracle_compose_fwht    the same, the sum over z per x-mask done by
 *                          the Walsh-Hadamard transform              O(n 4^n)
 *   oracle_num_threads     OpenMP threads used
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static int popc64(uint64_t v) {
  int c = 0;
  while (v) { v &= v - 1; ++c; }
  return c;
}

/* Pauli index at qubit bit beta from the X and Z masks:
 * (x,z) = (0,0) I=0, (1,0) X=1, (1,1) Y=2, (0,1) Z=3  (Sec. II.A ordering). */
static unsigned pauli_of(uint64_t x, uint64_t z, int beta) {
  unsigned xb = (unsigned)(x >> beta) & 1u, zb = (unsigned)(z >> beta) & 1u;
  if (!xb && !zb) return 0u;
  if (xb && !zb) return 1u;
  if (xb && zb) return 2u;
  return 3u;
}

static uint64_t string_index(uint64_t x, uint64_t z, int n) {
  uint64_t s = 0;
  for (int beta = 0; beta < n; ++beta) s |= (uint64_t)pauli_of(x, z, beta) << (2 * beta);
  return s;
}

static void string_masks(uint64_t s, int n, uint64_t* x, uint64_t* z) {
  uint64_t xm = 0, zm = 0;
  for (int beta = 0; beta < n; ++beta) {
    unsigned t = (unsigned)(s >> (2 * beta)) & 3u;
    if (t == 1u || t == 2u) xm |= (uint64_t)1 << beta;
    if (t == 2u || t == 3u) zm |= (uint64_t)1 << beta;
  }
  *x = xm; *z = zm;
}

/* multiply by (-i)^k, exact */
static cplx times_minus_i_pow(cplx v, int k) {
  cplx o;
  switch (k & 3) {
    case 0: o = v; break;
    case 1: o.re = v.im; o.im = -v.re; break;      /* -i (a+ib) = b - ia */
    case 2: o.re = -v.re; o.im = -v.im; break;
    default: o.re = -v.im; o.im = v.re; break;     /*  i (a+ib) = -b + ia */
  }
  return o;
}

/* (*) for one string, given the gathered diagonal v[r] = A[r^x][r] */
static cplx signed_sum(const cplx* v, uint64_t N, uint64_t z) {
  cplx acc = {0.0, 0.0};
  for (uint64_t r = 0; r < N; ++r) {
    if (popc64(z & r) & 1) { acc.re -= v[r].re; acc.im -= v[r].im; }
    else                   { acc.re += v[r].re; acc.im += v[r].im; }
  }
  return acc;
}

static cplx finish(cplx acc, int n, uint64_t x, uint64_t z) {
  cplx w = times_minus_i_pow(acc, popc64(x & z));
  w.re = ldexp(w.re, -n);
  w.im = ldexp(w.im, -n);
  return w;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* All 4^n coefficients by (*).  out: 4^n complex in string order. */
int oracle_coeffs(const double* A_, int n, double* out_) {
  if (n < 0 || n > 15) return 1;
  const cplx* A = (const cplx*)A_;
  cplx* out = (cplx*)out_;
  const uint64_t N = (uint64_t)1 << n;
  int bad = 0;
#pragma omp parallel
  {
    cplx* v = (cplx*)malloc(sizeof(cplx) * N);
    if (!v) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t xi = 0; xi < (int64_t)N; ++xi) {
        uint64_t x = (uint64_t)xi;
        for (uint64_t r = 0; r < N; ++r) v[r] = A[(r ^ x) * N + r];
        for (uint64_t z = 0; z < N; ++z)
          out[string_index(x, z, n)] = finish(signed_sum(v, N, z), n, x, z);
      }
      free(v);
    }
  }
  return bad;
}

/* w_t for count strings s[0..count) by (*).  out: count complex. */
int oracle_coeffs_at(const double* A_, int n, const uint64_t* s, int64_t count, double* out_) {
  if (n < 0 || n > 20) return 1;
  const cplx* A = (const cplx*)A_;
  cplx* out = (cplx*)out_;
  const uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < count; ++i) {
    uint64_t x, z;
    string_masks(s[i], n, &x, &z);
    cplx acc = {0.0, 0.0};
    for (uint64_t r = 0; r < N; ++r) {
      cplx a = A[(r ^ x) * N + r];
      if (popc64(z & r) & 1) { acc.re -= a.re; acc.im -= a.im; }
      else                   { acc.re += a.re; acc.im += a.im; }
    }
    out[i] = finish(acc, n, x, z);
  }
  return 0;
}

/* In-place Walsh-Hadamard transform, natural order:
 * v[z] <- sum_r (-1)^{popc(z&r)} v[r].  Textbook radix-2 form. */
static void wht(cplx* v, uint64_t N) {
  for (uint64_t h = 1; h < N; h <<= 1)
    for (uint64_t i = 0; i < N; i += 2 * h)
      for (uint64_t j = i; j < i + h; ++j) {
        cplx a = v[j], b = v[j + h];
        v[j].re = a.re + b.re;     v[j].im = a.im + b.im;
        v[j + h].re = a.re - b.re; v[j + h].im = a.im - b.im;
      }
}

/* For each of count masks x[i], all N coefficients w_{(x,z)}, z = 0..N-1.
 * out: count x N complex, row i holds z = 0..N-1 (NOT string order); the
 * string of entry (i, z) is string_index(x[i], z). */
int oracle_coeffs_xrows(const double* A_, int n, const uint64_t* xs, int64_t count, double* out_) {
  if (n < 0 || n > 20) return 1;
  const cplx* A = (const cplx*)A_;
  cplx* out = (cplx*)out_;
  const uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < count; ++i) {
    uint64_t x = xs[i];
    cplx* v = out + (uint64_t)i * N;
    for (uint64_t r = 0; r < N; ++r) v[r] = A[(r ^ x) * N + r];
    wht(v, N);
    for (uint64_t z = 0; z < N; ++z) v[z] = finish(v[z], n, x, z);
  }
  return 0;
}

/* The same rows from the gathered entries: V (count x N complex, in place)
 * holds V[i][r] = A[r ^ x[i]][r] on entry and w_{(x[i], z)} at [i][z] on
 * return -- for matrices the caller holds in another storage type (the
 * entries gathered and widened to double exactly by the caller). */
int oracle_coeffs_xdiags(double* V_, int n, const uint64_t* xs, int64_t count) {
  if (n < 0 || n > 20) return 1;
  cplx* V = (cplx*)V_;
  const uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < count; ++i) {
    uint64_t x = xs[i];
    cplx* v = V + (uint64_t)i * N;
    wht(v, N);
    for (uint64_t z = 0; z < N; ++z) v[z] = finish(v[z], n, x, z);
  }
  return 0;
}

/* All 4^n coefficients, string order, by the x-row transform above. */
int oracle_coeffs_fwht(const double* A_, int n, double* out_) {
  if (n < 0 || n > 20) return 1;
  const cplx* A = (const cplx*)A_;
  cplx* out = (cplx*)out_;
  const uint64_t N = (uint64_t)1 << n;
  int bad = 0;
#pragma omp parallel
  {
    cplx* v = (cplx*)malloc(sizeof(cplx) * N);
    if (!v) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t xi = 0; xi < (int64_t)N; ++xi) {
        uint64_t x = (uint64_t)xi;
        for (uint64_t r = 0; r < N; ++r) v[r] = A[(r ^ x) * N + r];
        wht(v, N);
        for (uint64_t z = 0; z < N; ++z) out[string_index(x, z, n)] = finish(v[z], n, x, z);
      }
      free(v);
    }
  }
  return bad;
}

/* A = sum_t w_t sigma^t (Eq. 2), w in string order.  Entry (r, r^x) collects
 * w_{(x,z)} (-i)^{popc(x&z)} (-1)^{popc(z&r)} over z. */
int oracle_compose(const double* w_, int n, double* A_) {
  if (n < 0 || n > 15) return 1;
  const cplx* w = (const cplx*)w_;
  cplx* A = (cplx*)A_;
  const uint64_t N = (uint64_t)1 << n;
  int bad = 0;
#pragma omp parallel
  {
    cplx* u = (cplx*)malloc(sizeof(cplx) * N);
    if (!u) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t xi = 0; xi < (int64_t)N; ++xi) {
        uint64_t x = (uint64_t)xi;
        for (uint64_t z = 0; z < N; ++z)
          u[z] = times_minus_i_pow(w[string_index(x, z, n)], popc64(x & z));
        for (uint64_t r = 0; r < N; ++r) A[r * N + (r ^ x)] = signed_sum(u, N, r);
      }
      free(u);
    }
  }
  return bad;
}

/* A = sum_t w_t sigma^t, w in string order; for each x the entries
 * A[r][r^x] = sum_z u[z] (-1)^{popc(z&r)} with u[z] = w_(x,z) (-i)^{popc(x&z)},
 * i.e. a Walsh-Hadamard transform of u. */
int oracle_compose_fwht(const double* w_, int n, double* A_) {
  if (n < 0 || n > 15) return 1;
  const cplx* w = (const cplx*)w_;
  cplx* A = (cplx*)A_;
  const uint64_t N = (uint64_t)1 << n;
  int bad = 0;
#pragma omp parallel
  {
    cplx* u = (cplx*)malloc(sizeof(cplx) * N);
    if (!u) {
#pragma omp atomic write
      bad = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t xi = 0; xi < (int64_t)N; ++xi) {
        uint64_t x = (uint64_t)xi;
        for (uint64_t z = 0; z < N; ++z)
          u[z] = times_minus_i_pow(w[string_index(x, z, n)], popc64(x & z));
        wht(u, N);
        for (uint64_t r = 0; r < N; ++r) A[r * N + (r ^ x)] = u[r];
      }
      free(u);
    }
  }
  return bad;
}
