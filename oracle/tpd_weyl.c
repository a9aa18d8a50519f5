/*
 * Plain CPU oracle for the decomposition in the Weyl (clock-and-shift) basis
 * of n qudits of dimension d -- the tensorized basis the paper names as the
 * natural next candidate for its method (Sec. V, Conclusion and Outlook).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load or run it.  It shares no code
 * with the CUDA path.
 *
 * Definitions (the reading this project takes; the paper names the basis
 * only).  For one qudit, with omega = exp(2 pi i / d):
 *     X |j> = |j + 1 mod d>      (shift),     Z |j> = omega^j |j>   (clock),
 *     W_{a,b} = X^a Z^b,   a, b in Z_d,  so  W_{a,b}[r][c] = omega^(b c) [r == c + a mod d].
 * The d^2 operators are orthogonal: tr(W_{a,b}^* W_{a',b'}) = d [a == a'][b == b'].
 * For n qudits W_{a,b} is the tensor product over the qudits (qudit 1 the
 * most significant base-d digit of the row / column index, as qubit 1 is the
 * top bit in the Pauli case), and the weights of A in Mat(d^n) are
 *     c_{a,b} = d^-n tr(W_{a,b}^* A),     A = sum_{a,b} c_{a,b} W_{a,b},
 * i.e. (trace over the one nonzero per column of W_{a,b})
 *     c_{a,b} = d^-n sum_{c in Z_d^n} omega^(-(b . c)) A[c + a][c]       (*)
 * with c + a digit-wise mod d and b . c = sum_j b_j c_j.  For d = 2,
 * W_{0,0} = I, W_{1,0} = X, W_{0,1} = Z, W_{1,1} = XZ = -iY, so c_{1,1} = i w_Y.
 *
 * Index conventions.  a, b, r, c are integers in [0, d^n) whose base-d digit
 * k (least significant k = 0) is the digit of qudit n - k.  Weights are
 * returned as out[a * d^n + b].  Matrices are row-major d^n x d^n complex128
 * (re, im interleaved).
 *
 * Functions:
 *   oracle_weyl_coeffs        all d^2n weights by (*)                    O(d^3n)
 *   oracle_weyl_rows          the weights of given shifts a, the sum over c
 *                             done as a tensor-product DFT over the digits
 *                                                                O(count n d^(n+1))
 *   oracle_weyl_diags         the same from the gathered diagonals A[c+a][c]
 *   oracle_weyl_coeffs_dft    the same for every shift                  O(n d^(2n+1))
 *   oracle_weyl_compose       A = sum c_{a,b} W_{a,b}                    O(d^3n)
 *
 * fp64, no FMA (compiled with -ffp-contract=off); the powers of omega come
 * from the C library's cos / sin of 2 pi k / d, values within a few ulps of
 * 0, +-1/2, +-1 taken exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } wcplx;

static int weyl_args_ok(int n, int d) { return d >= 2 && d <= 16 && n >= 1 && pow((double)d, 3.0 * n) <= 1e12; }

static int64_t ipow(int d, int n) {
  int64_t p = 1;
  for (int k = 0; k < n; ++k) p *= d;
  return p;
}

/* A cosine or sine value within a few ulps of 0, +-1/2 or +-1 is that value
 * exactly (the library's cos(pi) has a tiny sine, its cos(2 pi / 3) may miss
 * -1/2 by an ulp): quarter and sixth turns then carry no rounding. */
static double snap(double v) {
  const double h = nearbyint(2.0 * v) * 0.5;
  return fabs(v - h) <= 4e-16 ? h : v;
}

/* omega^k for k = 0..d-1 */
static void omega_table(int d, wcplx* w) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < d; ++k) {
    w[k].re = snap(cos(2.0 * pi * (double)k / (double)d));
    w[k].im = snap(sin(2.0 * pi * (double)k / (double)d));
  }
}

/* digit-wise (x + y) mod d of two base-d integers with n digits */
static int64_t dadd(int64_t x, int64_t y, int d, int n) {
  int64_t r = 0, p = 1;
  for (int k = 0; k < n; ++k) {
    r += ((x % d + y % d) % d) * p;
    x /= d; y /= d; p *= d;
  }
  return r;
}

/* sum of digit products mod d */
static int ddot(int64_t x, int64_t y, int d, int n) {
  int s = 0;
  for (int k = 0; k < n; ++k) {
    s = (s + (int)(x % d) * (int)(y % d)) % d;
    x /= d; y /= d;
  }
  return s;
}

int oracle_weyl_coeffs(const double* A_, int n, int d, double* out_) {
  if (!weyl_args_ok(n, d)) return 1;
  const wcplx* A = (const wcplx*)A_;
  wcplx* out = (wcplx*)out_;
  const int64_t N = ipow(d, n);
  wcplx w[16];
  omega_table(d, w);
  const double scale = 1.0 / (double)N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t a = 0; a < N; ++a) {
    for (int64_t b = 0; b < N; ++b) {
      double sr = 0.0, si = 0.0;
      for (int64_t c = 0; c < N; ++c) {
        const wcplx x = A[dadd(c, a, d, n) * N + c];
        const int k = (d - ddot(b, c, d, n)) % d;           /* omega^(-(b . c)) */
        sr += x.re * w[k].re - x.im * w[k].im;
        si += x.re * w[k].im + x.im * w[k].re;
      }
      out[a * N + b].re = sr * scale;
      out[a * N + b].im = si * scale;
    }
  }
  return 0;
}

/* In place on V (count x d^n): row i holds v[c] = A[c + a][c] of some shift
 * a on entry and c_{a,b} = d^-n sum_c omega^(-(b . c)) v[c], b = 0..d^n-1, on
 * return: the n-dimensional DFT over the digits of c done one digit at a
 * time (a textbook tensor-product DFT), then the scale. */
int oracle_weyl_diags(double* V_, int n, int d, int64_t count) {
  if (!(d >= 2 && d <= 16 && n >= 1 && pow((double)d, (double)n) <= 70000.0)) return 1;
  wcplx* V = (wcplx*)V_;
  const int64_t N = ipow(d, n);
  wcplx w[16];
  omega_table(d, w);
  const double scale = 1.0 / (double)N;
  int bad = 0;
#pragma omp parallel
  {
    wcplx* tmp = (wcplx*)malloc(sizeof(wcplx) * (size_t)d);
    if (!tmp) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < count; ++i) {
      if (!tmp) continue;
      wcplx* v = V + i * N;
      int64_t stride = 1;
      for (int k = 0; k < n; ++k, stride *= d) {          /* digit k of c -> digit k of b */
        for (int64_t base = 0; base < N; ++base) {
          if ((base / stride) % d != 0) continue;           /* base has digit k = 0 */
          for (int bk = 0; bk < d; ++bk) {
            double sr = 0.0, si = 0.0;
            for (int ck = 0; ck < d; ++ck) {
              const wcplx x = v[base + ck * stride];
              const int e = (d - (bk * ck) % d) % d;
              sr += x.re * w[e].re - x.im * w[e].im;
              si += x.re * w[e].im + x.im * w[e].re;
            }
            tmp[bk].re = sr; tmp[bk].im = si;
          }
          for (int bk = 0; bk < d; ++bk) v[base + bk * stride] = tmp[bk];
        }
      }
      for (int64_t b = 0; b < N; ++b) { v[b].re *= scale; v[b].im *= scale; }
    }
    free(tmp);
  }
  return bad ? 2 : 0;
}

/* The weights of the given shifts a = as[i]: the gathered diagonals
 * v[c] = A[c + a][c], then oracle_weyl_diags.  out: count x d^n. */
int oracle_weyl_rows(const double* A_, int n, int d, const int64_t* as, int64_t count, double* out_) {
  if (!(d >= 2 && d <= 16 && n >= 1 && pow((double)d, (double)n) <= 70000.0)) return 1;
  const wcplx* A = (const wcplx*)A_;
  wcplx* out = (wcplx*)out_;
  const int64_t N = ipow(d, n);
  for (int64_t i = 0; i < count; ++i)
    if (as[i] < 0 || as[i] >= N) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i)
    for (int64_t c = 0; c < N; ++c) out[i * N + c] = A[dadd(c, as[i], d, n) * N + c];
  return oracle_weyl_diags(out_, n, d, count);
}

/* All d^2n weights: the rows of every shift a. */
int oracle_weyl_coeffs_dft(const double* A_, int n, int d, double* out_) {
  if (!(d >= 2 && d <= 16 && n >= 1 && pow((double)d, 2.0 * n) <= 4e9)) return 1;
  const int64_t N = ipow(d, n);
  int64_t* as = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  if (!as) return 2;
  for (int64_t a = 0; a < N; ++a) as[a] = a;
  const int r = oracle_weyl_rows(A_, n, d, as, N, out_);
  free(as);
  return r;
}

/* A = sum_{a,b} c_{a,b} W_{a,b}: A[c + a][c] = sum_b c_{a,b} omega^(b . c). */
int oracle_weyl_compose(const double* C_, int n, int d, double* A_) {
  if (!weyl_args_ok(n, d)) return 1;
  const wcplx* C = (const wcplx*)C_;
  wcplx* A = (wcplx*)A_;
  const int64_t N = ipow(d, n);
  wcplx w[16];
  omega_table(d, w);
  memset(A, 0, sizeof(wcplx) * (size_t)(N * N));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t a = 0; a < N; ++a) {
    for (int64_t c = 0; c < N; ++c) {
      double sr = 0.0, si = 0.0;
      for (int64_t b = 0; b < N; ++b) {
        const wcplx x = C[a * N + b];
        const int k = ddot(b, c, d, n);
        sr += x.re * w[k].re - x.im * w[k].im;
        si += x.re * w[k].im + x.im * w[k].re;
      }
      A[dadd(c, a, d, n) * N + c].re = sr;
      A[dadd(c, a, d, n) * N + c].im = si;
    }
  }
  return 0;
}
