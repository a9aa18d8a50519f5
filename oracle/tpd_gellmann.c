/*
 * Plain CPU oracle for the decomposition in the generalized Gell-Mann basis
 * of n qudits of dimension d -- the other tensorized basis the paper names as
 * a natural candidate for its method (Sec. V, Conclusion and Outlook).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load or run it.  It shares no code
 * with the CUDA path.
 *
 * Definitions (the reading this project takes; the paper names the basis
 * only).  For one qudit, with E_jk the matrix unit (1 at row j, column k),
 * the d^2 Hermitian basis elements are labelled by a position (r, c) of the
 * d x d grid:
 *     (0, 0)          I                                     norm d
 *     (l, l), l >= 1  D_l = sqrt(2 / (l (l+1))) (sum_{m<l} E_mm - l E_ll)   norm 2
 *     (j, k), j < k   S_jk = E_jk + E_kj          (symmetric)               norm 2
 *     (k, j), j < k   A_jk = -i E_jk + i E_kj     (antisymmetric)           norm 2
 * where "norm" is tr(G^2); distinct elements are orthogonal, tr(G G') = 0.
 * For d = 2 these are I, X (0,1), Y (1,0), Z (1,1): the Pauli matrices at the
 * positions Eq. 4 gives their weights.  For d = 3 the eight traceless ones are
 * Gell-Mann's lambda_1..lambda_8.
 *
 * For n qudits the element of label (r, c) -- r, c in [0, d^n), base-d digit
 * k (least significant k = 0) the digit of qudit n - k, qudit 1 the most
 * significant as qubit 1 is the top bit in the Pauli case -- is the tensor
 * product of the single-qudit elements of the digit pairs (r_j, c_j), with
 * norm N_(r,c) = prod_j norm_j, and
 *     A = sum_(r,c) g_(r,c) G_(r,c),     g_(r,c) = tr(G_(r,c) A) / N_(r,c)      (*)
 * (the analogue of Eq. 2).  Coefficients are returned at out[r * d^n + c].
 *
 * Functions:
 *   oracle_gm_coeffs      all d^2n coefficients by (*): the trace written out
 *                         over the nonzero entries of each tensor product
 *   oracle_gm_coeffs_at   the coefficients of given labels by (*)
 *   oracle_gm_compose     A = sum g_(r,c) G_(r,c), entry by entry
 *
 * fp64, no FMA (compiled with -ffp-contract=off); sqrt from the C library
 * (correctly rounded in IEEE arithmetic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } gcplx;

/* one nonzero entry G[u][v] of a single-qudit element */
typedef struct {
  int u, v;
  double re, im;
} gm_entry;

#define GM_MAXD 16
#define GM_MAXN 32

static int gm_args_ok(int n, int d) { return d >= 2 && d <= GM_MAXD && n >= 1 && n <= GM_MAXN; }

static int64_t gm_ipow(int d, int n) {
  int64_t p = 1;
  for (int k = 0; k < n; ++k) p *= d;
  return p;
}

/* The nonzero entries of the single-qudit element labelled (r, c); returns
 * their count (at most d) and sets *norm to tr(G^2). */
static int gm_single(int d, int r, int c, gm_entry* e, double* norm) {
  int cnt = 0;
  if (r == 0 && c == 0) {                       /* identity */
    for (int m = 0; m < d; ++m) e[cnt++] = (gm_entry){m, m, 1.0, 0.0};
    *norm = (double)d;
  } else if (r == c) {                          /* D_l, l = r */
    const int l = r;
    const double f = sqrt(2.0 / ((double)l * (double)(l + 1)));
    for (int m = 0; m < l; ++m) e[cnt++] = (gm_entry){m, m, f, 0.0};
    e[cnt++] = (gm_entry){l, l, -(double)l * f, 0.0};
    *norm = 2.0;
  } else if (r < c) {                           /* S_rc */
    e[cnt++] = (gm_entry){r, c, 1.0, 0.0};
    e[cnt++] = (gm_entry){c, r, 1.0, 0.0};
    *norm = 2.0;
  } else {                                      /* A_jk with j = c < k = r */
    e[cnt++] = (gm_entry){c, r, 0.0, -1.0};
    e[cnt++] = (gm_entry){r, c, 0.0, 1.0};
    *norm = 2.0;
  }
  return cnt;
}

/* Per-qudit entry lists of the label (r, c): list j (qudit j + 1, digit
 * n - 1 - j) in e[j * d ..], its length in len[j]; returns the norm N. */
static double gm_label(int n, int d, int64_t r, int64_t c, gm_entry* e, int* len) {
  double norm = 1.0;
  for (int j = n - 1; j >= 0; --j) {            /* least significant digit: qudit n */
    double nj;
    len[j] = gm_single(d, (int)(r % d), (int)(c % d), e + (size_t)j * d, &nj);
    norm *= nj;
    r /= d;
    c /= d;
  }
  return norm;
}

/* g_(r,c) = tr(G A) / N = (1 / N) sum over the nonzeros (u, v) of G of
 * G[u][v] A[v][u]; the nonzeros of the tensor product are the products of
 * one entry per qudit (a mixed-radix counter over the lists). */
static gcplx gm_coeff(const gcplx* A, int n, int d, int64_t N, int64_t r, int64_t c) {
  gm_entry e[GM_MAXN * GM_MAXD];
  int len[GM_MAXN], idx[GM_MAXN];
  const double norm = gm_label(n, d, r, c, e, len);
  memset(idx, 0, sizeof(idx));
  double sr = 0.0, si = 0.0;
  for (;;) {
    double gr = 1.0, gi = 0.0;
    int64_t u = 0, v = 0;
    for (int j = 0; j < n; ++j) {               /* qudit 1 first: most significant digit */
      const gm_entry* x = e + (size_t)j * d + idx[j];
      const double tr = gr * x->re - gi * x->im;
      const double ti = gr * x->im + gi * x->re;
      gr = tr;
      gi = ti;
      u = u * d + x->u;
      v = v * d + x->v;
    }
    const gcplx a = A[v * N + u];               /* G[u][v] A[v][u] */
    sr += gr * a.re - gi * a.im;
    si += gr * a.im + gi * a.re;
    int j = n - 1;
    while (j >= 0 && ++idx[j] == len[j]) idx[j--] = 0;
    if (j < 0) break;
  }
  return (gcplx){sr / norm, si / norm};
}

int oracle_gm_coeffs(const double* A_, int n, int d, double* out_) {
  if (!gm_args_ok(n, d) || pow((double)d, 2.0 * n) > 4e9) return 1;
  const gcplx* A = (const gcplx*)A_;
  gcplx* out = (gcplx*)out_;
  const int64_t N = gm_ipow(d, n);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < N * N; ++t) out[t] = gm_coeff(A, n, d, N, t / N, t % N);
  return 0;
}

int oracle_gm_coeffs_at(const double* A_, int n, int d, const int64_t* rows, const int64_t* cols, int64_t count,
                        double* out_) {
  if (!gm_args_ok(n, d) || pow((double)d, (double)n) > 1e6) return 1;
  const gcplx* A = (const gcplx*)A_;
  gcplx* out = (gcplx*)out_;
  const int64_t N = gm_ipow(d, n);
  for (int64_t i = 0; i < count; ++i)
    if (rows[i] < 0 || rows[i] >= N || cols[i] < 0 || cols[i] >= N) return 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < count; ++i) out[i] = gm_coeff(A, n, d, N, rows[i], cols[i]);
  return 0;
}

/* A[u][v] = sum over labels (r, c) of g_(r,c) G_(r,c)[u][v]: each label's
 * nonzeros added into A in label order (serial: labels share entries). */
int oracle_gm_compose(const double* C_, int n, int d, double* A_) {
  if (!gm_args_ok(n, d) || pow((double)d, 2.0 * n) > 4e9) return 1;
  const gcplx* C = (const gcplx*)C_;
  gcplx* A = (gcplx*)A_;
  const int64_t N = gm_ipow(d, n);
  memset(A, 0, sizeof(gcplx) * (size_t)(N * N));
  gm_entry e[GM_MAXN * GM_MAXD];
  int len[GM_MAXN], idx[GM_MAXN];
  for (int64_t t = 0; t < N * N; ++t) {
    gm_label(n, d, t / N, t % N, e, len);
    const gcplx g = C[t];
    memset(idx, 0, sizeof(idx));
    for (;;) {
      double gr = 1.0, gi = 0.0;
      int64_t u = 0, v = 0;
      for (int j = 0; j < n; ++j) {
        const gm_entry* x = e + (size_t)j * d + idx[j];
        const double tr = gr * x->re - gi * x->im;
        const double ti = gr * x->im + gi * x->re;
        gr = tr;
        gi = ti;
        u = u * d + x->u;
        v = v * d + x->v;
      }
      A[u * N + v].re += g.re * gr - g.im * gi;
      A[u * N + v].im += g.re * gi + g.im * gr;
      int j = n - 1;
      while (j >= 0 && ++idx[j] == len[j]) idx[j--] = 0;
      if (j < 0) break;
    }
  }
  return 0;
}
