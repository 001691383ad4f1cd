/*
 * oracle.c -- plain, slow CPU reference for the dense N x N FP64 product.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file; only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no -ffast-math).
 * Contraction is off so that every a*b is rounded before it is added, as the
 * paper's C loops do on its 2010 x86 CPUs.
 *
 * Layout: row-major, dense.  Sections 1-4 take square n x n matrices;
 * section 5 takes C (m x n) = A (m x k) . B (k x n).
 *
 * Contents
 *   1. The product as the paper defines it (Alg. 1, Sec. 3.1; the same
 *      arithmetic appears in the worker loop of Alg. 3 and in Alg. 4).
 *   2. Helpers for judging a GPU result: |A||B|, a compensated dot product
 *      reference, Freivalds' check and sampled rows.
 *   3. A model of the split-precision emulation, step by step: row/column
 *      exponents, the integer split into base-2^8 digits, the exact level
 *      sums of digit products, and the single rounding to FP64.  This part
 *      has no counterpart in the paper (the paper computes in native FP64
 *      only); it follows the error-free splitting of Ozaki, Ogita, Oishi and
 *      Rump (Numer. Algorithms 59, 2012) with a fixed-point reading that is
 *      spelled out at each function.
 *   4. The exact product of fixed-point operands, rounded once (the model
 *      of the library's modular form; no counterpart in the paper).
 *   5. Sections 1, 2 (|A||B|), 3 and 4 for rectangular shapes (the paper's
 *      NRA x NCA times NCA x NCB of Alg. 2).
 *   6. A model of the INT8 slice form: section 3's splitting with a width
 *      one bit narrower, so that every digit is a signed byte.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__FAST_MATH__)
#error "the oracle must not be built with -ffast-math"
#endif

/* ------------------------------------------------------------------------ */
/* 1. The product C = A.B                                                    */
/* ------------------------------------------------------------------------ */

/* Alg. 1 (Sec. 3.1) written out literally: for i, for k, for j,
 * c(i,k) <- c(i,k) + a(i,j) * b(j,k), with c(i,k) starting from 0.0 as in
 * Alg. 3 and Alg. 4.  Every c(i,k) is a left-to-right sum over j. */
void or_gemm_alg1(int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double c = 0.0;
      for (int j = 0; j < n; ++j) c = c + A[(size_t)i * n + j] * B[(size_t)j * n + k];
      C[(size_t)i * n + k] = c;
    }
}

/* The same arithmetic with the j loop hoisted above k, and the rows of C
 * shared among threads as the "omp for" over I does in Alg. 4.  Each
 * c(i,k) still receives its products in increasing j, starting from 0.0,
 * so the result equals or_gemm_alg1 bit for bit for any thread count. */
void or_gemm(int n, const double* A, const double* B, double* C, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int i = 0; i < n; ++i) {
    double* c = C + (size_t)i * n;
    for (int k = 0; k < n; ++k) c[k] = 0.0;
    for (int j = 0; j < n; ++j) {
      const double a = A[(size_t)i * n + j];
      const double* b = B + (size_t)j * n;
      for (int k = 0; k < n; ++k) c[k] = c[k] + a * b[k];
    }
  }
  (void)nthreads;
}

/* Rows `rows[0..nrows)` of C = A.B, same arithmetic as or_gemm; row r of
 * the output goes to out[r * n ...]. */
void or_gemm_rows(int n, const double* A, const double* B, const int* rows, int nrows,
                  double* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int r = 0; r < nrows; ++r) {
    const int i = rows[r];
    double* c = out + (size_t)r * n;
    for (int k = 0; k < n; ++k) c[k] = 0.0;
    for (int j = 0; j < n; ++j) {
      const double a = A[(size_t)i * n + j];
      const double* b = B + (size_t)j * n;
      for (int k = 0; k < n; ++k) c[k] = c[k] + a * b[k];
    }
  }
  (void)nthreads;
}

/* ------------------------------------------------------------------------ */
/* 2. Judging a result                                                       */
/* ------------------------------------------------------------------------ */

/* |A||B|: the componentwise denominator of the error measure
 * |C - C_ref| / (|A||B|).  Same loop as or_gemm on absolute values. */
void or_absgemm(int n, const double* A, const double* B, double* C, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int i = 0; i < n; ++i) {
    double* c = C + (size_t)i * n;
    for (int k = 0; k < n; ++k) c[k] = 0.0;
    for (int j = 0; j < n; ++j) {
      const double a = fabs(A[(size_t)i * n + j]);
      const double* b = B + (size_t)j * n;
      for (int k = 0; k < n; ++k) c[k] = c[k] + a * fabs(b[k]);
    }
  }
  (void)nthreads;
}

/* Error-free transformations (Knuth's TwoSum; Dekker's TwoProduct with
 * Veltkamp's split, which needs no FMA).  Valid while no intermediate
 * overflows, i.e. for |a|, |b| well below 2^996. */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static void split(double a, double* hi, double* lo) {
  const double factor = 134217729.0; /* 2^27 + 1 */
  double c = factor * a;
  double h = c - (c - a);
  *hi = h;
  *lo = a - h;
}

static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  double ah, al, bh, bl;
  split(a, &ah, &al);
  split(b, &bh, &bl);
  *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
  *p = x;
}

/* Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): the dot
 * product computed as if in twice the working precision, then rounded.
 * Used only to report how far a result is from the exact product, so that
 * the oracle's own rounding is not charged to the GPU. */
void or_gemm_dot2(int n, const double* A, const double* B, double* C, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double p = 0.0, s = 0.0;
      for (int j = 0; j < n; ++j) {
        double h, r, q;
        two_prod(A[(size_t)i * n + j], B[(size_t)j * n + k], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
      }
      C[(size_t)i * n + k] = p + s;
    }
  (void)nthreads;
}

/* Freivalds' check (Freivalds 1977) with one probe vector x:
 *   y   = A (B x) - C x
 *   tol = (|A| (|B| |x|) + |C| |x|) * n * 2^-53 * slack
 * Writes y and tol (length n each) and returns the number of rows with
 * |y_i| > tol_i.  A product within 2 n 2^-53 |A||B| of the exact one, and
 * the rounding of the two matrix-vector products here, each contribute at
 * most a few n 2^-53 of those sums; `slack` covers them (4 is enough). */
int or_freivalds(int n, const double* A, const double* B, const double* C, const double* x,
                 double slack, double* y, double* tol) {
  double* bx = (double*)malloc(sizeof(double) * (size_t)n);
  double* abx = (double*)malloc(sizeof(double) * (size_t)n);
  if (!bx || !abx) { free(bx); free(abx); return -1; }
  for (int j = 0; j < n; ++j) {
    double s = 0.0, sa = 0.0;
    for (int k = 0; k < n; ++k) {
      s = s + B[(size_t)j * n + k] * x[k];
      sa = sa + fabs(B[(size_t)j * n + k]) * fabs(x[k]);
    }
    bx[j] = s;
    abx[j] = sa;
  }
  int bad = 0;
  const double u = ldexp(1.0, -53);
  for (int i = 0; i < n; ++i) {
    double s = 0.0, sa = 0.0, cx = 0.0, cxa = 0.0;
    for (int j = 0; j < n; ++j) {
      s = s + A[(size_t)i * n + j] * bx[j];
      sa = sa + fabs(A[(size_t)i * n + j]) * abx[j];
    }
    for (int k = 0; k < n; ++k) {
      cx = cx + C[(size_t)i * n + k] * x[k];
      cxa = cxa + fabs(C[(size_t)i * n + k]) * fabs(x[k]);
    }
    y[i] = s - cx;
    tol[i] = (sa + cxa) * (double)n * u * slack;
    if (!(fabs(y[i]) <= tol[i])) ++bad;
  }
  free(bx);
  free(abx);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* 3. Model of the split-precision emulation                                 */
/* ------------------------------------------------------------------------ */
/*
 * Notation: s slices, radix 2^8.
 *   e_i  smallest integer with max_j |a_ij| < 2^e_i   (0 for a zero row)
 *   f_k  smallest integer with max_j |b_jk| < 2^f_k   (0 for a zero column)
 *   D_ij = round-half-even(a_ij * 2^(8s - 1 - e_i)), an integer with
 *          |D_ij| <= 2^(8s-1)
 *   digits d_t(a_ij), t = 1..s:  D_ij = sum_t d_t 2^(8(s - t)),
 *          d_2..d_s in [-128, 127] (balanced base-256 residues taken from
 *          the least significant end), d_1 in [-128, 128]
 *   E_jk, digits d_u(b_jk) likewise with f_k.
 *   S_L(i,k) = sum_j sum_{t+u=L} d_t(a_ij) d_u(b_jk),  L = 2..s+1
 *          (the pairs with t + u <= s + 1; products of smaller weight are
 *          dropped, as in Ozaki's scheme)
 *   T(i,k) = sum_L S_L(i,k) 2^(8(s + 1 - L))           (exact integer)
 *   c_ik   = RN(T(i,k)) * 2^(e_i + f_k - 8s - 6)
 * where RN is one round-to-nearest-even to FP64.  The power-of-two scaling is
 * exact unless the result leaves the normal FP64 range.
 */

#define OR_EMU_MAX_SLICES 8

/* Smallest e with |v| < 2^e for the largest |v| of the n values at
 * p[0], p[stride], ...; 0 if they are all zero. */
static int exponent_of_max(const double* p, int n, size_t stride) {
  double m = 0.0;
  for (int j = 0; j < n; ++j) {
    double v = fabs(p[(size_t)j * stride]);
    if (v > m) m = v;
  }
  if (m == 0.0) return 0;
  int e;
  (void)frexp(m, &e); /* m = f 2^e with f in [0.5, 1), hence m < 2^e */
  return e;
}

void or_emu_row_exponents(int n, const double* A, int* e) {
  for (int i = 0; i < n; ++i) e[i] = exponent_of_max(A + (size_t)i * n, n, 1);
}

void or_emu_col_exponents(int n, const double* B, int* f) {
  for (int k = 0; k < n; ++k) f[k] = exponent_of_max(B + k, n, (size_t)n);
}

/* D = round-half-even(v * 2^(8s - 1 - e)).  ldexp is exact here (the
 * scaled magnitude stays below 2^63 and, when it is tiny, rounds to 0 under
 * any rounding), and nearbyint rounds half to even in the default mode. */
int64_t or_emu_fixed(double v, int e, int s) {
  return (int64_t)nearbyint(ldexp(v, 8 * s - 1 - e));
}

/* Digits d_1..d_s (written to d[0..s-1]) of the integer D.  Valid for
 * |D| <= 2^(8s-1); at s = 8 the fixed-point values stay below 2^63 - 2^10
 * (|x| <= 1 - 2^-53), so D - d_t never overflows. */
void or_emu_digits_of(int64_t D, int s, int* d) {
  for (int t = s; t >= 2; --t) {
    int r = (int)(D & 255);          /* D mod 256 in [0, 255] */
    int dt = r >= 128 ? r - 256 : r; /* balanced residue in [-128, 127] */
    d[t - 1] = dt;
    D = (D - dt) / 256;              /* exact division */
  }
  d[0] = (int)D;
}

/* Digit planes of a whole operand.  For A (col_major = 0) plane t holds
 * d_{t+1}(a_ij) at [t][i][j] using row exponents e; for B (col_major = 1)
 * plane u holds d_{u+1}(b_jk) at [u][j][k] using column exponents f. */
void or_emu_digit_planes(int n, int s, const double* M, const int* ex, int col_major,
                         int16_t* planes /* s*n*n */) {
  int d[OR_EMU_MAX_SLICES];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      int e = col_major ? ex[j] : ex[i];
      int64_t D = or_emu_fixed(M[(size_t)i * n + j], e, s);
      or_emu_digits_of(D, s, d);
      for (int t = 0; t < s; ++t) {
        size_t at = (size_t)t * n * n + (size_t)i * n + j;
        planes[at] = (int16_t)d[t];
      }
    }
}

/* Exact level sums S_L for L = 2..s+1, stored at S[(L-2)][i][k] (int64).
 * Integer products and sums: no rounding anywhere. */
void or_emu_level_sums(int n, int s, const int16_t* dA, const int16_t* dB, int64_t* S,
                       int nthreads) {
  const size_t nn = (size_t)n * n;
  memset(S, 0, sizeof(int64_t) * (size_t)s * nn);
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
#endif
  {
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int i = 0; i < n; ++i) {
      for (int t = 1; t <= s; ++t)
        for (int u = 1; t + u <= s + 1; ++u) {
          /* one pair product row: |sum| <= n 2^14 < 2^31 for n <= 2^16 */
          for (int k = 0; k < n; ++k) acc[k] = 0;
          const int16_t* a = dA + (size_t)(t - 1) * nn + (size_t)i * n;
          const int16_t* b = dB + (size_t)(u - 1) * nn;
          for (int j = 0; j < n; ++j) {
            const int32_t aj = a[j];
            const int16_t* bj = b + (size_t)j * n;
            for (int k = 0; k < n; ++k) acc[k] += aj * (int32_t)bj[k];
          }
          int64_t* SL = S + (size_t)(t + u - 2) * nn + (size_t)i * n;
          for (int k = 0; k < n; ++k) SL[k] += acc[k];
        }
    }
    free(acc);
  }
  (void)nthreads;
}

/* One rounding of T = sum_L S_L 2^(8(s+1-L)) to FP64, then the exact
 * power-of-two scaling 2^(e + f - 8s - 6).  The conversion of a 128-bit
 * integer to double rounds to nearest even (C Annex F; gcc's __floattidf). */
double or_emu_combine(const int64_t* S_levels /* S_2..S_{s+1} */, int s, int e, int f) {
  __int128 T = 0;
  for (int L = 2; L <= s + 1; ++L) T = T * 256 + (__int128)S_levels[L - 2];
  double r = (double)T;
  return ldexp(r, e + f - 8 * s - 6);
}

/* The whole emulated product C = A.B with s slices, from the definitions
 * above.  Scratch is allocated here. Returns 0 on success. */
int or_emu_gemm(int n, int s, const double* A, const double* B, double* C, int nthreads) {
  if (s < 1 || s > OR_EMU_MAX_SLICES || n < 0) return -1;
  if (n == 0) return 0;
  const size_t nn = (size_t)n * n;
  int* e = (int*)malloc(sizeof(int) * (size_t)n);
  int* f = (int*)malloc(sizeof(int) * (size_t)n);
  int16_t* dA = (int16_t*)malloc(sizeof(int16_t) * (size_t)s * nn);
  int16_t* dB = (int16_t*)malloc(sizeof(int16_t) * (size_t)s * nn);
  int64_t* S = (int64_t*)malloc(sizeof(int64_t) * (size_t)s * nn);
  if (!e || !f || !dA || !dB || !S) {
    free(e); free(f); free(dA); free(dB); free(S);
    return -2;
  }
  or_emu_row_exponents(n, A, e);
  or_emu_col_exponents(n, B, f);
  or_emu_digit_planes(n, s, A, e, 0, dA);
  or_emu_digit_planes(n, s, B, f, 1, dB);
  or_emu_level_sums(n, s, dA, dB, S, nthreads);
  int64_t lv[OR_EMU_MAX_SLICES];
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      for (int L = 0; L < s; ++L) lv[L] = S[(size_t)L * nn + (size_t)i * n + k];
      C[(size_t)i * n + k] = or_emu_combine(lv, s, e[i], f[k]);
    }
  free(e); free(f); free(dA); free(dB); free(S);
  return 0;
}

/* Rows `rows[0..nrows)` of the emulated product (for sizes where the full
 * model is too slow).  Same definitions; only the selected rows of A are
 * split, all of B is. Returns 0 on success. */
int or_emu_gemm_rows(int n, int s, const double* A, const double* B, const int* rows, int nrows,
                     double* out, int nthreads) {
  if (s < 1 || s > OR_EMU_MAX_SLICES || n < 0) return -1;
  if (n == 0 || nrows == 0) return 0;
  const size_t nn = (size_t)n * n;
  int* f = (int*)malloc(sizeof(int) * (size_t)n);
  int16_t* dB = (int16_t*)malloc(sizeof(int16_t) * (size_t)s * nn);
  if (!f || !dB) { free(f); free(dB); return -2; }
  or_emu_col_exponents(n, B, f);
  or_emu_digit_planes(n, s, B, f, 1, dB);
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(nthreads) reduction(+ : bad)
#endif
  for (int r = 0; r < nrows; ++r) {
    const int i = rows[r];
    const double* a = A + (size_t)i * n;
    int e = exponent_of_max(a, n, 1);
    int16_t* da = (int16_t*)malloc(sizeof(int16_t) * (size_t)s * n);
    int64_t* S = (int64_t*)calloc((size_t)s * n, sizeof(int64_t));
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!da || !S || !acc) { free(da); free(S); free(acc); ++bad; continue; }
    int d[OR_EMU_MAX_SLICES];
    for (int j = 0; j < n; ++j) {
      or_emu_digits_of(or_emu_fixed(a[j], e, s), s, d);
      for (int t = 0; t < s; ++t) da[(size_t)t * n + j] = (int16_t)d[t];
    }
    for (int t = 1; t <= s; ++t)
      for (int u = 1; t + u <= s + 1; ++u) {
        for (int k = 0; k < n; ++k) acc[k] = 0;
        for (int j = 0; j < n; ++j) {
          const int32_t aj = da[(size_t)(t - 1) * n + j];
          const int16_t* bj = dB + (size_t)(u - 1) * nn + (size_t)j * n;
          for (int k = 0; k < n; ++k) acc[k] += aj * (int32_t)bj[k];
        }
        for (int k = 0; k < n; ++k) S[(size_t)(t + u - 2) * n + k] += acc[k];
      }
    int64_t lv[OR_EMU_MAX_SLICES];
    for (int k = 0; k < n; ++k) {
      for (int L = 0; L < s; ++L) lv[L] = S[(size_t)L * n + k];
      out[(size_t)r * n + k] = or_emu_combine(lv, s, e, f[k]);
    }
    free(da); free(S); free(acc);
  }
  free(f); free(dB);
  return bad ? -2 : 0;
}

/* Number of OpenMP threads the oracle would use by default. */
int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* The double nearest (ties to even) to the 128-bit integer hi*2^64 + lo,
 * exposed so that tests can pin the conversion against exact arithmetic. */
double or_int128_to_double(int64_t hi, uint64_t lo) {
  __int128 T = ((__int128)hi << 64) | (__int128)lo;
  return (double)T;
}

/* ------------------------------------------------------------------------ */
/* 4. Exact product of fixed-point operands (model of the modular form)      */
/* ------------------------------------------------------------------------ */
/*
 * The library's second emulation form (no counterpart in the paper, which
 * computes in native FP64) rounds every operand to a fixed-point integer and
 * recovers the exact integer product from its residues modulo several small
 * moduli (Chinese remainder theorem), after Ozaki, Uchino and Imamura's
 * "Ozaki scheme II" (2025).  The residues are only the means; what it
 * computes has a plain definition, written out here without any modular
 * arithmetic:
 *   A_int(i,j) = round-half-even(a_ij 2^(beta - e_i)),  e_i as in section 3
 *   B_int(j,k) = round-half-even(b_jk 2^(beta - f_k)),  f_k likewise
 *   X(i,k)     = sum_j A_int(i,j) B_int(j,k)        (exact, 128-bit)
 *   c_ik       = RN(X(i,k)) 2^(e_i + f_k - 2 beta)
 * |A_int|, |B_int| <= 2^beta, so |X| <= n 2^(2 beta), below 2^126 whenever
 * 2 beta plus the bit length of n is at most 126 (checked; beta <= 62).
 */

/* round-half-even(v 2^(beta - e)); exact scaling as in or_emu_fixed. */
int64_t or_fix(double v, int e, int beta) { return (int64_t)nearbyint(ldexp(v, beta - e)); }

static int fixed_args_ok(int n, int beta) {
  int bits = 0;
  for (int v = n; v > 0; v >>= 1) ++bits;
  return n >= 0 && n < (1 << 17) && beta >= 1 && beta <= 62 && 2 * beta + bits <= 126;
}

/* Row i of the product from A_int row `ai` and all of B_int (row-major [j][k]). */
static void fixed_row(int n, int beta, const int64_t* ai, const int64_t* Bi, int e, const int* f,
                      __int128* acc, double* out) {
  for (int k = 0; k < n; ++k) acc[k] = 0;
  for (int j = 0; j < n; ++j) {
    const __int128 a = ai[j];
    const int64_t* b = Bi + (size_t)j * n;
    for (int k = 0; k < n; ++k) acc[k] += a * (__int128)b[k];
  }
  for (int k = 0; k < n; ++k) out[k] = ldexp((double)acc[k], e + f[k] - 2 * beta);
}

static int64_t* fixed_B(int n, int beta, const double* B, int* f) {
  int64_t* Bi = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * n);
  if (!Bi) return NULL;
  or_emu_col_exponents(n, B, f);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) Bi[(size_t)j * n + k] = or_fix(B[(size_t)j * n + k], f[k], beta);
  return Bi;
}

/* Rows `rows[0..nrows)` of the fixed-point product into out[nrows][n].
 * Returns 0 on success. */
int or_fixed_gemm_rows(int n, int beta, const double* A, const double* B, const int* rows, int nrows,
                       double* out, int nthreads) {
  if (!fixed_args_ok(n, beta)) return -1;
  if (n == 0 || nrows == 0) return 0;
  int* f = (int*)malloc(sizeof(int) * (size_t)n);
  int64_t* Bi = f ? fixed_B(n, beta, B, f) : NULL;
  if (!f || !Bi) { free(f); free(Bi); return -2; }
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(+ : bad)
#endif
  {
    int64_t* ai = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    __int128* acc = (__int128*)malloc(sizeof(__int128) * (size_t)n);
    if (!ai || !acc) {
      ++bad;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic)
#endif
      for (int r = 0; r < nrows; ++r) {
        const double* a = A + (size_t)rows[r] * n;
        const int e = exponent_of_max(a, n, 1);
        for (int j = 0; j < n; ++j) ai[j] = or_fix(a[j], e, beta);
        fixed_row(n, beta, ai, Bi, e, f, acc, out + (size_t)r * n);
      }
    }
    free(ai);
    free(acc);
  }
  (void)nthreads;
  free(f);
  free(Bi);
  return bad ? -2 : 0;
}

/* The whole fixed-point product C (n x n).  Returns 0 on success. */
int or_fixed_gemm(int n, int beta, const double* A, const double* B, double* C, int nthreads) {
  if (!fixed_args_ok(n, beta)) return -1;
  if (n == 0) return 0;
  int* rows = (int*)malloc(sizeof(int) * (size_t)n);
  if (!rows) return -2;
  for (int i = 0; i < n; ++i) rows[i] = i;
  const int r = or_fixed_gemm_rows(n, beta, A, B, rows, n, C, nthreads);
  free(rows);
  return r;
}

/* ------------------------------------------------------------------------ */
/* 5. Rectangular products: C (m x n) = A (m x k) . B (k x n)                */
/* ------------------------------------------------------------------------ */
/*
 * The paper's experiments are square, but its master/worker program names
 * the three dimensions separately (NRA rows of A, NCA columns of A = rows
 * of B, NCB columns of B; Alg. 2) and the product is defined for any of
 * them.  The functions below are the sections above with the three
 * dimensions kept apart; every matrix is row-major and dense (leading
 * dimension = its column count).  `rows` selects output rows (NULL: all m,
 * nrows = m); output row r goes to C[r * n ...].
 */

/* Section 1's product: c(i,l) = sum_j a(i,j) b(j,l), j increasing from 0.0. */
void or_gemm_mnk(int m, int n, int k, const double* A, const double* B, const int* rows, int nrows,
                 double* C, int nthreads) {
  if (!rows) nrows = m;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int r = 0; r < nrows; ++r) {
    const int i = rows ? rows[r] : r;
    double* c = C + (size_t)r * n;
    for (int l = 0; l < n; ++l) c[l] = 0.0;
    for (int j = 0; j < k; ++j) {
      const double a = A[(size_t)i * k + j];
      const double* b = B + (size_t)j * n;
      for (int l = 0; l < n; ++l) c[l] = c[l] + a * b[l];
    }
  }
  (void)nthreads;
}

/* |A||B| for the componentwise error measure. */
void or_absgemm_mnk(int m, int n, int k, const double* A, const double* B, double* C, int nthreads) {
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int i = 0; i < m; ++i) {
    double* c = C + (size_t)i * n;
    for (int l = 0; l < n; ++l) c[l] = 0.0;
    for (int j = 0; j < k; ++j) {
      const double a = fabs(A[(size_t)i * k + j]);
      const double* b = B + (size_t)j * n;
      for (int l = 0; l < n; ++l) c[l] = c[l] + a * fabs(b[l]);
    }
  }
  (void)nthreads;
}

/* Section 4's fixed-point product: e_i over the k entries of row i of A,
 * f_l over the k entries of column l of B, X = sum_j A_int B_int exactly,
 * c = RN(X) 2^(e_i + f_l - 2 beta).  |X| <= k 2^(2 beta).  0 on success. */
int or_fixed_gemm_mnk(int m, int n, int k, int beta, const double* A, const double* B, const int* rows,
                      int nrows, double* C, int nthreads) {
  if (m < 0 || n < 0 || !fixed_args_ok(k, beta)) return -1;
  if (!rows) nrows = m;
  if (nrows == 0 || n == 0) return 0;
  int* f = (int*)malloc(sizeof(int) * (size_t)n);
  int64_t* Bi = (int64_t*)malloc(sizeof(int64_t) * (size_t)k * n + 1);
  if (!f || !Bi) { free(f); free(Bi); return -2; }
  for (int l = 0; l < n; ++l) f[l] = exponent_of_max(B + l, k, (size_t)n);
  for (int j = 0; j < k; ++j)
    for (int l = 0; l < n; ++l) Bi[(size_t)j * n + l] = or_fix(B[(size_t)j * n + l], f[l], beta);
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(nthreads) reduction(+ : bad)
#endif
  for (int r = 0; r < nrows; ++r) {
    const double* a = A + (size_t)(rows ? rows[r] : r) * k;
    const int e = exponent_of_max(a, k, 1);
    __int128* acc = (__int128*)malloc(sizeof(__int128) * (size_t)n);
    if (!acc) { ++bad; continue; }
    for (int l = 0; l < n; ++l) acc[l] = 0;
    for (int j = 0; j < k; ++j) {
      const __int128 aj = or_fix(a[j], e, beta);
      const int64_t* b = Bi + (size_t)j * n;
      for (int l = 0; l < n; ++l) acc[l] += aj * (__int128)b[l];
    }
    for (int l = 0; l < n; ++l) C[(size_t)r * n + l] = ldexp((double)acc[l], e + f[l] - 2 * beta);
    free(acc);
  }
  (void)nthreads;
  free(f);
  free(Bi);
  return bad ? -2 : 0;
}

/* Section 3's digit model with s digits: the same exponents as above, the
 * digits d_t of D = round-half-even(v 2^(8s-1-e)), the exact level sums over
 * the pairs t + u <= s + 1 (one int32 sum per pair: k 2^14 < 2^31), and one
 * rounding per output (or_emu_combine).  0 on success. */
int or_emu_gemm_mnk(int m, int n, int k, int s, const double* A, const double* B, const int* rows, int nrows,
                    double* C, int nthreads) {
  if (s < 1 || s > OR_EMU_MAX_SLICES || m < 0 || n < 0 || k < 0 || k >= (1 << 17)) return -1;
  if (!rows) nrows = m;
  if (nrows == 0 || n == 0) return 0;
  int* f = (int*)malloc(sizeof(int) * (size_t)n);
  int16_t* dB = (int16_t*)malloc(sizeof(int16_t) * (size_t)s * k * n + 1);
  if (!f || !dB) { free(f); free(dB); return -2; }
  int d[OR_EMU_MAX_SLICES];
  for (int l = 0; l < n; ++l) f[l] = exponent_of_max(B + l, k, (size_t)n);
  for (int j = 0; j < k; ++j)
    for (int l = 0; l < n; ++l) {
      or_emu_digits_of(or_emu_fixed(B[(size_t)j * n + l], f[l], s), s, d);
      for (int u = 0; u < s; ++u) dB[((size_t)u * k + j) * n + l] = (int16_t)d[u];
    }
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(nthreads) reduction(+ : bad)
#endif
  for (int r = 0; r < nrows; ++r) {
    const double* a = A + (size_t)(rows ? rows[r] : r) * k;
    const int e = exponent_of_max(a, k, 1);
    int16_t* da = (int16_t*)malloc(sizeof(int16_t) * (size_t)s * k + 1);
    int64_t* S = (int64_t*)calloc((size_t)s * n, sizeof(int64_t));
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!da || !S || !acc) { free(da); free(S); free(acc); ++bad; continue; }
    int dd[OR_EMU_MAX_SLICES];
    for (int j = 0; j < k; ++j) {
      or_emu_digits_of(or_emu_fixed(a[j], e, s), s, dd);
      for (int t = 0; t < s; ++t) da[(size_t)t * k + j] = (int16_t)dd[t];
    }
    for (int t = 1; t <= s; ++t)
      for (int u = 1; t + u <= s + 1; ++u) {
        for (int l = 0; l < n; ++l) acc[l] = 0;
        for (int j = 0; j < k; ++j) {
          const int32_t aj = da[(size_t)(t - 1) * k + j];
          const int16_t* bj = dB + ((size_t)(u - 1) * k + j) * n;
          for (int l = 0; l < n; ++l) acc[l] += aj * (int32_t)bj[l];
        }
        for (int l = 0; l < n; ++l) S[(size_t)(t + u - 2) * n + l] += acc[l];
      }
    int64_t lv[OR_EMU_MAX_SLICES];
    for (int l = 0; l < n; ++l) {
      for (int L = 0; L < s; ++L) lv[L] = S[(size_t)L * n + l];
      C[(size_t)r * n + l] = or_emu_combine(lv, s, e, f[l]);
    }
    free(da); free(S); free(acc);
  }
  (void)nthreads;
  free(f);
  free(dB);
  return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* 6. Model of the INT8 slice form                                           */
/* ------------------------------------------------------------------------ */
/*
 * The library's third emulation form (no counterpart in the paper) is
 * Ozaki's error-free splitting with int8 slices and int32 accumulation, as
 * the integer tensor cores take it.  A signed byte holds -128..127, so the
 * fixed-point width is one bit narrower than section 3's, which keeps the
 * leading digit within [-64, 64]:
 *   D      = round-half-even(v 2^(8s - 2 - e)),  e the row (A) or column (B)
 *            exponent of section 3, so |D| <= 2^(8s - 2)
 *   D      = sum_{t=1..s} d_t 2^(8(s - t)), d_2..d_s in [-128, 127] (the
 *            balanced residues modulo 256, lowest first), d_1 the rest
 *   S_L    = sum_j sum_{t+u=L} d_t(a_ij) d_u(b_jk), L = 2..s+1, exact
 *   c_ik   = RN( sum_L S_L 2^(8(s+1-L)) ) 2^(e_i + f_k - 8s - 4)
 * (D_A D_B 2^(e+f-2(8s-2)) is the product of the rounded operands; of its
 * digit pairs only those with t + u <= s + 1 are kept, as in section 3.)
 * Written apart from section 3 so that each model reads on its own.
 */

/* round-half-even(v 2^(8s - 2 - e)); exact as in or_emu_fixed. */
int64_t or_i8_fixed(double v, int e, int s) { return (int64_t)nearbyint(ldexp(v, 8 * s - 2 - e)); }

/* Digits d_1..d_s of D (|D| <= 2^(8s-2)) into d[0..s-1]. */
void or_i8_digits_of(int64_t D, int s, int* d) {
  for (int t = s; t >= 2; --t) {
    const int r = (int)(D & 255);
    const int dt = r >= 128 ? r - 256 : r;
    d[t - 1] = dt;
    D = (D - dt) / 256;
  }
  d[0] = (int)D;
}

/* RN(sum_L S_L 2^(8(s+1-L))) 2^(e + f - 8s - 4), levels S_2..S_{s+1}. */
double or_i8_combine(const int64_t* S_levels, int s, int e, int f) {
  __int128 T = 0;
  for (int L = 2; L <= s + 1; ++L) T = T * 256 + (__int128)S_levels[L - 2];
  return ldexp((double)T, e + f - 8 * s - 4);
}

/* C (rows of A listed in `rows`, or all m rows if rows is NULL) of the INT8
 * slice model for A (m x k) and B (k x n), row-major.  Each digit pair's sum
 * over j is formed in int32 (|d_t d_u| <= 2^14, k < 2^17) and added into the
 * level in int64.  0 on success. */
int or_i8_gemm_mnk(int m, int n, int k, int s, const double* A, const double* B, const int* rows, int nrows,
                   double* C, int nthreads) {
  if (s < 1 || s > OR_EMU_MAX_SLICES || m < 0 || n < 0 || k < 0 || k >= (1 << 17)) return -1;
  if (!rows) nrows = m;
  if (nrows == 0 || n == 0) return 0;
  int* f = (int*)malloc(sizeof(int) * (size_t)n);
  int8_t* dB = (int8_t*)malloc((size_t)s * k * n + 1);
  if (!f || !dB) { free(f); free(dB); return -2; }
  int d[OR_EMU_MAX_SLICES];
  for (int l = 0; l < n; ++l) f[l] = exponent_of_max(B + l, k, (size_t)n);
  for (int j = 0; j < k; ++j)
    for (int l = 0; l < n; ++l) {
      or_i8_digits_of(or_i8_fixed(B[(size_t)j * n + l], f[l], s), s, d);
      for (int u = 0; u < s; ++u) dB[((size_t)u * k + j) * n + l] = (int8_t)d[u];
    }
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(nthreads) reduction(+ : bad)
#endif
  for (int r = 0; r < nrows; ++r) {
    const double* a = A + (size_t)(rows ? rows[r] : r) * k;
    const int e = exponent_of_max(a, k, 1);
    int8_t* da = (int8_t*)malloc((size_t)s * k + 1);
    int64_t* S = (int64_t*)calloc((size_t)s * n, sizeof(int64_t));
    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!da || !S || !acc) { free(da); free(S); free(acc); ++bad; continue; }
    int dd[OR_EMU_MAX_SLICES];
    for (int j = 0; j < k; ++j) {
      or_i8_digits_of(or_i8_fixed(a[j], e, s), s, dd);
      for (int t = 0; t < s; ++t) da[(size_t)t * k + j] = (int8_t)dd[t];
    }
    for (int t = 1; t <= s; ++t)
      for (int u = 1; t + u <= s + 1; ++u) {
        for (int l = 0; l < n; ++l) acc[l] = 0;
        for (int j = 0; j < k; ++j) {
          const int32_t aj = da[(size_t)(t - 1) * k + j];
          const int8_t* bj = dB + ((size_t)(u - 1) * k + j) * n;
          for (int l = 0; l < n; ++l) acc[l] += aj * (int32_t)bj[l];
        }
        for (int l = 0; l < n; ++l) S[(size_t)(t + u - 2) * n + l] += acc[l];
      }
    int64_t lv[OR_EMU_MAX_SLICES];
    for (int l = 0; l < n; ++l) {
      for (int L = 0; L < s; ++L) lv[L] = S[(size_t)L * n + l];
      C[(size_t)r * n + l] = or_i8_combine(lv, s, e, f[l]);
    }
    free(da); free(S); free(acc);
  }
  (void)nthreads;
  free(f);
  free(dB);
  return bad ? -2 : 0;
}
