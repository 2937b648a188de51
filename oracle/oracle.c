/*
 * oracle.c -- plain, slow, single-threaded CPU restatement of the mixed-precision
 * ILU(0)-preconditioned multi-component Krylov path (Kouya, "Assessing the Performance of
 * Mixed-Precision ILU(0)-Preconditioned Multiple-Precision Real and Complex Krylov Subspace
 * Methods", arXiv 2504.14498).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load this library.  The CUDA library never links, includes or calls it, and
 * the two share no code.
 *
 * What follows which passage:
 *   number formats D / DD / TD / QD ........ Sec. 2 (binary64 with 1, 2, 3, 4 components)
 *   mixed SpMV (binary64 matrix, MP vector) Sec. 3, last paragraph; Sec. 4 ("_d" variants)
 *   MP-matrix SpMV (matrix promoted to MP) . Sec. 4 (the rows without "_d": matrix in the same
 *                                             multi-component type as the vectors)
 *   ILU(0) in MP (orc_ilu0_mp) .............. Algorithm 1 in the working precision (Sec. 4, the
 *                                             rows without "_d")
 *   ILU(0) .................................. Algorithm 1 (KIJ form, no fill)
 *   forward / backward substitution ......... Algorithm 2
 *   preconditioned BiCG ..................... Algorithm 3
 *   CGS, BiCGSTAB, GPBiCG ................... named in Sec. 3 without a listing; written in the
 *                                             standard right-preconditioned forms (Sonneveld
 *                                             1989; van der Vorst 1992; Zhang 1997)
 *   stopping rule ||r|| < eps_r ||r0|| + eps_a  Algorithm 3 and Sec. 4
 *   inner products <a,b> = sum conj(a_i) b_i  Algorithm 3, summed left to right (the paper gives
 *                                             no order; this is the plain definition)
 *
 * Arithmetic definitions used here (the paper does not say which variants its library uses):
 *   DD  : Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic building blocks
 *         of double-word arithmetic", ACM TOMS 44(2), 2017 -- Alg. 6 (accurate DW+DW),
 *         Alg. 7 (DW*FP, used inside Alg. 17), Alg. 9 (DW*FP with FMA), Alg. 12 (DW*DW with
 *         FMA), Alg. 15 (DW/FP), Alg. 17 (DW/DW); square root by one Newton correction.
 *   TD, QD : every operation is evaluated exactly with Shewchuk's nonoverlapping expansions
 *         (Grow-Expansion with zero elimination, Compress; DCG 18(3), 1997) and the exact value
 *         is then rounded greedily to w components (c_k = leading part of the remainder).
 *         Division uses w+1 steps of long division with exact remainders; square root uses
 *         Newton's iteration in w-component arithmetic.
 *   D   : plain binary64, one rounding per operation (no fused multiply-add).
 * Built with -ffp-contract=off so that every a*b+c written below is two roundings unless
 * fma() is called explicitly.
 *
 * Paper-like "_p" build (the paper's 32-thread OpenMP rows, Sec. 4): compiled once more with
 * -fopenmp into liboracle_p.so, the SpMV, the vector updates and the inner products run on all
 * host threads (static row ranges).  Each row and each entry is computed as above; an inner
 * product is summed left to right within each thread's contiguous range, and the thread sums
 * are added in thread order.  ILU(0) and the substitutions stay sequential, as in the paper.
 * The plain build (no -fopenmp) ignores the pragmas: it is the oracle the tests use.
 *
 * Layout: an MP real number is w doubles (leading component first); a complex one is 2w
 * doubles (real part, then imaginary part).  A vector of n entries is n*c*w doubles, c = 1
 * (real) or 2 (complex).  Matrices are CSR with int32 row pointers and column indices and
 * binary64 values (interleaved re,im when complex).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_MAXIT 1
#define ORC_BREAKDOWN 2
#define ORC_ZERO_PIVOT 3
#define ORC_MISSING_DIAG 4
#define ORC_NAN 5
#define ORC_INVALID 6

/* ------------------------------------------------------------------------------------------
 * Error-free transformations (Knuth TwoSum, Dekker Fast2Sum, FMA-based TwoProd)
 * ---------------------------------------------------------------------------------------- */
static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  double db = b - bv;
  double da = a - av;
  *s = x;
  *e = da + db;
}
static inline void fast_two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *s = x;
  *e = b - z;
}
static inline void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

void orc_two_sum(double a, double b, double *out) { two_sum(a, b, &out[0], &out[1]); }
/* Threads of the "_p" build (no effect in the plain build); returns the count in use. */
int orc_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
  return omp_get_max_threads();
#else
  (void)k;
  return 1;
#endif
}
void orc_two_prod(double a, double b, double *out) { two_prod(a, b, &out[0], &out[1]); }

/* ------------------------------------------------------------------------------------------
 * Double-word (DD) arithmetic, Joldes-Muller-Popescu 2017
 * ---------------------------------------------------------------------------------------- */
typedef struct { double c[4]; } mp; /* components c[0] (leading) .. c[w-1] */

static mp dd_add(mp x, mp y) { /* Alg. 6, relative error <= 3u^2 + 13u^3 */
  double sh, sl, th, tl, c, vh, vl, w;
  mp z = {{0, 0, 0, 0}};
  two_sum(x.c[0], y.c[0], &sh, &sl);
  two_sum(x.c[1], y.c[1], &th, &tl);
  c = sl + th;
  fast_two_sum(sh, c, &vh, &vl);
  w = tl + vl;
  fast_two_sum(vh, w, &z.c[0], &z.c[1]);
  return z;
}
static mp dd_mul_d(mp x, double y) { /* Alg. 9, relative error <= 2u^2 */
  double ch, cl1, cl3;
  mp z = {{0, 0, 0, 0}};
  two_prod(x.c[0], y, &ch, &cl1);
  cl3 = fma(x.c[1], y, cl1);
  fast_two_sum(ch, cl3, &z.c[0], &z.c[1]);
  return z;
}
static mp dd_mul_d_alg7(mp x, double y) { /* Alg. 7, relative error <= 3/2 u^2 + 4u^3 */
  double ch, cl1, cl2, th, tl1, tl2;
  mp z = {{0, 0, 0, 0}};
  two_prod(x.c[0], y, &ch, &cl1);
  cl2 = x.c[1] * y;
  fast_two_sum(ch, cl2, &th, &tl1);
  tl2 = tl1 + cl1;
  fast_two_sum(th, tl2, &z.c[0], &z.c[1]);
  return z;
}
static mp dd_mul(mp x, mp y) { /* Alg. 12, relative error <= 5u^2 */
  double ch, cl1, tl0, tl1, cl2, cl3;
  mp z = {{0, 0, 0, 0}};
  two_prod(x.c[0], y.c[0], &ch, &cl1);
  tl0 = x.c[1] * y.c[1];
  tl1 = fma(x.c[0], y.c[1], tl0);
  cl2 = fma(x.c[1], y.c[0], tl1);
  cl3 = cl1 + cl2;
  fast_two_sum(ch, cl3, &z.c[0], &z.c[1]);
  return z;
}
static mp dd_div_d(mp x, double y) { /* Alg. 15, relative error <= 3u^2 */
  double th, ph, pl, dh, dt, d, tl;
  mp z = {{0, 0, 0, 0}};
  th = x.c[0] / y;
  two_prod(th, y, &ph, &pl);
  dh = x.c[0] - ph;
  dt = dh - pl;
  d = dt + x.c[1];
  tl = d / y;
  fast_two_sum(th, tl, &z.c[0], &z.c[1]);
  return z;
}
static mp dd_div(mp x, mp y) { /* Alg. 17, relative error <= 15u^2 + 56u^3 */
  double th, ph, dl, d, tl;
  mp r, z = {{0, 0, 0, 0}};
  th = x.c[0] / y.c[0];
  r = dd_mul_d_alg7(y, th);
  ph = x.c[0] - r.c[0];
  dl = x.c[1] - r.c[1];
  d = ph + dl;
  tl = d / y.c[0];
  fast_two_sum(th, tl, &z.c[0], &z.c[1]);
  return z;
}
static mp dd_sqrt(mp x) { /* s = sqrt(xh), one Newton correction (x - s^2)/(2s) */
  double s, d, t;
  mp z = {{0, 0, 0, 0}};
  if (x.c[0] <= 0.0) { z.c[0] = sqrt(x.c[0]); return z; }
  s = sqrt(x.c[0]);
  d = fma(-s, s, x.c[0]); /* exact: xh - s^2 */
  d = d + x.c[1];
  t = d / (2.0 * s);
  fast_two_sum(s, t, &z.c[0], &z.c[1]);
  return z;
}

/* ------------------------------------------------------------------------------------------
 * Exact expansion arithmetic for TD / QD (Shewchuk 1997)
 * An expansion holds nonoverlapping doubles in increasing magnitude, without zeros.
 * ---------------------------------------------------------------------------------------- */
#define EXP_MAX 256
typedef struct { int m; double e[EXP_MAX]; } expn;

/* Grow-Expansion with zero elimination: x := x + b exactly. */
static void expn_add_d(expn *x, double b) {
  double q = b, h;
  int k = 0, i;
  for (i = 0; i < x->m; ++i) {
    two_sum(q, x->e[i], &q, &h);
    if (h != 0.0) x->e[k++] = h;
  }
  if (q != 0.0 || k == 0) x->e[k++] = q;
  x->m = k;
  if (x->m == 1 && x->e[0] == 0.0) x->m = 0;
}
/* Leading component of Shewchuk's Compress: approximates the sum within one ulp. */
static double expn_top(const expn *x) {
  double g[EXP_MAX], q, qq;
  int m = x->m, bottom, i;
  if (m == 0) return 0.0;
  q = x->e[m - 1];
  bottom = m - 1;
  for (i = m - 2; i >= 0; --i) {
    fast_two_sum(q, x->e[i], &q, &qq);
    if (qq != 0.0) { g[bottom--] = q; q = qq; }
  }
  g[bottom] = q;
  for (i = bottom + 1; i < m; ++i) {
    fast_two_sum(g[i], q, &q, &qq);
  }
  return q;
}
/* Greedy rounding of the exact value to w components: c_k = top(x - c_0 - ... - c_{k-1}). */
static mp expn_round(expn x, int w) {
  mp z = {{0, 0, 0, 0}};
  int k;
  for (k = 0; k < w; ++k) {
    double t = expn_top(&x);
    z.c[k] = t;
    if (t == 0.0) break;
    expn_add_d(&x, -t);
  }
  return z;
}
static mp ex_add(mp a, mp b, int w) {
  expn x;
  int k;
  x.m = 0;
  for (k = 0; k < w; ++k) { expn_add_d(&x, a.c[k]); expn_add_d(&x, b.c[k]); }
  return expn_round(x, w);
}
static mp ex_mul_d(mp a, double d, int w) {
  expn x;
  int k;
  double p, e;
  x.m = 0;
  for (k = 0; k < w; ++k) { two_prod(a.c[k], d, &p, &e); expn_add_d(&x, p); expn_add_d(&x, e); }
  return expn_round(x, w);
}
static mp ex_mul(mp a, mp b, int w) {
  expn x;
  int i, j;
  double p, e;
  x.m = 0;
  for (i = 0; i < w; ++i)
    for (j = 0; j < w; ++j) { two_prod(a.c[i], b.c[j], &p, &e); expn_add_d(&x, p); expn_add_d(&x, e); }
  return expn_round(x, w);
}
/* Long division: w+1 quotient digits, each q_k = top(remainder)/b_0, remainder updated exactly. */
static mp ex_div(mp a, mp b, int w) {
  expn rem, quo;
  int k, i;
  double p, e, q;
  rem.m = 0;
  quo.m = 0;
  for (i = 0; i < w; ++i) expn_add_d(&rem, a.c[i]);
  for (k = 0; k <= w; ++k) {
    q = expn_top(&rem) / b.c[0];
    if (q == 0.0 || !isfinite(q)) { if (!isfinite(q)) expn_add_d(&quo, q); break; }
    expn_add_d(&quo, q);
    for (i = 0; i < w; ++i) { two_prod(q, b.c[i], &p, &e); expn_add_d(&rem, -p); expn_add_d(&rem, -e); }
  }
  return expn_round(quo, w);
}

/* ------------------------------------------------------------------------------------------
 * Generic real MP operations dispatching on w
 * ---------------------------------------------------------------------------------------- */
static mp mp_zero(void) { mp z = {{0, 0, 0, 0}}; return z; }
static mp mp_from_d(double d) { mp z = {{d, 0, 0, 0}}; return z; }
static mp mp_neg(mp a) { mp z = {{-a.c[0], -a.c[1], -a.c[2], -a.c[3]}}; return z; }

static mp mp_add(mp a, mp b, int w) {
  if (w == 1) return mp_from_d(a.c[0] + b.c[0]);
  if (w == 2) return dd_add(a, b);
  return ex_add(a, b, w);
}
static mp mp_sub(mp a, mp b, int w) { return mp_add(a, mp_neg(b), w); }
static mp mp_mul(mp a, mp b, int w) {
  if (w == 1) return mp_from_d(a.c[0] * b.c[0]);
  if (w == 2) return dd_mul(a, b);
  return ex_mul(a, b, w);
}
static mp mp_mul_d(mp a, double d, int w) {
  if (w == 1) return mp_from_d(a.c[0] * d);
  if (w == 2) return dd_mul_d(a, d);
  return ex_mul_d(a, d, w);
}
static mp mp_div(mp a, mp b, int w) {
  if (w == 1) return mp_from_d(a.c[0] / b.c[0]);
  if (w == 2) return dd_div(a, b);
  return ex_div(a, b, w);
}
static mp mp_div_d(mp a, double d, int w) {
  if (w == 1) return mp_from_d(a.c[0] / d);
  if (w == 2) return dd_div_d(a, d);
  return ex_div(a, mp_from_d(d), w);
}
static mp mp_sqrt(mp a, int w) {
  mp s, two_s, d;
  int it;
  if (w == 1) return mp_from_d(sqrt(a.c[0]));
  if (w == 2) return dd_sqrt(a);
  if (a.c[0] <= 0.0) return mp_from_d(sqrt(a.c[0]));
  s = mp_from_d(sqrt(a.c[0]));
  for (it = 0; it < 3; ++it) { /* 53 -> 106 -> 212 -> 424 bits */
    d = mp_sub(a, mp_mul(s, s, w), w);
    two_s = mp_mul_d(s, 2.0, w);
    s = mp_add(s, mp_div(d, two_s, w), w);
  }
  return s;
}

/* Exposed scalar entry points (used by the exactness pins). */
static mp load_mp(const double *p, int w) { mp z = {{0, 0, 0, 0}}; int k; for (k = 0; k < w; ++k) z.c[k] = p[k]; return z; }
static void store_mp(double *p, mp z, int w) { int k; for (k = 0; k < w; ++k) p[k] = z.c[k]; }

void orc_mp_op(int op, int w, const double *a, const double *b, double *out) {
  mp x = load_mp(a, w), y = load_mp(b, w), z;
  switch (op) {
    case 0: z = mp_add(x, y, w); break;
    case 1: z = mp_sub(x, y, w); break;
    case 2: z = mp_mul(x, y, w); break;
    case 3: z = mp_mul_d(x, b[0], w); break;
    case 4: z = mp_div(x, y, w); break;
    case 5: z = mp_div_d(x, b[0], w); break;
    case 6: z = mp_sqrt(x, w); break;
    default: z = mp_zero();
  }
  store_mp(out, z, w);
}

/* ------------------------------------------------------------------------------------------
 * Numbers: real (c = 1) or complex (c = 2) over MP reals.  Fixed operation orders:
 *   (a+bi)(c+di)      = (ac - bd) + (ad + bc)i
 *   conj(a+bi)(c+di)  = (ac + bd) + (ad - bc)i
 *   (a+bi)/(c+di)     = ((ac + bd) + (bc - ad)i) / (cc + dd), after scaling a, b, c, d by the
 *                       power of two 2^-e that brings max(|c|,|d|) (leading parts) into [0.5, 1)
 * ---------------------------------------------------------------------------------------- */
typedef struct { mp re, im; } num;
typedef struct { int w, c, mm; } ctx; /* mm: matrix entries promoted to w components */

static num n_zero(void) { num z; z.re = mp_zero(); z.im = mp_zero(); return z; }
static num n_load(const double *p, ctx t) {
  num z = n_zero();
  z.re = load_mp(p, t.w);
  if (t.c == 2) z.im = load_mp(p + t.w, t.w);
  return z;
}
static void n_store(double *p, num z, ctx t) {
  store_mp(p, z.re, t.w);
  if (t.c == 2) store_mp(p + t.w, z.im, t.w);
}
static num n_add(num a, num b, ctx t) {
  num z = n_zero();
  z.re = mp_add(a.re, b.re, t.w);
  if (t.c == 2) z.im = mp_add(a.im, b.im, t.w);
  return z;
}
static num n_sub(num a, num b, ctx t) {
  num z = n_zero();
  z.re = mp_sub(a.re, b.re, t.w);
  if (t.c == 2) z.im = mp_sub(a.im, b.im, t.w);
  return z;
}
static num n_neg(num a) { num z; z.re = mp_neg(a.re); z.im = mp_neg(a.im); return z; }
static num n_conj(num a) { num z = a; z.im = mp_neg(a.im); return z; }
static num n_mul(num a, num b, ctx t) {
  num z = n_zero();
  if (t.c == 1) { z.re = mp_mul(a.re, b.re, t.w); return z; }
  z.re = mp_sub(mp_mul(a.re, b.re, t.w), mp_mul(a.im, b.im, t.w), t.w);
  z.im = mp_add(mp_mul(a.re, b.im, t.w), mp_mul(a.im, b.re, t.w), t.w);
  return z;
}
static num n_mul_conj(num a, num b, ctx t) { /* conj(a) * b */
  num z = n_zero();
  if (t.c == 1) { z.re = mp_mul(a.re, b.re, t.w); return z; }
  z.re = mp_add(mp_mul(a.re, b.re, t.w), mp_mul(a.im, b.im, t.w), t.w);
  z.im = mp_sub(mp_mul(a.re, b.im, t.w), mp_mul(a.im, b.re, t.w), t.w);
  return z;
}
static mp mp_ldexp(mp a, int e) { mp z; int k; for (k = 0; k < 4; ++k) z.c[k] = ldexp(a.c[k], e); return z; }
static num n_div(num a, num b, ctx t) {
  num z = n_zero();
  mp den, nr, ni;
  double m;
  int e = 0;
  if (t.c == 1) { z.re = mp_div(a.re, b.re, t.w); return z; }
  /* both operands are first scaled by 2^-e (exact), e = frexp exponent of the larger leading
   * part of b, so that forming |b|^2 neither underflows nor overflows */
  m = fmax(fabs(b.re.c[0]), fabs(b.im.c[0]));
  if (m > 0.0 && isfinite(m)) {
    frexp(m, &e);
    a.re = mp_ldexp(a.re, -e); a.im = mp_ldexp(a.im, -e);
    b.re = mp_ldexp(b.re, -e); b.im = mp_ldexp(b.im, -e);
  }
  den = mp_add(mp_mul(b.re, b.re, t.w), mp_mul(b.im, b.im, t.w), t.w);
  nr = mp_add(mp_mul(a.re, b.re, t.w), mp_mul(a.im, b.im, t.w), t.w);
  ni = mp_sub(mp_mul(a.im, b.re, t.w), mp_mul(a.re, b.im, t.w), t.w);
  z.re = mp_div(nr, den, t.w);
  z.im = mp_div(ni, den, t.w);
  return z;
}
/* x * (fr + fi i) with a binary64 (complex) factor */
static num n_mul_d(num x, double fr, double fi, ctx t) {
  num z = n_zero();
  if (t.c == 1) { z.re = mp_mul_d(x.re, fr, t.w); return z; }
  z.re = mp_sub(mp_mul_d(x.re, fr, t.w), mp_mul_d(x.im, fi, t.w), t.w);
  z.im = mp_add(mp_mul_d(x.im, fr, t.w), mp_mul_d(x.re, fi, t.w), t.w);
  return z;
}
/* x / (fr + fi i) with a binary64 (complex) divisor */
static num n_div_d(num x, double fr, double fi, ctx t) {
  num z = n_zero();
  mp den, nr, ni;
  if (t.c == 1) { z.re = mp_div_d(x.re, fr, t.w); return z; }
  den = mp_add(mp_mul_d(mp_from_d(fr), fr, t.w), mp_mul_d(mp_from_d(fi), fi, t.w), t.w);
  nr = mp_add(mp_mul_d(x.re, fr, t.w), mp_mul_d(x.im, fi, t.w), t.w);
  ni = mp_sub(mp_mul_d(x.im, fr, t.w), mp_mul_d(x.re, fi, t.w), t.w);
  z.re = mp_div(nr, den, t.w);
  z.im = mp_div(ni, den, t.w);
  return z;
}
static int n_is_zero(num a) { return a.re.c[0] == 0.0 && a.im.c[0] == 0.0; }

/* ------------------------------------------------------------------------------------------
 * Vector kernels: mixed SpMV y = A x (binary64 matrix, MP vector; CSR order, starting from 0; a
 * real D row accumulates each entry with one fused multiply-add, acc := fma(a_ij, x_j, acc)),
 * inner product <a,b> = sum conj(a_i) b_i (sequential), 2-norm = sqrt(Re <r,r>).
 * With t.mm the matrix entry is first promoted to a w-component number (a, 0, ..., 0) -- the
 * value is unchanged, the paper's matrices being binary64 -- and the product is the format's
 * full multiplication with the matrix entry first: the SpMV of the rows without "_d".
 * ---------------------------------------------------------------------------------------- */
static void spmv(int n, const int *rp, const int *ci, const double *val, ctx t, const double *x, double *y) {
  int s = t.c * t.w, i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (i = 0; i < n; ++i) {
    int p;
    num acc = n_zero();
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      num xj = n_load(x + (size_t)ci[p] * s, t);
      double ar = t.c == 2 ? val[2 * (size_t)p] : val[p];
      double ai = t.c == 2 ? val[2 * (size_t)p + 1] : 0.0;
      if (t.w == 1 && t.c == 1) {
        acc.re.c[0] = fma(ar, xj.re.c[0], acc.re.c[0]); /* D, real: one fused multiply-add per entry */
      } else if (t.mm) {
        num a = n_zero();
        a.re.c[0] = ar;
        a.im.c[0] = ai;
        acc = n_add(acc, n_mul(a, xj, t), t);
      } else {
        acc = n_add(acc, n_mul_d(xj, ar, ai, t), t);
      }
    }
    n_store(y + (size_t)i * s, acc, t);
  }
}
void orc_spmv(int n, const int *rp, const int *ci, const double *val, int c, int w, const double *x, double *y) {
  ctx t = {w, c, 0};
  spmv(n, rp, ci, val, t, x, y);
}
void orc_spmv_mm(int n, const int *rp, const int *ci, const double *val, int c, int w, const double *x, double *y) {
  ctx t = {w, c, 1};
  spmv(n, rp, ci, val, t, x, y);
}
/* Inner product <a,b> = sum_i conj(a_i) b_i (Algorithm 3), accumulated left to right from 0
 * in the working format: acc := acc + conj(a_i) b_i for i = 0, 1, ..., n-1.  The paper gives
 * no summation order; this is the plain definition. */
static num dot(int n, ctx t, const double *a, const double *b) {
  int s = t.c * t.w, i;
  num acc = n_zero();
#ifdef _OPENMP
  if (omp_get_max_threads() > 1 && n >= 4096) { /* "_p" build: per-thread ranges, sums in thread order */
    int nth = omp_get_max_threads(), k;
    num *part = (num *)malloc(sizeof(num) * (size_t)nth);
#pragma omp parallel num_threads(nth)
    {
      int tid = omp_get_thread_num(), j;
      int lo = (int)((long long)n * tid / nth), hi = (int)((long long)n * (tid + 1) / nth);
      num pa = n_zero();
      for (j = lo; j < hi; ++j) pa = n_add(pa, n_mul_conj(n_load(a + (size_t)j * s, t), n_load(b + (size_t)j * s, t), t), t);
      part[tid] = pa;
    }
    for (k = 0; k < nth; ++k) acc = n_add(acc, part[k], t);
    free(part);
    return acc;
  }
#endif
  for (i = 0; i < n; ++i) acc = n_add(acc, n_mul_conj(n_load(a + (size_t)i * s, t), n_load(b + (size_t)i * s, t), t), t);
  return acc;
}
void orc_dot(int n, int c, int w, const double *a, const double *b, double *out) {
  ctx t = {w, c, 0};
  n_store(out, dot(n, t, a, b), t);
}
static mp nrm2(int n, ctx t, const double *a) { return mp_sqrt(dot(n, t, a, a).re, t.w); }

/* ------------------------------------------------------------------------------------------
 * ILU(0), Algorithm 1 in its KIJ order.  "A_ij != 0" is read as membership of (i,j) in the
 * stored pattern of A.  A zero pivot U_kk is reported (the listing silently skips it, which
 * later divides by zero in Algorithm 2).  The update A_ij := A_ij - L_ik U_kj is one fused
 * multiply-add.  prec 0: binary64; 1: binary32 (A rounded to nearest binary32 first);
 * 2: binary32 computation, every factor entry then rounded to nearest-even bfloat16.
 * The factor is returned on A's pattern (strict lower part = L~ without its unit diagonal,
 * upper part with diagonal = U~), widened to double.
 * Complex scalar steps, in binary64 or binary32:
 *   division  x/y : den = fma(yr,yr,yi*yi); nr = fma(xr,yr,xi*yi); ni = fma(xi,yr,-(xr*yi));
 *                   result (nr/den, ni/den)
 *   update a -= l*u : re = fma(-lr,ur,ar); re = fma(li,ui,re); im = fma(-lr,ui,ai); im = fma(-li,ur,im)
 * ---------------------------------------------------------------------------------------- */
static int find_col(const int *ci, int lo, int hi, int col) {
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (ci[mid] < col) lo = mid + 1; else hi = mid;
  }
  return lo;
}
static float bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) { u |= 0x00400000u; } /* quiet NaN */
  else { u += 0x7fffu + ((u >> 16) & 1u); }
  u &= 0xffff0000u;
  memcpy(&f, &u, 4);
  return f;
}

int orc_check_pattern(int n, const int *rp, const int *ci, int *diag, int *fail_row) {
  int i, p;
  for (i = 0; i < n; ++i) {
    int d = -1;
    if (rp[i + 1] < rp[i]) { *fail_row = i; return ORC_INVALID; }
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n) { *fail_row = i; return ORC_INVALID; }
      if (p > rp[i] && ci[p] <= ci[p - 1]) { *fail_row = i; return ORC_INVALID; }
      if (ci[p] == i) d = p;
    }
    if (d < 0) { *fail_row = i; return ORC_MISSING_DIAG; }
    if (diag) diag[i] = d;
  }
  return ORC_OK;
}

int orc_ilu0(int n, const int *rp, const int *ci, const double *val, int c, int prec, double *fac, int *fail_row) {
  int nnz = rp[n], i, k, p, q, st;
  int *diag = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
  int *cptr = (int *)calloc((size_t)n + 1, sizeof(int));
  int *crow = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  int *cpos = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  double *ad = NULL;
  float *af = NULL;
  *fail_row = -1;
  st = orc_check_pattern(n, rp, ci, diag, fail_row);
  if (st != ORC_OK) goto done;
  /* column lists of the strictly lower part (rows ascending), i.e. { i > k : (i,k) in pattern } */
  for (i = 0; i < n; ++i)
    for (p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] < i) cnt[ci[p]]++;
  for (k = 0; k < n; ++k) cptr[k + 1] = cptr[k] + cnt[k];
  memset(cnt, 0, sizeof(int) * (size_t)n);
  for (i = 0; i < n; ++i)
    for (p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] < i) { int k2 = ci[p]; crow[cptr[k2] + cnt[k2]] = i; cpos[cptr[k2] + cnt[k2]] = p; cnt[k2]++; }
  if (prec == 0) {
    ad = (double *)malloc(sizeof(double) * (size_t)nnz * c + 1);
    memcpy(ad, val, sizeof(double) * (size_t)nnz * c);
  } else {
    af = (float *)malloc(sizeof(float) * (size_t)nnz * c + 1);
    for (p = 0; p < nnz * c; ++p) af[p] = (float)val[p];
  }
  for (k = 0; k < n; ++k) {
    int dk = diag[k], e;
    /* pivot U_kk := A_kk (already updated by the earlier steps) */
    if (prec == 0) {
      if (ad[(size_t)dk * c] == 0.0 && (c == 1 || ad[(size_t)dk * c + 1] == 0.0)) { *fail_row = k; st = ORC_ZERO_PIVOT; goto done; }
    } else {
      if (af[(size_t)dk * c] == 0.0f && (c == 1 || af[(size_t)dk * c + 1] == 0.0f)) { *fail_row = k; st = ORC_ZERO_PIVOT; goto done; }
    }
    for (e = cptr[k]; e < cptr[k + 1]; ++e) {
      int ii = crow[e], pik = cpos[e];
      /* L_ik := A_ik / U_kk */
      if (prec == 0) {
        if (c == 1) ad[pik] = ad[pik] / ad[dk];
        else {
          double xr = ad[2 * (size_t)pik], xi = ad[2 * (size_t)pik + 1], yr = ad[2 * (size_t)dk], yi = ad[2 * (size_t)dk + 1];
          double den = fma(yr, yr, yi * yi), nr = fma(xr, yr, xi * yi), ni = fma(xi, yr, -(xr * yi));
          ad[2 * (size_t)pik] = nr / den;
          ad[2 * (size_t)pik + 1] = ni / den;
        }
      } else {
        if (c == 1) af[pik] = af[pik] / af[dk];
        else {
          float xr = af[2 * (size_t)pik], xi = af[2 * (size_t)pik + 1], yr = af[2 * (size_t)dk], yi = af[2 * (size_t)dk + 1];
          float den = fmaf(yr, yr, yi * yi), nr = fmaf(xr, yr, xi * yi), ni = fmaf(xi, yr, -(xr * yi));
          af[2 * (size_t)pik] = nr / den;
          af[2 * (size_t)pik + 1] = ni / den;
        }
      }
      /* for each j > k with (k,j) in pattern: if (i,j) in pattern, A_ij := A_ij - L_ik U_kj */
      for (q = dk + 1; q < rp[k + 1]; ++q) {
        int j = ci[q];
        int pij = find_col(ci, rp[ii], rp[ii + 1], j);
        if (pij >= rp[ii + 1] || ci[pij] != j) continue;
        if (prec == 0) {
          if (c == 1) ad[pij] = fma(-ad[pik], ad[q], ad[pij]);
          else {
            double lr = ad[2 * (size_t)pik], li = ad[2 * (size_t)pik + 1], ur = ad[2 * (size_t)q], ui = ad[2 * (size_t)q + 1];
            double re = fma(-lr, ur, ad[2 * (size_t)pij]), im = fma(-lr, ui, ad[2 * (size_t)pij + 1]);
            re = fma(li, ui, re);
            im = fma(-li, ur, im);
            ad[2 * (size_t)pij] = re;
            ad[2 * (size_t)pij + 1] = im;
          }
        } else {
          if (c == 1) af[pij] = fmaf(-af[pik], af[q], af[pij]);
          else {
            float lr = af[2 * (size_t)pik], li = af[2 * (size_t)pik + 1], ur = af[2 * (size_t)q], ui = af[2 * (size_t)q + 1];
            float re = fmaf(-lr, ur, af[2 * (size_t)pij]), im = fmaf(-lr, ui, af[2 * (size_t)pij + 1]);
            re = fmaf(li, ui, re);
            im = fmaf(-li, ur, im);
            af[2 * (size_t)pij] = re;
            af[2 * (size_t)pij + 1] = im;
          }
        }
      }
    }
  }
  for (p = 0; p < nnz * c; ++p) {
    if (prec == 0) fac[p] = ad[p];
    else if (prec == 1) fac[p] = (double)af[p];
    else fac[p] = (double)bf16_round(af[p]);
  }
done:
  free(diag); free(cnt); free(cptr); free(crow); free(cpos); free(ad); free(af);
  return st;
}

/* ILU(0) in the working multi-component precision w (the paper's rows without "_d": factor
 * entries are w-component numbers).  Algorithm 1 in the same KIJ order as orc_ilu0, every step
 * in w-component arithmetic: L_ik := A_ik / U_kk, then A_ij := A_ij - L_ik * U_kj (the product
 * with L_ik as its first operand).  The pivot test reads the leading components.  fac receives
 * nnz * c * w doubles (entry p: real components, then imaginary components). */
int orc_ilu0_mp(int n, const int *rp, const int *ci, const double *val, int c, int w, double *fac, int *fail_row) {
  int nnz = rp[n], i, k, p, q, st;
  ctx t = {w, c, 0};
  int s = c * w;
  int *diag = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
  int *cptr = (int *)calloc((size_t)n + 1, sizeof(int));
  int *crow = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  int *cpos = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  *fail_row = -1;
  st = orc_check_pattern(n, rp, ci, diag, fail_row);
  if (st != ORC_OK) goto done;
  for (i = 0; i < n; ++i)
    for (p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] < i) cnt[ci[p]]++;
  for (k = 0; k < n; ++k) cptr[k + 1] = cptr[k] + cnt[k];
  memset(cnt, 0, sizeof(int) * (size_t)n);
  for (i = 0; i < n; ++i)
    for (p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] < i) { int k2 = ci[p]; crow[cptr[k2] + cnt[k2]] = i; cpos[cptr[k2] + cnt[k2]] = p; cnt[k2]++; }
  memset(fac, 0, sizeof(double) * (size_t)nnz * s);
  for (p = 0; p < nnz; ++p) {
    fac[(size_t)p * s] = c == 2 ? val[2 * (size_t)p] : val[p];
    if (c == 2) fac[(size_t)p * s + w] = val[2 * (size_t)p + 1];
  }
  for (k = 0; k < n; ++k) {
    int dk = diag[k], e;
    num ukk = n_load(fac + (size_t)dk * s, t);
    if (n_is_zero(ukk)) { *fail_row = k; st = ORC_ZERO_PIVOT; goto done; }
    for (e = cptr[k]; e < cptr[k + 1]; ++e) {
      int ii = crow[e], pik = cpos[e];
      num l = n_div(n_load(fac + (size_t)pik * s, t), ukk, t);
      n_store(fac + (size_t)pik * s, l, t);
      for (q = dk + 1; q < rp[k + 1]; ++q) {
        int j = ci[q];
        int pij = find_col(ci, rp[ii], rp[ii + 1], j);
        if (pij >= rp[ii + 1] || ci[pij] != j) continue;
        n_store(fac + (size_t)pij * s,
                n_sub(n_load(fac + (size_t)pij * s, t), n_mul(l, n_load(fac + (size_t)q * s, t), t), t), t);
      }
    }
  }
done:
  free(diag); free(cnt); free(cptr); free(crow); free(cpos);
  return st;
}

/* ------------------------------------------------------------------------------------------
 * Substitutions, Algorithm 2, on CSR patterns (column order ascending within a row).
 * Factor layout as returned by orc_ilu0.  M z = r: forward with unit L~, backward with U~.
 * M^H z = r: U~^H w = r (forward, divide by conj(U_ii)) then L~^H z = w (backward, unit),
 * both evaluated row-wise on the explicitly conjugate-transposed factor.
 *
 * prec 0 ("_d"): binary64 factor entries times MP vector entries, subtracted in MP, divided in MP.
 * prec 3 (full MP, the rows without "_d"): w-component factor entries (orc_ilu0_mp) times MP
 *   vector entries, factor first in every product, divided in MP.
 * prec 1, 2: the MP right-hand side is scaled by 2^-e, e = frexp exponent of the largest
 *   |leading component| (real and imaginary parts), each scaled leading component is rounded
 *   to binary32, both triangles are solved in binary32 (y := fma(-l, y_j, y); division
 *   correctly rounded), and the result is widened and scaled back by 2^e (lower components 0).
 * ---------------------------------------------------------------------------------------- */
typedef struct { int n; int *rp, *ci; double *v; } csr_t; /* v: c doubles per entry */

/* entries of s doubles; the last nneg of them (imaginary components) change sign */
static csr_t csr_conj_transpose_s(int n, const int *rp, const int *ci, const double *v, int s, int nneg) {
  csr_t t;
  int nnz = rp[n], i, p, k;
  int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
  t.n = n;
  t.rp = (int *)calloc((size_t)n + 1, sizeof(int));
  t.ci = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  t.v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1) * s);
  for (p = 0; p < nnz; ++p) cnt[ci[p]]++;
  for (i = 0; i < n; ++i) t.rp[i + 1] = t.rp[i] + cnt[i];
  memset(cnt, 0, sizeof(int) * (size_t)n);
  for (i = 0; i < n; ++i)
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p], dst = t.rp[j] + cnt[j]++;
      t.ci[dst] = i;
      for (k = 0; k < s; ++k) t.v[(size_t)dst * s + k] = k >= s - nneg ? -v[(size_t)p * s + k] : v[(size_t)p * s + k];
    }
  free(cnt);
  return t;
}
static csr_t csr_conj_transpose(int n, const int *rp, const int *ci, const double *v, int c) {
  csr_t t;
  int nnz = rp[n], i, p;
  int *cnt = (int *)calloc((size_t)n + 1, sizeof(int));
  t.n = n;
  t.rp = (int *)calloc((size_t)n + 1, sizeof(int));
  t.ci = (int *)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
  t.v = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1) * c);
  for (p = 0; p < nnz; ++p) cnt[ci[p]]++;
  for (i = 0; i < n; ++i) t.rp[i + 1] = t.rp[i] + cnt[i];
  memset(cnt, 0, sizeof(int) * (size_t)n);
  for (i = 0; i < n; ++i) /* rows ascending => transposed rows get ascending columns */
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p], dst = t.rp[j] + cnt[j]++;
      t.ci[dst] = i;
      if (c == 1) t.v[dst] = v[p];
      else { t.v[2 * (size_t)dst] = v[2 * (size_t)p]; t.v[2 * (size_t)dst + 1] = -v[2 * (size_t)p + 1]; }
    }
  free(cnt);
  return t;
}
static void csr_free(csr_t *t) { free(t->rp); free(t->ci); free(t->v); }

/* Solve with the lower (lower != 0) or upper triangle of the combined factor f; unit != 0 means
 * the diagonal is 1 and is not read, otherwise divide by the stored diagonal. */
static void tri_mp(int n, const int *rp, const int *ci, const double *f, ctx t, int lower, int unit, const double *r, double *z) {
  int s = t.c * t.w, ii, p;
  for (ii = 0; ii < n; ++ii) {
    int i = lower ? ii : n - 1 - ii, pd = -1;
    num acc = n_load(r + (size_t)i * s, t);
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      double fr = t.c == 2 ? f[2 * (size_t)p] : f[p], fi = t.c == 2 ? f[2 * (size_t)p + 1] : 0.0;
      if (j == i) { pd = p; continue; }
      if ((lower && j < i) || (!lower && j > i)) acc = n_sub(acc, n_mul_d(n_load(z + (size_t)j * s, t), fr, fi, t), t);
    }
    if (!unit && pd >= 0) {
      double dr = t.c == 2 ? f[2 * (size_t)pd] : f[pd], di = t.c == 2 ? f[2 * (size_t)pd + 1] : 0.0;
      acc = n_div_d(acc, dr, di, t);
    }
    n_store(z + (size_t)i * s, acc, t);
  }
}
/* The same with w-component factor entries (stride c * w): acc -= f_p * z_j (factor first). */
static void tri_mpf(int n, const int *rp, const int *ci, const double *f, ctx t, int lower, int unit, const double *r, double *z) {
  int s = t.c * t.w, ii, p;
  for (ii = 0; ii < n; ++ii) {
    int i = lower ? ii : n - 1 - ii, pd = -1;
    num acc = n_load(r + (size_t)i * s, t);
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      if (j == i) { pd = p; continue; }
      if ((lower && j < i) || (!lower && j > i))
        acc = n_sub(acc, n_mul(n_load(f + (size_t)p * s, t), n_load(z + (size_t)j * s, t), t), t);
    }
    if (!unit && pd >= 0) acc = n_div(acc, n_load(f + (size_t)pd * s, t), t);
    n_store(z + (size_t)i * s, acc, t);
  }
}
static void tri_f32(int n, const int *rp, const int *ci, const double *f, int c, int lower, int unit, const float *r, float *z) {
  int ii, p;
  for (ii = 0; ii < n; ++ii) {
    int i = lower ? ii : n - 1 - ii, pd = -1;
    float ar = r[(size_t)i * c], ai = c == 2 ? r[(size_t)i * c + 1] : 0.0f;
    for (p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      if (j == i) { pd = p; continue; }
      if (!((lower && j < i) || (!lower && j > i))) continue;
      if (c == 1) ar = fmaf(-(float)f[p], z[j], ar);
      else {
        float lr = (float)f[2 * (size_t)p], li = (float)f[2 * (size_t)p + 1];
        float yr = z[2 * (size_t)j], yi = z[2 * (size_t)j + 1];
        ar = fmaf(-lr, yr, ar); ar = fmaf(li, yi, ar);
        ai = fmaf(-lr, yi, ai); ai = fmaf(-li, yr, ai);
      }
    }
    if (!unit && pd >= 0) {
      if (c == 1) ar = ar / (float)f[pd];
      else {
        float yr = (float)f[2 * (size_t)pd], yi = (float)f[2 * (size_t)pd + 1];
        float den = fmaf(yr, yr, yi * yi), nr = fmaf(ar, yr, ai * yi), ni = fmaf(ai, yr, -(ar * yi));
        ar = nr / den;
        ai = ni / den;
      }
    }
    z[(size_t)i * c] = ar;
    if (c == 2) z[(size_t)i * c + 1] = ai;
  }
}

static void precond_apply(int n, const int *rp, const int *ci, const double *fac, ctx t, int prec, int trans, const double *r, double *z) {
  int s = t.c * t.w, i, k;
  const int *frp = rp, *fci = ci;
  const double *fv = fac;
  csr_t tr;
  int have_tr = 0;
  if (trans) {
    tr = prec == 3 ? csr_conj_transpose_s(n, rp, ci, fac, s, t.c == 2 ? t.w : 0) : csr_conj_transpose(n, rp, ci, fac, t.c);
    have_tr = 1; frp = tr.rp; fci = tr.ci; fv = tr.v;
  }
  /* M: lower unit then upper with division.  M^H: lower with division then upper unit. */
  if (prec == 3) {
    double *y = (double *)malloc(sizeof(double) * (size_t)n * s + 1);
    tri_mpf(n, frp, fci, fv, t, 1, trans ? 0 : 1, r, y);
    tri_mpf(n, frp, fci, fv, t, 0, trans ? 1 : 0, y, z);
    free(y);
  } else if (prec == 0) {
    double *y = (double *)malloc(sizeof(double) * (size_t)n * s + 1);
    tri_mp(n, frp, fci, fv, t, 1, trans ? 0 : 1, r, y);
    tri_mp(n, frp, fci, fv, t, 0, trans ? 1 : 0, y, z);
    free(y);
  } else {
    double mx = 0.0;
    int e = 0;
    float *r32 = (float *)calloc((size_t)n * t.c + 1, sizeof(float));
    float *y32 = (float *)malloc(sizeof(float) * (size_t)n * t.c + 1);
    float *z32 = (float *)malloc(sizeof(float) * (size_t)n * t.c + 1);
    for (i = 0; i < n; ++i)
      for (k = 0; k < t.c; ++k) { double a = fabs(r[(size_t)i * s + (size_t)k * t.w]); if (a > mx) mx = a; }
    if (mx > 0.0) frexp(mx, &e);
    for (i = 0; i < n; ++i)
      for (k = 0; k < t.c; ++k) r32[(size_t)i * t.c + k] = (float)ldexp(r[(size_t)i * s + (size_t)k * t.w], -e);
    tri_f32(n, frp, fci, fv, t.c, 1, trans ? 0 : 1, r32, y32);
    tri_f32(n, frp, fci, fv, t.c, 0, trans ? 1 : 0, y32, z32);
    for (i = 0; i < n; ++i)
      for (k = 0; k < t.c; ++k) {
        double *dst = z + (size_t)i * s + (size_t)k * t.w;
        int q;
        dst[0] = ldexp((double)z32[(size_t)i * t.c + k], e);
        for (q = 1; q < t.w; ++q) dst[q] = 0.0;
      }
    free(r32); free(y32); free(z32);
  }
  if (have_tr) csr_free(&tr);
}
void orc_precond(int n, const int *rp, const int *ci, const double *fac, int c, int w, int prec, int trans, const double *r, double *z) {
  ctx t = {w, c, 0};
  precond_apply(n, rp, ci, fac, t, prec, trans, r, z);
}

/* ------------------------------------------------------------------------------------------
 * Krylov methods.  ilu < 0: no preconditioner (M = I).  r is always the unpreconditioned
 * residual b - A x, so the stopping rule of Algorithm 3 tests the original system; it compares
 * leading components: ||r||_0 < eps_r ||r0||_0 + eps_a.  The shadow residual is r~ = r0.
 * Breakdown: an exactly zero denominator (rho, <r~,v>, <t,t> with t != 0, LS determinant, zeta).
 * hist[k] = leading component of ||r_k||, k = 0..iters.
 *
 * Residual replacement (the paper recomputes nothing; this is the periodic true residual that the
 * stated method adds).  With a period P > 0, after the stopping test of iteration k, whenever k is
 * a multiple of P or the recursive norm passed the test, the true residual b - A x_k is formed in
 * the working format exactly as r0 was (SpMV, then b + (-1) * (A x)) and its norm taken.  If that
 * norm is above 10 (eps_r ||r0|| + eps_a), r is replaced by the true residual and a passed test is
 * withdrawn (the iteration goes on from the replaced r); otherwise nothing changes and a passed
 * test stands.  hist_true[k] (if given) receives the leading component of ||b - A x_k|| at every
 * such check; *nrep counts the replacements.  P = 0: no check, the test on the recursive r alone.
 * ---------------------------------------------------------------------------------------- */
enum { M_BICG = 0, M_CGS = 1, M_BICGSTAB = 2, M_GPBICG = 3 };

typedef struct {
  int n; const int *rp, *ci; const double *val; ctx t; int ilu; const double *fac;
  csr_t ah; int have_ah;
} sys_t;

static double *vnew(const sys_t *S) { return (double *)calloc((size_t)S->n * S->t.c * S->t.w + 1, sizeof(double)); }
static void vcopy(const sys_t *S, double *dst, const double *src) { memcpy(dst, src, sizeof(double) * (size_t)S->n * S->t.c * S->t.w); }
static void apply_m(const sys_t *S, int trans, const double *r, double *z) {
  if (S->ilu < 0) vcopy(S, z, r);
  else precond_apply(S->n, S->rp, S->ci, S->fac, S->t, S->ilu, trans, r, z);
}
/* y := a + alpha * b  (alpha multiplies the vector entry from the left: alpha * b_i) */
static void vaxpy(const sys_t *S, double *y, const double *a, num alpha, const double *b) {
  int s = S->t.c * S->t.w, i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (i = 0; i < S->n; ++i) {
    num v = n_add(n_load(a + (size_t)i * s, S->t), n_mul(alpha, n_load(b + (size_t)i * s, S->t), S->t), S->t);
    n_store(y + (size_t)i * s, v, S->t);
  }
}
static int nan_mp(mp a) { return a.c[0] != a.c[0]; }

/* The stopping decision of iteration it with the residual replacement described above; returns
 * 1 when the solve stops with OK.  rtrue: scratch vector. */
typedef struct { int period; double *hist_true; int nrep; } repl_t;
static int stop_check(const sys_t *S, repl_t *R, const double *b, const double *x, double *r, double *rtrue,
                      double nrec, double tol, int it) {
  int cand = nrec < tol;
  mp nt;
  if (R->period <= 0) return cand;
  if (!cand && it % R->period != 0) return 0;
  spmv(S->n, S->rp, S->ci, S->val, S->t, x, rtrue);
  vaxpy(S, rtrue, b, n_neg((num){mp_from_d(1.0), mp_zero()}), rtrue); /* b - A x */
  nt = nrm2(S->n, S->t, rtrue);
  if (R->hist_true) R->hist_true[it] = nt.c[0];
  if (nt.c[0] > 10.0 * tol) {
    vcopy(S, r, rtrue);
    R->nrep++;
    return 0;
  }
  return cand;
}

/* Test hooks (set by orc_krylov_hooks around one call, NULL otherwise):
 *   g_shadow: the initial shadow residual r~0 instead of r0 (n*c*w doubles);
 *   g_trace:  per iteration k (1-based), the moduli of normalised inner products that exact
 *             arithmetic makes zero (leading components): BiCGSTAB |<t, r_k>| / (|t| |r_k|) and
 *             0; GPBiCG |<c, r_k>| / (|c| |r_k|) and |<y, r_k>| / (|y| |r_k|) (y from the second
 *             step).  For complex systems the modulus covers the imaginary part as well.
 *             2 * (maxit + 1) doubles. */
static const double *g_shadow = NULL;
static double *g_trace = NULL;
static double ortho(int n, ctx t, const double *a, const double *b) {
  num ab = dot(n, t, a, b);
  mp aa = nrm2(n, t, a), bb = nrm2(n, t, b);
  double den = aa.c[0] * bb.c[0];
  return den > 0.0 ? hypot(ab.re.c[0], ab.im.c[0]) / den : 0.0;
}

int orc_krylov(int method, int n, const int *rp, const int *ci, const double *val, int c, int w, int ilu,
               const double *fac, const double *b, double *x, double tol_rel, double tol_abs, int maxit, int flags,
               double *hist, int *iters_out, double *relres_true, int true_res_period, double *hist_true,
               int *nrep_out) {
  sys_t S;
  repl_t R;
  ctx t = {w, c, (flags >> 1) & 1}; /* flags bit 1: every SpMV with the matrix promoted to MP */
  int s = c * w, it = 0, st = ORC_MAXIT, i;
  double r0n, tol;
  double *r, *rt, *tmp, *rtrue;
  mp nr;
  memset(&S, 0, sizeof(S));
  S.n = n; S.rp = rp; S.ci = ci; S.val = val; S.t = t; S.ilu = ilu; S.fac = fac;
  R.period = true_res_period; R.hist_true = hist_true; R.nrep = 0;
  r = vnew(&S); rt = vnew(&S); tmp = vnew(&S); rtrue = vnew(&S);
  spmv(n, rp, ci, val, t, x, tmp);
  vaxpy(&S, r, b, n_neg((num){mp_from_d(1.0), mp_zero()}), tmp); /* r = b - A x */
  if (g_shadow) vcopy(&S, rt, g_shadow);
  else vcopy(&S, rt, r);
  nr = nrm2(n, t, r);
  r0n = nr.c[0];
  if (hist) hist[0] = r0n;
  tol = tol_rel * r0n + tol_abs;
  if (nan_mp(nr)) { st = ORC_NAN; goto finish; }
  if (r0n < tol || r0n == 0.0) { st = ORC_OK; goto finish; }

  if (method == M_BICG) {
    double *z = vnew(&S), *zt = vnew(&S), *p = vnew(&S), *pt = vnew(&S), *q = vnew(&S), *qt = vnew(&S);
    num rho, rhon, alpha, beta, sig;
    S.ah = csr_conj_transpose(n, rp, ci, val, c); S.have_ah = 1;
    apply_m(&S, 0, r, z);
    apply_m(&S, 1, rt, zt);
    vcopy(&S, p, z); vcopy(&S, pt, zt);
    rho = dot(n, t, zt, r);
    for (it = 1; it <= maxit; ++it) {
      spmv(n, rp, ci, val, t, p, q);                  /* q = A p */
      spmv(n, S.ah.rp, S.ah.ci, S.ah.v, t, pt, qt);   /* q~ = A^H p~ */
      sig = dot(n, t, pt, q);
      if (n_is_zero(rho) || n_is_zero(sig)) { st = ORC_BREAKDOWN; it--; break; }
      alpha = n_div(rho, sig, t);
      vaxpy(&S, x, x, alpha, p);
      vaxpy(&S, r, r, n_neg(alpha), q);
      vaxpy(&S, rt, rt, n_neg(n_conj(alpha)), qt);
      nr = nrm2(n, t, r);
      if (hist) hist[it] = nr.c[0];
      if (nan_mp(nr)) { st = ORC_NAN; break; }
      if (stop_check(&S, &R, b, x, r, rtrue, nr.c[0], tol, it)) { st = ORC_OK; break; }
      apply_m(&S, 0, r, z);
      apply_m(&S, 1, rt, zt);
      rhon = dot(n, t, zt, r);
      beta = n_div(rhon, rho, t);
      vaxpy(&S, p, z, beta, p);
      vaxpy(&S, pt, zt, n_conj(beta), pt);
      rho = rhon;
    }
    free(z); free(zt); free(p); free(pt); free(q); free(qt);
  } else if (method == M_CGS) {
    double *u = vnew(&S), *p = vnew(&S), *q = vnew(&S), *ph = vnew(&S), *v = vnew(&S), *uh = vnew(&S), *uq = vnew(&S);
    num rho, rho_old = n_zero(), alpha, beta, sig;
    for (it = 1; it <= maxit; ++it) {
      rho = dot(n, t, rt, r);
      if (n_is_zero(rho)) { st = ORC_BREAKDOWN; it--; break; }
      if (it == 1) { vcopy(&S, u, r); vcopy(&S, p, u); }
      else {
        beta = n_div(rho, rho_old, t);
        vaxpy(&S, u, r, beta, q);          /* u = r + beta q */
        vaxpy(&S, tmp, q, beta, p);        /* q + beta p */
        vaxpy(&S, p, u, beta, tmp);        /* p = u + beta (q + beta p) */
      }
      apply_m(&S, 0, p, ph);
      spmv(n, rp, ci, val, t, ph, v);
      sig = dot(n, t, rt, v);
      if (n_is_zero(sig)) { st = ORC_BREAKDOWN; it--; break; }
      alpha = n_div(rho, sig, t);
      vaxpy(&S, q, u, n_neg(alpha), v);    /* q = u - alpha v */
      vaxpy(&S, uq, u, (num){mp_from_d(1.0), mp_zero()}, q); /* u + q */
      apply_m(&S, 0, uq, uh);
      vaxpy(&S, x, x, alpha, uh);
      spmv(n, rp, ci, val, t, uh, tmp);
      vaxpy(&S, r, r, n_neg(alpha), tmp);
      nr = nrm2(n, t, r);
      if (hist) hist[it] = nr.c[0];
      if (nan_mp(nr)) { st = ORC_NAN; break; }
      if (stop_check(&S, &R, b, x, r, rtrue, nr.c[0], tol, it)) { st = ORC_OK; break; }
      rho_old = rho;
    }
    free(u); free(p); free(q); free(ph); free(v); free(uh); free(uq);
  } else if (method == M_BICGSTAB) {
    double *p = vnew(&S), *v = vnew(&S), *ph = vnew(&S), *sv = vnew(&S), *sh = vnew(&S), *tv = vnew(&S);
    num rho, rho_old = n_zero(), alpha = n_zero(), omega = n_zero(), beta, sig, ts, tt;
    for (it = 1; it <= maxit; ++it) {
      rho = dot(n, t, rt, r);
      if (n_is_zero(rho)) { st = ORC_BREAKDOWN; it--; break; }
      if (it == 1) vcopy(&S, p, r);
      else {
        beta = n_mul(n_div(rho, rho_old, t), n_div(alpha, omega, t), t);
        vaxpy(&S, tmp, p, n_neg(omega), v);   /* p - omega v */
        vaxpy(&S, p, r, beta, tmp);            /* p = r + beta (p - omega v) */
      }
      apply_m(&S, 0, p, ph);
      spmv(n, rp, ci, val, t, ph, v);
      sig = dot(n, t, rt, v);
      if (n_is_zero(sig)) { st = ORC_BREAKDOWN; it--; break; }
      alpha = n_div(rho, sig, t);
      vaxpy(&S, sv, r, n_neg(alpha), v);       /* s = r - alpha v */
      apply_m(&S, 0, sv, sh);
      spmv(n, rp, ci, val, t, sh, tv);         /* t = A s^ */
      ts = dot(n, t, tv, sv);
      tt = dot(n, t, tv, tv);
      omega = n_is_zero(tt) ? n_zero() : n_div(ts, tt, t);
      vaxpy(&S, x, x, alpha, ph);
      vaxpy(&S, x, x, omega, sh);
      vaxpy(&S, r, sv, n_neg(omega), tv);      /* r = s - omega t */
      if (g_trace) g_trace[2 * it] = ortho(n, t, tv, r);
      nr = nrm2(n, t, r);
      if (hist) hist[it] = nr.c[0];
      if (nan_mp(nr)) { st = ORC_NAN; break; }
      if (stop_check(&S, &R, b, x, r, rtrue, nr.c[0], tol, it)) { st = ORC_OK; break; }
      if (n_is_zero(omega)) { st = ORC_BREAKDOWN; break; }
      rho_old = rho;
    }
    free(p); free(v); free(ph); free(sv); free(sh); free(tv);
  } else if (method == M_GPBICG) {
    /* Zhang's GPBiCG applied to A M^-1 (right preconditioning), carried in "hat" vectors
     * v^ = M^-1 v so that only r and q are preconditioned:  r^ = M^-1 r, q = A p^,
     * q^ = M^-1 q, t = r - alpha q, t^ = r^ - alpha q^, c = A t^, y = t_prev - t - alpha w,
     * (zeta, eta) = argmin || t - eta y - zeta c || (eta = 0 at the first step),
     * u^ = zeta q^ + eta (t^_prev - r^ + beta u^), z^ = zeta r^ + eta z^ - alpha u^,
     * x += alpha p^ + z^, r = t - eta y - zeta c, beta = (alpha/zeta) <r~,r_new>/<r~,r>,
     * w = c + beta q, p^ = r^ + beta (p^ - u^). */
    double *rh = vnew(&S), *ph = vnew(&S), *q = vnew(&S), *qh = vnew(&S), *tv = vnew(&S), *th = vnew(&S);
    double *cv = vnew(&S), *y = vnew(&S), *uh = vnew(&S), *zh = vnew(&S), *wv = vnew(&S), *tprev = vnew(&S), *thprev = vnew(&S);
    num rho, rhon, alpha, beta = n_zero(), zeta, eta, sig, one = {mp_from_d(1.0), mp_zero()};
    rho = dot(n, t, rt, r);
    for (it = 1; it <= maxit; ++it) {
      if (n_is_zero(rho)) { st = ORC_BREAKDOWN; it--; break; }
      apply_m(&S, 0, r, rh);
      vaxpy(&S, tmp, ph, n_neg(one), uh);     /* p^ - u^ */
      vaxpy(&S, ph, rh, beta, tmp);           /* p^ = r^ + beta (p^ - u^) */
      spmv(n, rp, ci, val, t, ph, q);         /* q = A p^ */
      sig = dot(n, t, rt, q);
      if (n_is_zero(sig)) { st = ORC_BREAKDOWN; it--; break; }
      alpha = n_div(rho, sig, t);
      apply_m(&S, 0, q, qh);
      vaxpy(&S, tv, r, n_neg(alpha), q);      /* t = r - alpha q */
      vaxpy(&S, th, rh, n_neg(alpha), qh);    /* t^ = r^ - alpha q^ */
      spmv(n, rp, ci, val, t, th, cv);        /* c = A t^ */
      vaxpy(&S, tmp, tprev, n_neg(one), tv);  /* t_prev - t */
      vaxpy(&S, y, tmp, n_neg(alpha), wv);    /* y = t_prev - t - alpha w */
      {
        num cc = dot(n, t, cv, cv), ct = dot(n, t, cv, tv);
        if (n_is_zero(cc)) {                  /* c = A t^ = 0: t is already zero */
          zeta = n_zero();
          eta = n_zero();
        } else if (it == 1 || (flags & 1)) {
          zeta = n_div(ct, cc, t);
          eta = n_zero();
        } else {
          num yy = dot(n, t, y, y), yt = dot(n, t, y, tv), cy = dot(n, t, cv, y), yc = dot(n, t, y, cv);
          num det = n_sub(n_mul(cc, yy, t), n_mul(cy, yc, t), t);
          if (n_is_zero(det)) { st = ORC_BREAKDOWN; it--; break; }
          zeta = n_div(n_sub(n_mul(yy, ct, t), n_mul(cy, yt, t), t), det, t);
          eta = n_div(n_sub(n_mul(cc, yt, t), n_mul(yc, ct, t), t), det, t);
        }
      }
      vaxpy(&S, tmp, thprev, n_neg(one), rh); /* t^_prev - r^ */
      vaxpy(&S, tmp, tmp, beta, uh);          /*   + beta u^ */
      {
        int s2 = s;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i = 0; i < n; ++i) {             /* u^ = zeta q^ + eta (...) */
          num a = n_mul(zeta, n_load(qh + (size_t)i * s2, t), t);
          num bb = n_mul(eta, n_load(tmp + (size_t)i * s2, t), t);
          n_store(uh + (size_t)i * s2, n_add(a, bb, t), t);
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i = 0; i < n; ++i) {             /* z^ = zeta r^ + eta z^ - alpha u^ */
          num a = n_mul(zeta, n_load(rh + (size_t)i * s2, t), t);
          num bb = n_mul(eta, n_load(zh + (size_t)i * s2, t), t);
          num cc2 = n_mul(alpha, n_load(uh + (size_t)i * s2, t), t);
          n_store(zh + (size_t)i * s2, n_sub(n_add(a, bb, t), cc2, t), t);
        }
      }
      vaxpy(&S, x, x, alpha, ph);             /* x += alpha p^ */
      vaxpy(&S, x, x, one, zh);               /*    + z^ */
      vaxpy(&S, tmp, tv, n_neg(eta), y);      /* t - eta y */
      vaxpy(&S, r, tmp, n_neg(zeta), cv);     /* r = t - eta y - zeta c */
      if (g_trace) {
        g_trace[2 * it] = ortho(n, t, cv, r);
        g_trace[2 * it + 1] = it > 1 ? ortho(n, t, y, r) : 0.0;
      }
      nr = nrm2(n, t, r);
      if (hist) hist[it] = nr.c[0];
      if (nan_mp(nr)) { st = ORC_NAN; break; }
      if (stop_check(&S, &R, b, x, r, rtrue, nr.c[0], tol, it)) { st = ORC_OK; break; }
      if (n_is_zero(zeta)) { st = ORC_BREAKDOWN; break; }
      rhon = dot(n, t, rt, r);
      beta = n_mul(n_div(alpha, zeta, t), n_div(rhon, rho, t), t);
      vaxpy(&S, wv, cv, beta, q);             /* w = c + beta q */
      vcopy(&S, tprev, tv);
      vcopy(&S, thprev, th);
      rho = rhon;
    }
    free(rh); free(ph); free(q); free(qh); free(tv); free(th); free(cv); free(y); free(uh); free(zh); free(wv);
    free(tprev); free(thprev);
  } else {
    st = ORC_INVALID;
  }
  if (it > maxit) it = maxit;
finish:
  if (iters_out) *iters_out = it;
  if (relres_true) { /* || b - A x || / || b - A x0 || with the final x (leading components) */
    spmv(n, rp, ci, val, t, x, tmp);
    vaxpy(&S, tmp, b, n_neg((num){mp_from_d(1.0), mp_zero()}), tmp);
    *relres_true = r0n > 0.0 ? nrm2(n, t, tmp).c[0] / r0n : 0.0;
  }
  if (nrep_out) *nrep_out = R.nrep;
  if (S.have_ah) csr_free(&S.ah);
  free(r); free(rt); free(tmp); free(rtrue);
  return st;
}

/* orc_krylov with the test hooks above (shadow and trace may be NULL). */
int orc_krylov_hooks(int method, int n, const int *rp, const int *ci, const double *val, int c, int w, int ilu,
                     const double *fac, const double *b, double *x, double tol_rel, double tol_abs, int maxit,
                     int flags, double *hist, int *iters_out, double *relres_true, const double *shadow,
                     double *trace, int true_res_period, double *hist_true, int *nrep_out) {
  int st;
  g_shadow = shadow;
  g_trace = trace;
  st = orc_krylov(method, n, rp, ci, val, c, w, ilu, fac, b, x, tol_rel, tol_abs, maxit, flags, hist, iters_out,
                  relres_true, true_res_period, hist_true, nrep_out);
  g_shadow = NULL;
  g_trace = NULL;
  return st;
}
