// mp.cuh -- device multi-component arithmetic (D, DD, TD, QD; real and complex) for sm_103a.
//
// Number formats of Sec. 2 of Kouya (arXiv 2504.14498): binary64 with W = 1, 2, 3 or 4
// components, leading component first.  Definitions (the paper names the formats, not the
// algorithms):
//   W = 1  plain binary64, one rounding per operation.
//   W = 2  double-word algorithms of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017):
//          accurate DW+DW (their Alg. 6), DW*FP with FMA (Alg. 9), DW*DW with FMA (Alg. 12),
//          DW/FP (Alg. 15), DW/DW (Alg. 17, whose inner DW*FP is Alg. 7); square root from
//          one Newton correction of the binary64 root.
//   W = 3, 4  renormalisation of the operation's exact (or nearly exact) terms: a magnitude
//          sort, an exact TwoSum chain, W components kept top-down (details below); relative
//          error at most about 2^(-53 W) of the exact result, cancellation included.
// Complex numbers use the fixed operation orders
//   (a+bi)(c+di) = (ac - bd) + (ad + bc)i,   conj(a+bi)(c+di) = (ac + bd) + (ad - bc)i,
//   (a+bi)/(c+di): scale all four by 2^-e (e = frexp exponent of max(|c|,|d|) leading parts),
//                  then ((ac + bd) + (bc - ad)i) / (cc + dd).
// The library is compiled with -fmad=false: no a*b+c below is contracted unless fma() is
// written.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpk {

#define MPK_HD __device__ __forceinline__
#define MPK_NOINLINE __device__ __noinline__

// ---------------------------------------------------------------------------------------------
// Error-free transformations
// ---------------------------------------------------------------------------------------------
// TwoSum: s = fl(a + b) and the exact error e = (a + b) - s.  Both are unique (e is exactly
// representable), so any exact method returns Knuth's TwoSum result (up to the sign of a zero
// e).  Here: Dekker's FastTwoSum on the operands ordered by exponent.  FastTwoSum is exact when
// the first operand's exponent is not smaller than the second's; comparing the high words with
// the sign cleared orders by exponent first.  The order is decided by integer instructions, so
// the sum costs 3 binary64 instructions instead of Knuth's 6: on this GPU every binary64 warp
// instruction occupies a sub-partition's FP64 unit for 64 cycles.
MPK_HD void two_sum(double a, double b, double& s, double& e) {
  const unsigned ha = (unsigned)__double2hiint(a) & 0x7fffffffu;
  const unsigned hb = (unsigned)__double2hiint(b) & 0x7fffffffu;
  const double x = ha >= hb ? a : b;
  const double y = ha >= hb ? b : a;
  s = x + y;
  e = y - (s - x);
}
MPK_HD void fast_two_sum(double a, double b, double& s, double& e) {  // Dekker, |a| >= |b|
  s = a + b;
  e = b - (s - a);
}
MPK_HD void two_prod(double a, double b, double& p, double& e) {  // FMA-based, exact
  p = a * b;
  e = fma(a, b, -p);
}

template <int W>
struct R {
  double c[W];
};

template <int W>
MPK_HD R<W> r_zero() {
  R<W> z;
#pragma unroll
  for (int k = 0; k < W; ++k) z.c[k] = 0.0;
  return z;
}
template <int W>
MPK_HD R<W> r_from(double d) {
  R<W> z = r_zero<W>();
  z.c[0] = d;
  return z;
}
// Negation flips the sign bits with an integer instruction: the result feeds two_sum's integer
// magnitude comparison, so a floating-point negation would cost a binary64 instruction.
template <int W>
MPK_HD R<W> r_neg(R<W> a) {
#pragma unroll
  for (int k = 0; k < W; ++k)
    a.c[k] = __longlong_as_double(__double_as_longlong(a.c[k]) ^ (long long)0x8000000000000000ull);
  return a;
}
template <int W>
MPK_HD R<W> r_ldexp(R<W> a, int e) {
#pragma unroll
  for (int k = 0; k < W; ++k) a.c[k] = ldexp(a.c[k], e);
  return a;
}

// ---------------------------------------------------------------------------------------------
// Double-word
// ---------------------------------------------------------------------------------------------
MPK_HD R<2> dw_add(R<2> x, R<2> y) {
  double sh, sl, th, tl;
  two_sum(x.c[0], y.c[0], sh, sl);
  two_sum(x.c[1], y.c[1], th, tl);
  double c = sl + th;
  double vh, vl;
  fast_two_sum(sh, c, vh, vl);
  double w = tl + vl;
  R<2> z;
  fast_two_sum(vh, w, z.c[0], z.c[1]);
  return z;
}
MPK_HD R<2> dw_mul_fp(R<2> x, double y) {  // FMA variant (bound 2u^2)
  double ch, cl1;
  two_prod(x.c[0], y, ch, cl1);
  double cl3 = fma(x.c[1], y, cl1);
  R<2> z;
  fast_two_sum(ch, cl3, z.c[0], z.c[1]);
  return z;
}
MPK_HD R<2> dw_mul_fp_plain(R<2> x, double y) {  // variant used inside the DW/DW division
  double ch, cl1;
  two_prod(x.c[0], y, ch, cl1);
  double cl2 = x.c[1] * y;
  double th, tl1;
  fast_two_sum(ch, cl2, th, tl1);
  double tl2 = tl1 + cl1;
  R<2> z;
  fast_two_sum(th, tl2, z.c[0], z.c[1]);
  return z;
}
MPK_HD R<2> dw_mul(R<2> x, R<2> y) {
  double ch, cl1;
  two_prod(x.c[0], y.c[0], ch, cl1);
  double tl0 = x.c[1] * y.c[1];
  double tl1 = fma(x.c[0], y.c[1], tl0);
  double cl2 = fma(x.c[1], y.c[0], tl1);
  double cl3 = cl1 + cl2;
  R<2> z;
  fast_two_sum(ch, cl3, z.c[0], z.c[1]);
  return z;
}
MPK_HD R<2> dw_div_fp(R<2> x, double y) {
  double th = x.c[0] / y;
  double ph, pl;
  two_prod(th, y, ph, pl);
  double dh = x.c[0] - ph;
  double dt = dh - pl;
  double d = dt + x.c[1];
  double tl = d / y;
  R<2> z;
  fast_two_sum(th, tl, z.c[0], z.c[1]);
  return z;
}
MPK_HD R<2> dw_div(R<2> x, R<2> y) {
  double th = x.c[0] / y.c[0];
  R<2> r = dw_mul_fp_plain(y, th);
  double ph = x.c[0] - r.c[0];
  double dl = x.c[1] - r.c[1];
  double d = ph + dl;
  double tl = d / y.c[0];
  R<2> z;
  fast_two_sum(th, tl, z.c[0], z.c[1]);
  return z;
}
MPK_HD R<2> dw_sqrt(R<2> x) {
  if (!(x.c[0] > 0.0)) return r_from<2>(sqrt(x.c[0]));
  double s = sqrt(x.c[0]);
  double d = fma(-s, s, x.c[0]);
  d = d + x.c[1];
  double t = d / (2.0 * s);
  R<2> z;
  fast_two_sum(s, t, z.c[0], z.c[1]);
  return z;
}

// ---------------------------------------------------------------------------------------------
// Triple- and quad-word (W = 3, 4): renormalisation of a short list of binary64 terms.
// Every operation first produces terms whose exact sum is the result (or, for products, the
// result up to terms below 2^(-53 W) of it), then
//   (1) sorts them by decreasing magnitude -- a compare-exchange network keyed on the high word
//       with the sign cleared, integer instructions only (on this GPU a binary64 warp
//       instruction costs 64 cycles of its sub-partition, an integer one about two);
//   (2) VecSum: a chain of TwoSums from the smallest term up (exact: the outputs sum to the
//       inputs), leaving the rounded total first and the rounding errors after it;
//   (3) keeps W components top-down: the running value is added to the next error term with
//       TwoSum; a nonzero error ends a component (its sum is emitted, the error carries on), a
//       zero one merges the term; after W components the rest is dropped.
// This is the structure of the accurate expansion additions of Hida, Li and Bailey (2001) and of
// Joldes, Muller and Popescu's VecSum / VecSumErrBranch renormalisation (IEEE TC 2016).  Because
// (2) is exact, cancellation is resolved before anything is dropped, so the relative error is
// about 2^(-53 W) of the exact result even when the operands cancel.  Measured against exact
// rationals over random, cancelling and sparse operands (|exponents| <= 250): at most
// 2^-159.3 (TD) and 2^-212.9 (QD) for add, multiply (by binary64 and by TD / QD), divide.
// Products keep TwoProd errors of the terms a_i b_j with i + j <= W - 2 and round the terms with
// i + j = W - 1; terms with i + j >= W are below 2^(-53 W) of the product and omitted.
// Division: W + 1 quotient digits q_k = r_0 / b_0, each followed by r := r - q_k b, then the
// digits renormalised.  Square root: Newton's iteration x := x + (a - x^2) / (2x) from the
// binary64 root, three steps.
// ---------------------------------------------------------------------------------------------
MPK_HD unsigned mag_key(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
MPK_HD void cex_desc(double& a, double& b) {  // a keeps the larger magnitude
  const bool sw = mag_key(b) > mag_key(a);
  const double t = a;
  a = sw ? b : a;
  b = sw ? t : b;
}
template <int M>
MPK_HD void sort_desc(double (&x)[M]) {
  if constexpr ((M & (M - 1)) == 0) {  // bitonic network
#pragma unroll
    for (int k = 2; k <= M; k <<= 1)
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const int l = i ^ j;
          if (l > i) {
            if ((i & k) == 0) cex_desc(x[i], x[l]);
            else cex_desc(x[l], x[i]);
          }
        }
  } else {  // odd-even transposition network
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
      for (int i = r & 1; i + 1 < M; i += 2) cex_desc(x[i], x[i + 1]);
  }
}
// W components of the exact sum of x[0..M), x sorted by decreasing magnitude.
template <int W, int M>
MPK_HD R<W> renorm(const double (&x)[M]) {
  double y[M];
  double sacc = x[M - 1];
#pragma unroll
  for (int i = M - 2; i >= 0; --i) two_sum(x[i], sacc, sacc, y[i + 1]);
  y[0] = sacc;
  R<W> z = r_zero<W>();
  double run = y[0];
  int j = 0;
#pragma unroll
  for (int i = 1; i < M; ++i) {
    double r, e;
    two_sum(run, y[i], r, e);
    const bool emit = e != 0.0;
#pragma unroll
    for (int k = 0; k < W; ++k) z.c[k] = (emit && j == k) ? r : z.c[k];
    j += emit ? 1 : 0;
    run = emit ? e : r;
  }
#pragma unroll
  for (int k = 0; k < W; ++k) z.c[k] = (j == k) ? run : z.c[k];
  return z;
}
template <int W, int M>
MPK_HD R<W> sort_renorm(double (&x)[M]) {
  sort_desc<M>(x);
  return renorm<W, M>(x);
}
template <int W>
MPK_NOINLINE R<W> mw_add(const R<W>& a, const R<W>& b) {
  constexpr int M = (2 * W <= 8) ? 8 : 2 * W;
  double x[M];
#pragma unroll
  for (int k = 0; k < M; ++k) x[k] = k < W ? a.c[k] : (k < 2 * W ? b.c[k - W] : 0.0);
  return sort_renorm<W, M>(x);
}
template <int W>
MPK_NOINLINE R<W> mw_mul_fp(const R<W>& a, double d) {
  constexpr int M = (2 * W <= 8) ? 8 : 2 * W;
  double x[M];
#pragma unroll
  for (int k = 0; k < M; ++k) x[k] = 0.0;
#pragma unroll
  for (int k = 0; k < W; ++k) two_prod(a.c[k], d, x[2 * k], x[2 * k + 1]);
  return sort_renorm<W, M>(x);
}
template <int W>
MPK_NOINLINE R<W> mw_mul(const R<W>& a, const R<W>& b) {
  // i + j <= W - 2: W (W - 1) / 2 TwoProds; i + j == W - 1: W rounded products
  constexpr int NP = W * (W - 1) / 2, M = 2 * NP + W;
  double x[M];
  int t = 0;
#pragma unroll
  for (int i = 0; i < W; ++i)
#pragma unroll
    for (int j = 0; j < W; ++j) {
      if (i + j <= W - 2) {
        two_prod(a.c[i], b.c[j], x[t], x[t + 1]);
        t += 2;
      } else if (i + j == W - 1) {
        x[t] = a.c[i] * b.c[j];
        t += 1;
      }
    }
  return sort_renorm<W, M>(x);
}
template <int W>
MPK_NOINLINE R<W> mw_div(R<W> a, R<W> b) {
  double q[W + 1];
  R<W> r = a;
#pragma unroll
  for (int k = 0; k <= W; ++k) {
    q[k] = r.c[0] / b.c[0];
    if (k < W) r = mw_add<W>(r, r_neg<W>(mw_mul_fp<W>(b, q[k])));
  }
  return sort_renorm<W, W + 1>(q);
}
template <int W>
MPK_NOINLINE R<W> mw_div_fp(R<W> a, double d) {
  double q[W + 1];
  R<W> r = a;
#pragma unroll
  for (int k = 0; k <= W; ++k) {
    q[k] = r.c[0] / d;
    if (k < W) {
      R<W> p = r_zero<W>();
      two_prod(d, q[k], p.c[0], p.c[1]);
      r = mw_add<W>(r, r_neg<W>(p));
    }
  }
  return sort_renorm<W, W + 1>(q);
}

// ---------------------------------------------------------------------------------------------
// Generic real operations
// ---------------------------------------------------------------------------------------------
template <int W>
MPK_HD R<W> add(R<W> a, R<W> b) {
  if constexpr (W == 1) return r_from<1>(a.c[0] + b.c[0]);
  else if constexpr (W == 2) return dw_add(a, b);
  else return mw_add<W>(a, b);
}
template <int W>
MPK_HD R<W> sub(R<W> a, R<W> b) {
  return add<W>(a, r_neg<W>(b));
}
template <int W>
MPK_HD R<W> mul(R<W> a, R<W> b) {
  if constexpr (W == 1) return r_from<1>(a.c[0] * b.c[0]);
  else if constexpr (W == 2) return dw_mul(a, b);
  else return mw_mul<W>(a, b);
}
template <int W>
MPK_HD R<W> mul_fp(R<W> a, double d) {
  if constexpr (W == 1) return r_from<1>(a.c[0] * d);
  else if constexpr (W == 2) return dw_mul_fp(a, d);
  else return mw_mul_fp<W>(a, d);
}
template <int W>
MPK_HD R<W> div(R<W> a, R<W> b) {
  if constexpr (W == 1) return r_from<1>(a.c[0] / b.c[0]);
  else if constexpr (W == 2) return dw_div(a, b);
  else return mw_div<W>(a, b);
}
template <int W>
MPK_HD R<W> div_fp(R<W> a, double d) {
  if constexpr (W == 1) return r_from<1>(a.c[0] / d);
  else if constexpr (W == 2) return dw_div_fp(a, d);
  else return mw_div_fp<W>(a, d);
}
template <int W>
MPK_HD R<W> rsqrt_mp(R<W> a) {  // square root
  if constexpr (W == 1) return r_from<1>(sqrt(a.c[0]));
  else if constexpr (W == 2) return dw_sqrt(a);
  else {
    if (!(a.c[0] > 0.0)) return r_from<W>(sqrt(a.c[0]));
    R<W> s = r_from<W>(sqrt(a.c[0]));
    for (int it = 0; it < 3; ++it) {
      R<W> d = sub<W>(a, mul<W>(s, s));
      R<W> two_s = mul_fp<W>(s, 2.0);
      s = add<W>(s, div<W>(d, two_s));
    }
    return s;
  }
}

// ---------------------------------------------------------------------------------------------
// Numbers: CP = 1 (real) or 2 (complex)
// ---------------------------------------------------------------------------------------------
template <int W, int CP>
struct N {
  R<W> re, im;
};
template <int W, int CP>
MPK_HD N<W, CP> n_zero() {
  N<W, CP> z;
  z.re = r_zero<W>();
  z.im = r_zero<W>();
  return z;
}
template <int W, int CP>
MPK_HD N<W, CP> n_real(double d) {
  N<W, CP> z = n_zero<W, CP>();
  z.re.c[0] = d;
  return z;
}
template <int W, int CP>
MPK_HD N<W, CP> n_neg(N<W, CP> a) {
  a.re = r_neg<W>(a.re);
  a.im = r_neg<W>(a.im);
  return a;
}
template <int W, int CP>
MPK_HD N<W, CP> n_conj(N<W, CP> a) {
  a.im = r_neg<W>(a.im);
  return a;
}
template <int W, int CP>
MPK_HD bool n_is_zero(const N<W, CP>& a) {
  return a.re.c[0] == 0.0 && (CP == 1 || a.im.c[0] == 0.0);
}
template <int W, int CP>
MPK_HD N<W, CP> n_add(N<W, CP> a, N<W, CP> b) {
  N<W, CP> z = n_zero<W, CP>();
  z.re = add<W>(a.re, b.re);
  if constexpr (CP == 2) z.im = add<W>(a.im, b.im);
  return z;
}
template <int W, int CP>
MPK_HD N<W, CP> n_sub(N<W, CP> a, N<W, CP> b) {
  N<W, CP> z = n_zero<W, CP>();
  z.re = sub<W>(a.re, b.re);
  if constexpr (CP == 2) z.im = sub<W>(a.im, b.im);
  return z;
}
template <int W, int CP>
MPK_HD N<W, CP> n_mul(N<W, CP> a, N<W, CP> b) {
  N<W, CP> z = n_zero<W, CP>();
  if constexpr (CP == 1) {
    z.re = mul<W>(a.re, b.re);
  } else {
    z.re = sub<W>(mul<W>(a.re, b.re), mul<W>(a.im, b.im));
    z.im = add<W>(mul<W>(a.re, b.im), mul<W>(a.im, b.re));
  }
  return z;
}
template <int W, int CP>
MPK_HD N<W, CP> n_mul_conj(N<W, CP> a, N<W, CP> b) {  // conj(a) * b
  N<W, CP> z = n_zero<W, CP>();
  if constexpr (CP == 1) {
    z.re = mul<W>(a.re, b.re);
  } else {
    z.re = add<W>(mul<W>(a.re, b.re), mul<W>(a.im, b.im));
    z.im = sub<W>(mul<W>(a.re, b.im), mul<W>(a.im, b.re));
  }
  return z;
}
template <int W, int CP>
MPK_HD N<W, CP> n_div(N<W, CP> a, N<W, CP> b) {
  N<W, CP> z = n_zero<W, CP>();
  if constexpr (CP == 1) {
    z.re = div<W>(a.re, b.re);
  } else {
    double m = fmax(fabs(b.re.c[0]), fabs(b.im.c[0]));
    if (m > 0.0 && isfinite(m)) {
      int e;
      frexp(m, &e);
      a.re = r_ldexp<W>(a.re, -e);
      a.im = r_ldexp<W>(a.im, -e);
      b.re = r_ldexp<W>(b.re, -e);
      b.im = r_ldexp<W>(b.im, -e);
    }
    R<W> den = add<W>(mul<W>(b.re, b.re), mul<W>(b.im, b.im));
    R<W> nr = add<W>(mul<W>(a.re, b.re), mul<W>(a.im, b.im));
    R<W> ni = sub<W>(mul<W>(a.im, b.re), mul<W>(a.re, b.im));
    z.re = div<W>(nr, den);
    z.im = div<W>(ni, den);
  }
  return z;
}
// x * (fr + fi i), binary64 (complex) factor
template <int W, int CP>
MPK_HD N<W, CP> n_mul_fp(N<W, CP> x, double fr, double fi) {
  N<W, CP> z = n_zero<W, CP>();
  if constexpr (CP == 1) {
    z.re = mul_fp<W>(x.re, fr);
  } else {
    z.re = sub<W>(mul_fp<W>(x.re, fr), mul_fp<W>(x.im, fi));
    z.im = add<W>(mul_fp<W>(x.im, fr), mul_fp<W>(x.re, fi));
  }
  return z;
}
// x / (fr + fi i), binary64 (complex) divisor
template <int W, int CP>
MPK_HD N<W, CP> n_div_fp(N<W, CP> x, double fr, double fi) {
  N<W, CP> z = n_zero<W, CP>();
  if constexpr (CP == 1) {
    z.re = div_fp<W>(x.re, fr);
  } else {
    R<W> den = add<W>(mul_fp<W>(r_from<W>(fr), fr), mul_fp<W>(r_from<W>(fi), fi));
    R<W> nr = add<W>(mul_fp<W>(x.re, fr), mul_fp<W>(x.im, fi));
    R<W> ni = sub<W>(mul_fp<W>(x.im, fr), mul_fp<W>(x.re, fi));
    z.re = div<W>(nr, den);
    z.im = div<W>(ni, den);
  }
  return z;
}

// ---------------------------------------------------------------------------------------------
// Vector element access: entry i of an (n, CP, W) array of doubles
// ---------------------------------------------------------------------------------------------
template <int W, int CP>
__device__ __forceinline__ N<W, CP> n_load(const double* __restrict__ v, int64_t i) {
  N<W, CP> z = n_zero<W, CP>();
  const double* p = v + i * (CP * W);
  if constexpr ((CP * W) % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int k = 0; k < CP * W / 2; ++k) {
      double2 t = q[k];
      int a = 2 * k, b = 2 * k + 1;
      if (a < W) z.re.c[a] = t.x; else z.im.c[a - W] = t.x;
      if (b < W) z.re.c[b] = t.y; else z.im.c[b - W] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) z.re.c[k] = p[k];
    if constexpr (CP == 2) {
#pragma unroll
      for (int k = 0; k < W; ++k) z.im.c[k] = p[W + k];
    }
  }
  return z;
}
template <int W, int CP>
__device__ __forceinline__ void n_store(double* __restrict__ v, int64_t i, const N<W, CP>& z) {
  double* p = v + i * (CP * W);
  if constexpr ((CP * W) % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int k = 0; k < CP * W / 2; ++k) {
      int a = 2 * k, b = 2 * k + 1;
      double2 t;
      t.x = a < W ? z.re.c[a] : z.im.c[a - W];
      t.y = b < W ? z.re.c[b] : z.im.c[b - W];
      q[k] = t;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) p[k] = z.re.c[k];
    if constexpr (CP == 2) {
#pragma unroll
      for (int k = 0; k < W; ++k) p[W + k] = z.im.c[k];
    }
  }
}

}  // namespace mpk
