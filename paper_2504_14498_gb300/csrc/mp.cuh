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
//   W = 3, 4  every operation is evaluated exactly as a nonoverlapping expansion (Shewchuk,
//          DCG 18(3), 1997: Grow-Expansion with zero elimination, Compress) and the exact
//          value is rounded greedily: c_k = leading part of (x - c_0 - ... - c_{k-1}).
//          Division: W+1 long-division digits with exact remainders.  Square root: Newton.
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
// Exact expansions (W = 3, 4).  Fixed capacity; components nonoverlapping, increasing
// magnitude, no zeros (an empty expansion is the value 0).
// ---------------------------------------------------------------------------------------------
template <int CAP>
struct Ex {
  int m;
  double e[CAP];
};
template <int CAP>
MPK_NOINLINE void ex_grow(Ex<CAP>& x, double b) {
  double q = b, h;
  int k = 0;
  for (int i = 0; i < x.m; ++i) {
    two_sum(q, x.e[i], q, h);
    if (h != 0.0) x.e[k++] = h;
  }
  if (q != 0.0) x.e[k++] = q;
  x.m = k;
}
template <int CAP>
MPK_NOINLINE double ex_top(const Ex<CAP>& x) {  // leading component after Compress
  if (x.m == 0) return 0.0;
  double g[CAP];
  double q = x.e[x.m - 1], qq;
  int bottom = x.m - 1;
  for (int i = x.m - 2; i >= 0; --i) {
    fast_two_sum(q, x.e[i], q, qq);
    if (qq != 0.0) {
      g[bottom--] = q;
      q = qq;
    }
  }
  g[bottom] = q;
  for (int i = bottom + 1; i < x.m; ++i) fast_two_sum(g[i], q, q, qq);
  return q;
}
template <int W, int CAP>
MPK_NOINLINE R<W> ex_round(Ex<CAP>& x) {
  R<W> z = r_zero<W>();
  for (int k = 0; k < W; ++k) {
    double t = ex_top(x);
    z.c[k] = t;
    if (t == 0.0) break;
    ex_grow(x, -t);
  }
  return z;
}
template <int W>
MPK_NOINLINE R<W> ex_add(R<W> a, R<W> b) {
  Ex<2 * W + W + 2> x;
  x.m = 0;
  for (int k = 0; k < W; ++k) {
    ex_grow(x, a.c[k]);
    ex_grow(x, b.c[k]);
  }
  return ex_round<W>(x);
}
template <int W>
MPK_NOINLINE R<W> ex_mul_fp(R<W> a, double d) {
  Ex<2 * W + W + 2> x;
  x.m = 0;
  for (int k = 0; k < W; ++k) {
    double p, e;
    two_prod(a.c[k], d, p, e);
    ex_grow(x, p);
    ex_grow(x, e);
  }
  return ex_round<W>(x);
}
template <int W>
MPK_NOINLINE R<W> ex_mul(R<W> a, R<W> b) {
  Ex<2 * W * W + W + 2> x;
  x.m = 0;
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < W; ++j) {
      double p, e;
      two_prod(a.c[i], b.c[j], p, e);
      ex_grow(x, p);
      ex_grow(x, e);
    }
  return ex_round<W>(x);
}
template <int W>
MPK_NOINLINE R<W> ex_div(R<W> a, R<W> b) {
  Ex<W + 2 * W * (W + 1) + 2> rem;
  Ex<W + 1 + W + 2> quo;
  rem.m = 0;
  quo.m = 0;
  for (int i = 0; i < W; ++i) ex_grow(rem, a.c[i]);
  for (int k = 0; k <= W; ++k) {
    double q = ex_top(rem) / b.c[0];
    if (q == 0.0 || !isfinite(q)) {
      if (!isfinite(q)) ex_grow(quo, q);
      break;
    }
    ex_grow(quo, q);
    for (int i = 0; i < W; ++i) {
      double p, e;
      two_prod(q, b.c[i], p, e);
      ex_grow(rem, -p);
      ex_grow(rem, -e);
    }
  }
  return ex_round<W>(quo);
}

// ---------------------------------------------------------------------------------------------
// Generic real operations
// ---------------------------------------------------------------------------------------------
template <int W>
MPK_HD R<W> add(R<W> a, R<W> b) {
  if constexpr (W == 1) return r_from<1>(a.c[0] + b.c[0]);
  else if constexpr (W == 2) return dw_add(a, b);
  else return ex_add<W>(a, b);
}
template <int W>
MPK_HD R<W> sub(R<W> a, R<W> b) {
  return add<W>(a, r_neg<W>(b));
}
template <int W>
MPK_HD R<W> mul(R<W> a, R<W> b) {
  if constexpr (W == 1) return r_from<1>(a.c[0] * b.c[0]);
  else if constexpr (W == 2) return dw_mul(a, b);
  else return ex_mul<W>(a, b);
}
template <int W>
MPK_HD R<W> mul_fp(R<W> a, double d) {
  if constexpr (W == 1) return r_from<1>(a.c[0] * d);
  else if constexpr (W == 2) return dw_mul_fp(a, d);
  else return ex_mul_fp<W>(a, d);
}
template <int W>
MPK_HD R<W> div(R<W> a, R<W> b) {
  if constexpr (W == 1) return r_from<1>(a.c[0] / b.c[0]);
  else if constexpr (W == 2) return dw_div(a, b);
  else return ex_div<W>(a, b);
}
template <int W>
MPK_HD R<W> div_fp(R<W> a, double d) {
  if constexpr (W == 1) return r_from<1>(a.c[0] / d);
  else if constexpr (W == 2) return dw_div_fp(a, d);
  else return ex_div<W>(a, r_from<W>(d));
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
