// mt_dd.cuh -- double-double ("double-word") arithmetic for the clustered
// roots that binary64 cannot separate (the MT_DD tier).
//
// A value is hi + lo with |lo| <= ulp(hi)/2.  The operations are the
// published error-free transforms and double-word algorithms:
//   TwoSum (Knuth / Moller), FastTwoSum (Dekker), TwoProd with one FMA, and
//   Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic
//   building blocks of double-word arithmetic" (ACM TOMS 2017):
//   AccurateDWPlusDW (relative error <= 3u^2 + 13u^3), DWTimesDW3 (<= 4u^2),
//   DWTimesFP3 (<= 2u^2), u = 2^-53.
// The certificate charges DD_REL_ERR * |result| per operation, a bound above
// all of these.
//
// The paper's counterpart is MPFR at 128 bits, used "only when necessary"
// (Sec. 1.1, Sec. 6.3.2: the roots of p_n near -2 for n >= 30 in FP80); in
// binary64 the same happens from n ~ 26 on.
#pragma once
#include "mt_common.cuh"

namespace mt {

struct dd {
  double hi, lo;
};

constexpr double DD_U2 = 1.2325951644078310e-32;  // u^2 = 2^-106
constexpr double DD_REL_ERR = 8.0 * DD_U2;        // per-operation bound used by the certificate

__device__ __forceinline__ dd dd_make(double a) { return dd{a, 0.0}; }

__device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  return dd{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {  // |a| >= |b|
  const double s = a + b;
  return dd{s, b - (s - a)};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = a * b;
  return dd{p, fma(a, b, -p)};
}

// AccurateDWPlusDW
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
// DWPlusFP
__device__ __forceinline__ dd dd_add_d(dd a, double b) {
  dd s = two_sum(a.hi, b);
  s.lo += a.lo;
  return fast_two_sum(s.hi, s.lo);
}
// DWTimesDW3
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd c = two_prod(a.hi, b.hi);
  const double tl0 = a.lo * b.lo;
  const double tl1 = fma(a.hi, b.lo, tl0);
  const double cl2 = fma(a.lo, b.hi, tl1);
  c.lo += cl2;
  return fast_two_sum(c.hi, c.lo);
}
// DWTimesFP3
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  dd c = two_prod(a.hi, b);
  c.lo = fma(a.lo, b, c.lo);
  return fast_two_sum(c.hi, c.lo);
}
__device__ __forceinline__ dd dd_twice(dd a) { return dd{twice_f64(a.hi), twice_f64(a.lo)}; }  // exact
__device__ __forceinline__ double dd_to_d(dd a) { return a.hi + a.lo; }

// ---------------------------------------------------------------------------
// Orbit of P_alpha = p_m + alpha p_lcap in double-double for the value; the
// c-derivative (the Newton denominator, needed to relative accuracy only) in
// binary64 from the hi parts.  Returns P (dd) and P' (binary64).
__device__ __forceinline__ void orbit_dd(int m, int lcap, double alpha, dd cr, dd ci, dd& vr, dd& vi,
                                         double& dr, double& di) {
  dd zr = dd_make(0.0), zi = dd_make(0.0), capr = dd_make(0.0), capi = dd_make(0.0);
  double dzr = 0.0, dzi = 0.0, capdr = 0.0, capdi = 0.0;
  for (int k = 1; k <= m; ++k) {
    const double tzr = twice_f64(zr.hi), tzi = twice_f64(zi.hi);
    const double ndr = fma(tzr, dzr, fma(-tzi, dzi, 1.0));
    const double ndi = fma(tzr, dzi, tzi * dzr);
    const dd xx = dd_mul(zr, zr), yy = dd_mul(zi, zi), xy = dd_mul(zr, zi);
    const dd nzr = dd_add(dd_sub(xx, yy), cr);
    const dd nzi = dd_add(dd_twice(xy), ci);
    zr = nzr; zi = nzi; dzr = ndr; dzi = ndi;
    if (k == lcap) { capr = zr; capi = zi; capdr = dzr; capdi = dzi; }
  }
  if (lcap >= 0) {
    vr = dd_add(zr, dd_mul_d(capr, alpha));
    vi = dd_add(zi, dd_mul_d(capi, alpha));
    dr = fma(alpha, capdr, dzr);
    di = fma(alpha, capdi, dzi);
  } else {
    vr = zr; vi = zi; dr = dzr; di = dzi;
  }
}

// Newton with target in double-double (the dd twin of newton_target_f64,
// same log predictor and stop rule, with the rounding floor at ~1e-30).
__device__ __forceinline__ int newton_target_dd(int m, int lcap, double alpha, dd& zr, dd& zi,
                                                dd tr, dd ti, double rel, int cap, double* first,
                                                bool pred = false, double tpr = 0.0, double tpi = 0.0,
                                                double Lr = 0.0, double Li = 0.0) {
  double thr2 = 0.0, prev2 = 0.0, h2 = 0.0;
  int it = 0;
  while (it < cap) {
    dd vr, vi;
    double dr, di;
    orbit_dd(m, lcap, alpha, zr, zi, vr, vi, dr, di);
    double nr, ni;
    if (it == 0 && pred) {  // P - Tp - L P, to binary64 accuracy (a predictor)
      const double pr = dd_to_d(vr), pi = dd_to_d(vi);
      nr = (pr - tpr) - fma(Lr, pr, -Li * pi);
      ni = (pi - tpi) - fma(Lr, pi, Li * pr);
    } else {
      nr = dd_to_d(dd_sub(vr, tr));
      ni = dd_to_d(dd_sub(vi, ti));
    }
    double qr, qi;
    cdiv_f64(nr, ni, dr, di, qr, qi);
    if (!finite2(qr, qi)) break;
    zr = dd_add_d(zr, -qr);
    zi = dd_add_d(zi, -qi);
    ++it;
    const double s2 = fma(qr, qr, qi * qi);
    const double mag = 1.0 + fabs(zr.hi) + fabs(zi.hi);
    const double floor2 = (1e-30 * mag) * (1e-30 * mag);
    if (it == 1) {
      h2 = s2;
      thr2 = rel * rel * s2;
    } else if (s2 <= thr2 || s2 <= floor2 || (it >= 3 && s2 > 0.25 * prev2)) {
      break;
    }
    prev2 = s2;
  }
  if (first) *first = sqrt(h2);
  return it;
}

}  // namespace mt
