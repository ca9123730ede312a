// mt_common.cuh -- device building blocks shared by the kernels of the
// level-line Newton splitter: the polynomial descriptor, the critical-orbit
// evaluation of P and P' in binary64, the Newton quotient, and small warp
// helpers.
//
// Polynomials (Mihalache & Vigneron, Sec. 1 and eq. polySimple):
//   p_0 = 0, p_{k+1} = p_k^2 + c                 P = p_n,             deg 2^(n-1)
//   s_{l,n} = p_{l+n-1} + p_{l-1}                P = s_{l,n},         deg 2^(l+n-2)
//   q_{l,n} = p_{l+n} - p_l                      P = q_{l,n},         deg 2^(l+n-1)
// All are evaluated through the critical orbit (length m), with the
// c-derivative carried along by differentiating the recurrence:
//   p'_{k+1} = 2 p_k p'_k + 1                    (eq. DerParamDyna, parameter form)
// so one evaluation costs O(m) = O(log d) (Sec. 3, "V_d = O(log_2 d)").
#pragma once
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "mt_internal.h"

namespace mt {

// twice_f64(x) = x + x, bit for bit, on the integer pipe: a normal x below
// 2^1023 gets its exponent field incremented; zero and subnormals shift
// their significand left (becoming normal where it carries into the
// exponent); 2^1023 and up overflow to inf; inf and NaN are returned as
// they are.  On GB300 binary64 arithmetic issues at 1/64 of the binary32
// rate, so every orbit step's doubling moves off the binary64 pipe.
__device__ __forceinline__ double twice_f64(double x) {
  const int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
  const int sgn = hi & (int)0x80000000;
  int rh = hi + 0x00100000, rl = lo;  // normal: exponent + 1
  if (e == 0u) {                      // zero, subnormal
    rh = sgn | (int)(((unsigned)hi << 1) & 0x7fffffffu) | (int)((unsigned)lo >> 31);
    rl = (int)((unsigned)lo << 1);
  } else if (e == 0x7feu) {  // overflow
    rh = sgn | 0x7ff00000;
    rl = 0;
  } else if (e == 0x7ffu) {  // inf, NaN
    rh = hi;
  }
  return __hiloint2double(rh, rl);
}


// ---------------------------------------------------------------------------
// 2^k as a binary64 built from its exponent field (-1022 <= k <= 1023):
// integer work only, off the binary64 pipe.
__device__ __forceinline__ double pow2_f64(int k) { return __hiloint2double((1023 + k) << 20, 0); }

// The derivative is carried scaled: e_k = p'_k / 2^k obeys
//   e_k = p_{k-1} e_{k-1} + 2^-k,
// which drops the doubling of Im p_{k-1} that p'_k = 2 p_{k-1} p'_{k-1} + 1
// needs.  Every rounding of the scaled recurrence is the rounding of the
// plain one times a power of two, so both give the same binary64 p'_m
// (barring subnormal intermediates): 8 binary64 instructions per orbit step
// (6 FMA, 1 mul, 1 add) instead of 9.  2^-k comes from pow2_f64's integer
// exponent arithmetic.
//
// Evaluation of P_alpha = p_m + alpha * p_lcap and its derivative at c.
// lcap < 0: plain p_m.  For s_{l,n}: m = l+n-1, lcap = l-1, alpha = 1.
__device__ __forceinline__ void orbit_f64(int m, int lcap, double alpha, double cr, double ci,
                                          double& vr, double& vi, double& dr, double& di) {
  double zr = 0.0, zi = 0.0, er = 0.0, ei = 0.0;
  double cap_r = 0.0, cap_i = 0.0, cape_r = 0.0, cape_i = 0.0;
  int hexp = (1023 - 1) << 20;  // exponent field of 2^-k, k = 1
#pragma unroll 4
  for (int k = 1; k <= m; ++k) {
    const double h = __hiloint2double(hexp, 0);
    hexp -= 1 << 20;
    const double ner = fma(zr, er, fma(-zi, ei, h));      // Re(z e + 2^-k)
    const double nei = fma(zr, ei, zi * er);               // Im(z e)
    const double nzr = fma(zr, zr, fma(-zi, zi, cr));      // Re(z^2 + c)
    const double nzi = fma(twice_f64(zr), zi, ci);               // Im(z^2 + c)
    zr = nzr; zi = nzi; er = ner; ei = nei;
    if (k == lcap) { cap_r = zr; cap_i = zi; cape_r = er; cape_i = ei; }
  }
  vr = fma(alpha, cap_r, zr);
  vi = fma(alpha, cap_i, zi);
  // p'_m + alpha p'_lcap = 2^m (e_m + alpha 2^(lcap-m) e_lcap), exact scalings
  const double a = lcap > 0 ? alpha * pow2_f64(lcap - m) : 0.0, s = pow2_f64(m);
  dr = fma(a, cape_r, er) * s;
  di = fma(a, cape_i, ei) * s;
}

// Plain p_n specialisation (no capture), the hot inner loop.
__device__ __forceinline__ void orbit_pn_f64(int m, double cr, double ci, double& vr, double& vi,
                                             double& dr, double& di) {
  double zr = 0.0, zi = 0.0, er = 0.0, ei = 0.0;
  int hexp = (1023 - 1) << 20;
#pragma unroll 4
  for (int k = 1; k <= m; ++k) {
    const double h = __hiloint2double(hexp, 0);
    hexp -= 1 << 20;
    const double ner = fma(zr, er, fma(-zi, ei, h));
    const double nei = fma(zr, ei, zi * er);
    const double nzr = fma(zr, zr, fma(-zi, zi, cr));
    const double nzi = fma(twice_f64(zr), zi, ci);
    zr = nzr; zi = nzi; er = ner; ei = nei;
  }
  const double s = pow2_f64(m);
  vr = zr; vi = zi; dr = er * s; di = ei * s;
}

// binary64 -> binary32 on the integer pipe.  A conversion instruction runs
// on the binary64 pipe, the scarce one on GB300 (2 lanes per SM per clock):
// in an orbit that converts z every step it is a third of that pipe's work.
// The binary64 value of a binary32 f, built on the integer pipe (exact for
// normal f and zero; binary32 subnormals, below 1.2e-38, give +-0).
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sg = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi = sg, lo = 0u;
  if (e == 0xffu) {  // inf, NaN
    hi = sg | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (e != 0u) {
    hi = sg | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// (a + ib) / (c + id) in binary32 with c + id first scaled by a power of two
// (exactly) into [1, 2) in modulus, so that |c + id|^2 cannot leave the
// binary32 range; false for a zero, subnormal, huge or non-finite divisor.
__device__ __forceinline__ bool cdiv_f32s(float a, float b, float c, float d, float& qr, float& qi) {
  const float mx = fmaxf(fabsf(c), fabsf(d));
  const int eb = __float_as_int(mx) & 0x7f800000;
  if (eb == 0 || eb >= 0x7f000000) return false;
  const float sc = __int_as_float(0x7f000000 - eb);  // 2^-E for mx in [2^E, 2^(E+1))
  c *= sc;
  d *= sc;
  const float inv = 1.0f / fmaf(c, c, d * d);
  qr = fmaf(a, c, b * d) * inv * sc;
  qi = fmaf(b, c, -a * d) * inv * sc;
  return isfinite(qr) && isfinite(qi);
}

// f32_trunc rounds toward zero: sign, the exponent rebiased (its low eight
// bits xor 0x80 are e - 896), the top 23 mantissa bits by a funnel shift.
// |x| below 2^-126 gives +-0 (error < 2^-126), |x| from 2^128 on or a
// non-finite x gives +-inf.  |x - f32_trunc(x)| < ulp(f32_trunc(x)) else.
__device__ __forceinline__ float f32_trunc(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
  const unsigned f = __funnelshift_l(lo, (unsigned)hi, 3) ^ 0x40000000u;  // exponent field fixed
  unsigned b = (f & 0x7fffffffu) | ((unsigned)hi & 0x80000000u);
  if (e - 897u >= 254u) b = ((unsigned)hi & 0x80000000u) | (e <= 896u ? 0u : 0x7f800000u);
  return __uint_as_float(b);
}

// An upper bound of |x| in binary32 on the integer pipe: f32_trunc(|x|)
// moved up one ulp (2^-126 below the normal range, +inf from 2^128 on or
// for a non-finite x).
__device__ __forceinline__ float f32_abs_up(double x) {
  const int hi = __double2hiint(x) & 0x7fffffff;
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
  unsigned b = ((__funnelshift_l(lo, (unsigned)hi, 3) ^ 0x40000000u) & 0x7fffffffu) + 1u;
  if (e - 897u >= 254u) b = (e <= 896u) ? 0x00800000u : 0x7f800000u;
  return __uint_as_float(b);
}

// The orbit with the value in binary64 and the c-derivative in binary32
// (the mixed tier's binary64 finish).  A Newton quotient P / P' only needs
// P' to a relative error eta: the iteration then contracts by eta per step
// near the root instead of quadratically, and eta ~ m 2^-23 is far below
// the 1e-7 relative accuracy the binary32 phase leaves.  The fixed point is
// decided by P alone, which stays binary64.  4 binary64 operations per step
// (3 FMA and 1 add for the value; z enters the derivative through
// f32_trunc on the integer pipe) instead of the 8 of orbit_f64.
__device__ __forceinline__ void orbit_f64_d32(int m, int lcap, double cr, double ci, double& vr,
                                              double& vi, float& dr, float& di) {
  double zr = 0.0, zi = 0.0, cap_r = 0.0, cap_i = 0.0;
  float dzr = 0.f, dzi = 0.f, capd_r = 0.f, capd_i = 0.f;
#pragma unroll 4
  for (int k = 1; k <= m; ++k) {
    const float fr = f32_trunc(zr), fi = f32_trunc(zi);
    const float tfr = fr + fr, tfi = fi + fi;
    const float ndr = fmaf(tfr, dzr, fmaf(-tfi, dzi, 1.f));
    const float ndi = fmaf(tfr, dzi, tfi * dzr);
    const double tzr = twice_f64(zr);
    const double nzr = fma(zr, zr, fma(-zi, zi, cr));
    const double nzi = fma(tzr, zi, ci);
    zr = nzr; zi = nzi; dzr = ndr; dzi = ndi;
    if (k == lcap) { cap_r = zr; cap_i = zi; capd_r = dzr; capd_i = dzi; }
  }
  if (lcap >= 0) {
    vr = zr + cap_r; vi = zi + cap_i;
    dr = dzr + capd_r; di = dzi + capd_i;
  } else {
    vr = zr; vi = zi; dr = dzr; di = dzi;
  }
}

// orbit_f64_d32 plus the curvature of the Newton map for the finish's stop
// rule: kr + i ki = P''(c) / (2 P'(c)) in binary32.  The second derivative
// follows p''_{k+1} = 2 (p'_k^2 + p_k p''_k), carried as u_k = p''_k / 4^k,
// u_{k+1} = ((p'_k / 2^k)^2 + p_k u_k) / 2 (no binary32 overflow up to
// n = 41), on the binary32 pipe, which the binary64 orbit leaves idle.  A
// Newton step q from c leaves c - q at about q^2 P''/(2P') from the root
// (the next step), which is what the rule reads.
__device__ __forceinline__ void orbit_f64_d32_k(int m, int lcap, double cr, double ci, double& vr,
                                                double& vi, float& dr, float& di, float& kr, float& ki) {
  double zr = 0.0, zi = 0.0, cap_r = 0.0, cap_i = 0.0;
  float dzr = 0.f, dzi = 0.f, capd_r = 0.f, capd_i = 0.f;
  float ur = 0.f, ui = 0.f, capu_r = 0.f, capu_i = 0.f;
  int hexp = 127 << 23;  // exponent field of 2^-(k-1), k = 1
#pragma unroll 4
  for (int k = 1; k <= m; ++k) {
    const float fr = f32_trunc(zr), fi = f32_trunc(zi);
    const float h = __int_as_float(hexp);
    hexp -= 1 << 23;
    const float sr = dzr * h, si = dzi * h;  // p'_{k-1} / 2^(k-1)
    const float nur = 0.5f * (fmaf(sr, sr, -si * si) + fmaf(fr, ur, -fi * ui));
    const float nui = 0.5f * fmaf(sr + sr, si, fmaf(fr, ui, fi * ur));
    const float tfr = fr + fr, tfi = fi + fi;
    const float ndr = fmaf(tfr, dzr, fmaf(-tfi, dzi, 1.f));
    const float ndi = fmaf(tfr, dzi, tfi * dzr);
    const double tzr = twice_f64(zr);
    const double nzr = fma(zr, zr, fma(-zi, zi, cr));
    const double nzi = fma(tzr, zi, ci);
    zr = nzr; zi = nzi; dzr = ndr; dzi = ndi; ur = nur; ui = nui;
    if (k == lcap) { cap_r = zr; cap_i = zi; capd_r = dzr; capd_i = dzi; capu_r = ur; capu_i = ui; }
  }
  float Ur = ur, Ui = ui;  // P'' / 4^m
  if (lcap >= 0) {
    vr = zr + cap_r; vi = zi + cap_i;
    dr = dzr + capd_r; di = dzi + capd_i;
    const float a = lcap > 0 ? __int_as_float((127 + 2 * (lcap - m)) << 23) : 0.f;  // 4^(lcap - m)
    Ur = fmaf(a, capu_r, ur);
    Ui = fmaf(a, capu_i, ui);
  } else {
    vr = zr; vi = zi; dr = dzr; di = dzi;
  }
  // P''/(2P') = (U 2^(m-1)) / (P' 2^-m), both scalings exact
  const float up = __int_as_float((127 + m - 1) << 23), dn = __int_as_float((127 - m) << 23);
  const float ar = Ur * up, ai = Ui * up, cr2 = dr * dn, ci2 = di * dn;
  const float den = fmaf(cr2, cr2, ci2 * ci2);
  const float inv = 1.f / den;
  kr = fmaf(ar, cr2, ai * ci2) * inv;
  ki = fmaf(ai, cr2, -ar * ci2) * inv;
}

// q_{l,n} as a product.  eq. polySimple gives s_{j,n} = q_{j,n} / q_{j-1,n},
// and q_{0,n} = p_n, so q_{l,n} = p_n prod_{j=1..l} s_{j,n}: with u_k =
// z_{k+n} - z_k (u_0 = p_n), u_{k+1} = z_{k+n}^2 - z_k^2 = u_k (z_{k+n} + z_k),
// and u_l = q_{l,n}.  Every factor has simple roots only, so near a multiple
// root of q -- where the difference p_{l+n} - p_l cancels to rounding noise
// within ~(unit roundoff)^(1/mu) of it -- the product keeps its relative
// accuracy, and Newton reaches the multiple root in binary64.  Two orbits n
// apart: n + 2l orbit steps and l complex product updates.
__device__ __forceinline__ void orbit_q_f64(int l, int n, double cr, double ci, double& vr, double& vi,
                                            double& dr, double& di) {
  double br = 0.0, bi = 0.0, dbr = 0.0, dbi = 0.0;  // z_{k+n}, z'_{k+n}
  for (int k = 1; k <= n; ++k) {
    const double tzr = twice_f64(br), tzi = twice_f64(bi);
    const double ndr = fma(tzr, dbr, fma(-tzi, dbi, 1.0));
    const double ndi = fma(tzr, dbi, tzi * dbr);
    const double nzr = fma(br, br, fma(-bi, bi, cr));
    const double nzi = fma(tzr, bi, ci);
    br = nzr; bi = nzi; dbr = ndr; dbi = ndi;
  }
  double ar = 0.0, ai = 0.0, dar = 0.0, dai = 0.0;  // z_k, z'_k
  double ur = br, ui = bi, dur = dbr, dui = dbi;     // u_0 = p_n, u_0'
  for (int k = 0; k < l; ++k) {
    const double fr = br + ar, fi = bi + ai, dfr = dbr + dar, dfi = dbi + dai;
    const double ndur = fma(dur, fr, fma(-dui, fi, fma(ur, dfr, -ui * dfi)));  // (u f)' = u' f + u f'
    const double ndui = fma(dur, fi, fma(dui, fr, fma(ur, dfi, ui * dfr)));
    const double nur = fma(ur, fr, -ui * fi);
    const double nui = fma(ur, fi, ui * fr);
    ur = nur; ui = nui; dur = ndur; dui = ndui;
    {
      const double tzr = ar + ar, tzi = ai + ai;
      const double ndr = fma(tzr, dar, fma(-tzi, dai, 1.0));
      const double ndi = fma(tzr, dai, tzi * dar);
      const double nzr = fma(ar, ar, fma(-ai, ai, cr));
      const double nzi = fma(tzr, ai, ci);
      ar = nzr; ai = nzi; dar = ndr; dai = ndi;
    }
    {
      const double tzr = twice_f64(br), tzi = twice_f64(bi);
      const double ndr = fma(tzr, dbr, fma(-tzi, dbi, 1.0));
      const double ndi = fma(tzr, dbi, tzi * dbr);
      const double nzr = fma(br, br, fma(-bi, bi, cr));
      const double nzi = fma(tzr, bi, ci);
      br = nzr; bi = nzi; dbr = ndr; dbi = ndi;
    }
  }
  vr = ur; vi = ui; dr = dur; di = dui;
}

// Sign of the captured orbit value in P: +1 for s_{l,n}, -1 for q_{l,n}.
__device__ __forceinline__ double cap_sign(const PolyDev& P) { return P.kind == 2 ? -1.0 : 1.0; }

__device__ __forceinline__ void eval_P(const PolyDev& P, double cr, double ci, double& vr, double& vi,
                                       double& dr, double& di) {
  if (P.kind == 2) orbit_q_f64(P.l, P.n, cr, ci, vr, vi, dr, di);
  else if (P.lcap < 0) orbit_pn_f64(P.m, cr, ci, vr, vi, dr, di);
  else orbit_f64(P.m, P.lcap, 1.0, cr, ci, vr, vi, dr, di);
}

// Newton quotient (a + ib) / (c + id) with one binary64 division.  When
// |c + id|^2 leaves [1e-290, 1e290] (an escaped orbit has |P'| > 1e154 and
// would give a zero quotient, a false convergence), both operands are first
// scaled by the same power of two 2^-E, E the exponent of max(|c|, |d|)
// (exact): the "simplify a common large factor" guard of Sec. 6.3.2 (remark
// on the exponent range).  Non-finite inputs give NaN.
// Non-negative binary64 values (+0 up to +inf) order as their bit patterns
// read as signed 64-bit integers, so such compares can run on the integer
// pipe instead of the binary64 one.  A NaN of either sign falls outside
// [ord(+0), ord(+inf)].
__device__ __forceinline__ long long ord_f64(double x) { return __double_as_longlong(x); }
constexpr long long ORD_1E290 = 0x7c2485ce9e7a065fll;   // ord_f64(1e290)
constexpr long long ORD_1EM290 = 0x03b8f2b061aea072ll;  // ord_f64(1e-290)
constexpr long long ORD_QUARTER = 2ll << 52;            // ord(x) - ORD_QUARTER = ord(x / 4), x/4 normal

__device__ __forceinline__ void cdiv_f64(double a, double b, double c, double d, double& qr,
                                         double& qi) {
  double den = fma(c, c, d * d);  // in [+0, +inf], or NaN
  const long long od = ord_f64(den);
  if (!(od <= ORD_1E290 && od >= ORD_1EM290)) {
    const double m = fmax(fabs(c), fabs(d));
    const long long eb = __double_as_longlong(m) & 0x7ff0000000000000ll;
    const double sc = __longlong_as_double(0x7fe0000000000000ll - eb);  // 2^-E
    c *= sc;
    d *= sc;
    a *= sc;
    b *= sc;
    den = fma(c, c, d * d);
    if (!(m < 1.0e308)) den = __longlong_as_double(0x7ff8000000000000ll);  // inf / NaN input
  }
  const double inv = 1.0 / den;
  qr = fma(a, c, b * d) * inv;
  qi = fma(b, c, -a * d) * inv;
}

// Both finite: exponent fields below all-ones (integer test on the high words).
__device__ __forceinline__ bool finite2(double a, double b) {
  return ((__double2hiint(a) & 0x7ff00000) != 0x7ff00000) &&
         ((__double2hiint(b) & 0x7ff00000) != 0x7ff00000);
}

// e^{2 i pi num / den} for integers with den a power of two <= 2^62.
__device__ __forceinline__ void unit_phase(uint64_t num, uint64_t den, double& c, double& s) {
  const uint64_t r = num & (den - 1);
  sincospi(2.0 * ((double)r / (double)den), &s, &c);
}

// Squared rounding floor of a binary64 Newton step at z: (16 ulp(1 + |z|))^2.
__device__ __forceinline__ double floor2_f64(double zr, double zi) {
  const double a = (1.0 + fabs(zr) + fabs(zi)) * 3.552713678800501e-15;  // 16 * 2^-52
  return a * a;
}

// ---------------------------------------------------------------------------
// Warp helpers.
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Min / max of per-lane 64-bit values over the warp, applied once to *dst
// (all 32 lanes call; a lane with nothing to report passes the neutral
// value ~0 for min, 0 for max).  One atomic per warp instead of per lane:
// per-lane atomics on one address serialise in L2.
__device__ __forceinline__ void warp_min_u64(unsigned long long* dst, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(dst, v);
}
__device__ __forceinline__ void warp_max_u64(unsigned long long* dst, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(dst, v);
}

// Sum a per-lane 64-bit counter over the warp and add it once to *dst.
__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Order-preserving map of a binary64 to an unsigned 64-bit key.
__device__ __forceinline__ uint64_t f64_key(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// f64_key with -0 mapped to +0: for non-NaN binary64 values a < b exactly
// when f64_key0(a) < f64_key0(b)
__device__ __forceinline__ uint64_t f64_key0(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  if ((b << 1) == 0) b = 0;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

}  // namespace mt
