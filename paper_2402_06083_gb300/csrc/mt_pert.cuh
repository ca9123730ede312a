// mt_pert.cuh -- binary32 perturbation orbits around a reference orbit
// (the mixed tier's walk and descents, and the double-double pass's walk
// and descents).  With Z_k the orbit of the anchor c0 (kept in shared
// memory as binary32) and c = c0 + delta,
//   e_{k+1} = (2 Z_k + e_k) e_k + delta,   p_k(c) = Z_k + e_k,
// so binary32 carries only the difference from the anchor and its relative
// precision applies to |delta|, not to |c| (the published perturbation
// technique of deep-zoom Mandelbrot renderers).  The derivative is carried
// as g_k = p'_k / 2^k.
#pragma once
#include "mt_common.cuh"

namespace mt {

// pert_eval for the descents and the walk.  z1 points to row 1 of the
// lane's orbit column (row k at z1[(k - 1) * STRIDE]); row 0 is Z_0 = 0, so
// the first step is exact and skipped: e_1 = delta, g_1 = 2^-1.  STRIDE: the
// shared-memory row stride (a compile-time constant, so each row's load
// takes an immediate offset).  MC: the orbit length when known at compile
// time (p_n, m = n: the loop is fully unrolled and 2^-(k+1) is an
// immediate), else 0 (P.m, unrolled by four).  The capture of p_lcap is
// compiled in only where the polynomial has one (s_{l,n}).
template <bool CAP, int MC, int STRIDE>
__device__ __forceinline__ void pert_eval_t(const PolyDev& P, const float2* z1, float dx, float dy, float& ex,
                                            float& ey, float& Dx, float& Dy) {
  float e_x = dx, e_y = dy, g_x = 0.5f, g_y = 0.f;
  float ce_x = 0.f, ce_y = 0.f, cg_x = 0.f, cg_y = 0.f;
  if (CAP && P.lcap == 1) { ce_x = e_x; ce_y = e_y; cg_x = g_x; cg_y = g_y; }
  auto step = [&](int k, float h) {
    const float2 Z = z1[(k - 1) * STRIDE];
    const float zx = Z.x + e_x, zy = Z.y + e_y;  // p_k(c)
    const float ng_x = fmaf(zx, g_x, fmaf(-zy, g_y, h));
    const float ng_y = fmaf(zx, g_y, zy * g_x);
    const float sx = Z.x + zx, sy = Z.y + zy;  // 2 Z_k + e_k
    const float ne_x = fmaf(sx, e_x, fmaf(-sy, e_y, dx));
    const float ne_y = fmaf(sx, e_y, fmaf(sy, e_x, dy));
    e_x = ne_x; e_y = ne_y; g_x = ng_x; g_y = ng_y;
    if (CAP && k + 1 == P.lcap) { ce_x = e_x; ce_y = e_y; cg_x = g_x; cg_y = g_y; }
  };
  if constexpr (MC > 0) {
#pragma unroll
    for (int k = 1; k < MC; ++k) step(k, __int_as_float((126 - k) << 23));  // 2^-(k+1)
  } else {
    int hexp = (127 - 2) << 23;  // exponent field of 2^-(k+1), k = 1
#pragma unroll 4
    for (int k = 1; k < P.m; ++k) {
      step(k, __int_as_float(hexp));
      hexp -= 1 << 23;
    }
  }
  const int m = MC > 0 ? MC : P.m;
  const float sc = __int_as_float((127 + m) << 23);
  if (CAP) {
    ex = e_x + ce_x;
    ey = e_y + ce_y;
    const float a = P.lcap > 0 ? __int_as_float((127 + P.lcap - m) << 23) : 0.f;
    Dx = fmaf(a, cg_x, g_x) * sc;
    Dy = fmaf(a, cg_y, g_y) * sc;
  } else {
    ex = e_x;
    ey = e_y;
    Dx = g_x * sc;
    Dy = g_y * sc;
  }
}


// binary32 quotient; false when |D|^2 leaves the safe binary32 range.
__device__ __forceinline__ bool cdiv_f32(float a, float b, float c, float d, float& qr, float& qi) {
  const float den = fmaf(c, c, d * d);
  if (!(den < 1e36f && den > 1e-36f)) return false;
  const float inv = __frcp_rn(den);
  qr = fmaf(a, c, b * d) * inv;
  qi = fmaf(b, c, -a * d) * inv;
  return isfinite(qr) && isfinite(qi);
}

// newton_target_pert on the descents' orbit loop (compile-time stride and,
// for p_n, orbit length).
// WIDE: the quotient by cdiv_f32s (no binary32 range limit on P'; the
// double-double pass's walk, where |P'| passes 1e18 at p_32).
template <bool CAP, int MC, int STRIDE, bool WIDE = false>
__device__ __forceinline__ int newton_target_walk(const PolyDev& P, const float2* zs, const float4& v, float& dx,
                                                  float& dy, float tx, float ty, float rel, int cap, float* first,
                                                  float tpx, float tpy, float Li, bool* bad, float Lr = 0.f,
                                                  bool pred = true) {
  float thr2 = 0.f, prev2 = 0.f, h2 = 0.f;
  int it = 0;
  while (it < cap) {
    float ex, ey, Dx, Dy;
    pert_eval_t<CAP, MC, STRIDE>(P, zs + STRIDE, dx, dy, ex, ey, Dx, Dy);
    float nr, ni;
    if (it == 0 && pred) {  // predictor: P - Tp - L P, L = Lr + i Li
      const float Pr = v.x + (v.z + ex), Pi = v.y + (v.w + ey);
      if (Lr == 0.f) {  // the walk's form
        nr = (Pr - tpx) + Li * Pi;
        ni = (Pi - tpy) - Li * Pr;
      } else {
        nr = (Pr - tpx) - fmaf(Lr, Pr, -Li * Pi);
        ni = (Pi - tpy) - fmaf(Lr, Pi, Li * Pr);
      }
    } else {
      nr = ((v.x - tx) + v.z) + ex;
      ni = ((v.y - ty) + v.w) + ey;
    }
    float qr, qi;
    if (!(WIDE ? cdiv_f32s(nr, ni, Dx, Dy, qr, qi) : cdiv_f32(nr, ni, Dx, Dy, qr, qi))) { *bad = true; break; }
    dx -= qr;
    dy -= qi;
    ++it;
    const float s2 = fmaf(qr, qr, qi * qi);
    if (it == 1) {
      h2 = s2;
      thr2 = rel * rel * s2;
    } else if (s2 <= thr2 || (it >= 3 && s2 > 0.25f * prev2)) {
      break;
    }
    prev2 = s2;
  }
  if (first) *first = sqrtf(h2);
  return it;
}

}  // namespace mt
