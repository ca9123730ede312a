// mt_levelline.cuh -- device functions of steps a1-a3 (the discrete level
// line), shared by the single-polynomial kernels (mt_levelline.cu) and the
// batched ones (mt_batch.cu).
#pragma once
#include "mt_common.cuh"

namespace mt {

// Newton map with target (Sec. 4.1): iterate z <- z - (P_alpha(z) - T) / P_alpha'(z).
//
// Predictor.  When the previous target Tp and L = log(T / Tp) are known
// (pred = true), the first step solves log P = log T instead of P = T:
//   z <- z + P log(T / P) / P',   log(T / P) ~ L + (Tp - P) / P,
// i.e. an Euler step of the level-line ODE lambda' = i P / P' (eq.
// LevelLinesFlow; L = i 2 pi / M for a walk sub-step) or of the Newton flow
// (real L for a radial shrink).  log P is d times less curved than P near
// the line, so the predictor lands almost on the target and one Newton
// correction usually meets the tolerance (a chord step P -> T leaves an
// error of order |L|^2 / 2 that needs ~4 more steps).
//
// Stop once a step falls below rel * h (h = the predictor's length; errors
// never accumulate along the walk because every target is an exact phase),
// or when steps stop shrinking after the third (rounding floor).  Returns
// the number of Newton steps; *first receives h.
__device__ __forceinline__ int newton_target_f64(int m, int lcap, double alpha, double& zr,
                                                 double& zi, double tr, double ti, double rel,
                                                 int cap, double* first, bool pred = false,
                                                 double tpr = 0.0, double tpi = 0.0,
                                                 double Lr = 0.0, double Li = 0.0) {
  double thr2 = 0.0, prev2 = 0.0, h2 = 0.0;
  int it = 0;
  while (it < cap) {
    double vr, vi, dr, di;
    if (lcap < 0) orbit_pn_f64(m, zr, zi, vr, vi, dr, di);
    else orbit_f64(m, lcap, alpha, zr, zi, vr, vi, dr, di);
    double nr, ni;
    if (it == 0 && pred) {  // P - Tp - L P
      nr = (vr - tpr) - fma(Lr, vr, -Li * vi);
      ni = (vi - tpi) - fma(Lr, vi, Li * vr);
    } else {
      nr = vr - tr;
      ni = vi - ti;
    }
    double qr, qi;
    cdiv_f64(nr, ni, dr, di, qr, qi);
    if (!finite2(qr, qi)) break;
    zr -= qr;
    zi -= qi;
    ++it;
    const double s2 = fma(qr, qr, qi * qi);
    if (it == 1) {
      h2 = s2;
      thr2 = rel * rel * s2;
    } else if (s2 <= thr2 || (it >= 3 && s2 > 0.25 * prev2)) {
      break;  // converged, or at the rounding floor
    }
    prev2 = s2;
  }
  if (first) *first = sqrt(h2);
  return it;
}

// a1 + a2: the seed at t = j / N0 (j = 0 .. N0/2), lifted through the
// nested family (Sec. 4.2): from z on |p_k| = lambda0 at phase 2 pi d_k t,
// solve p_{k+1} = lambda0^2 e^{2 i pi d_{k+1} t} (a valid start since
// p_{k+1}(z) = lambda0^2 e^{...} + z), then shrink the modulus back to
// lambda0 along the iso-angle ray in 'shrink' geometric steps.  For
// s_{l,n}, a final homotopy p_m + alpha p_{l-1}, alpha: 0 -> 1, at fixed
// target moves the point from |p_m| = lambda0 to |s_{l,n}| = lambda0.
__device__ __forceinline__ double2 lift_seed(const PolyDev& P, double lambda0, int64_t N0,
                                             int log2N0, int shrink, int64_t j,
                                             unsigned long long& steps) {
  double c, s;
  unit_phase((uint64_t)j, (uint64_t)N0, c, s);
  double zr = lambda0 * c, zi = lambda0 * s;  // |p_1| = |c| = lambda0 at angle t
  const double lam2 = lambda0 * lambda0;
  const double Lq = -log(lambda0) / shrink;  // log of the radius ratio per shrink step
  for (int k = 1; k < P.m; ++k) {
    // phase of level k+1: d_{k+1} t = 2^k j / N0 (exact in integers)
    const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
    unit_phase(num, (uint64_t)N0, c, s);
    steps += newton_target_f64(k + 1, -1, 0.0, zr, zi, lam2 * c, lam2 * s, 1e-3, 40, nullptr);
    for (int q = 1; q <= shrink; ++q) {
      const double rp = pow(lambda0, 2.0 - (double)(q - 1) / shrink);
      const double r = pow(lambda0, 2.0 - (double)q / shrink);
      steps += newton_target_f64(k + 1, -1, 0.0, zr, zi, r * c, r * s, 1e-3, 40, nullptr, true,
                                 rp * c, rp * s, Lq, 0.0);
    }
  }
  if (P.kind == 1) {
    // homotopy p_m -> p_m + p_{l-1} at target lambda0 e^{2 i pi d t}, d = 2^(m-1)
    const int k = P.m - 1;
    const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
    unit_phase(num, (uint64_t)N0, c, s);
    const int A = 8;
    for (int a = 1; a <= A; ++a) {
      const double alpha = (double)a / A;
      steps += newton_target_f64(P.m, P.lcap, alpha, zr, zi, lambda0 * c, lambda0 * s, 1e-3, 40,
                                 nullptr);
    }
  }
  if (j == 0 || j == N0 / 2) zi = 0.0;  // the two real end points of the line
  return make_double2(zr, zi);
}

// a3: walk chunk j = [j/N0, (j+1)/N0] in L sub-steps of 1/M turn (sub-step
// g has P = lambda0 e^{2 i pi g / M}, ph[q] = lambda0 e^{2 i pi q / M});
// every 'every'-th point is a descent start with index g / every.  Returns
// true if the chunk did not end on the next seed (a skipped turn).
__device__ __forceinline__ bool walk_chunk(const PolyDev& P, const double2* ph, int M, int every,
                                           int64_t L, int64_t nchunks, int64_t j,
                                           const double2* __restrict__ seeds,
                                           double2* __restrict__ starts,
                                           unsigned long long& steps) {
  const double2 z0 = seeds[j];
  double zr = z0.x, zi = z0.y;
  uint64_t g = (uint64_t)j * (uint64_t)L;
  double h = 0.0;
  const double Li = 6.283185307179586 / M;  // L = log(T / Tp) = i 2 pi / M
  for (int64_t i = 0; i < L; ++i, ++g) {
    if ((g & (uint64_t)(every - 1)) == 0) starts[g / every] = make_double2(zr, zi);
    const double2 Tp = ph[g & (uint64_t)(M - 1)];
    const double2 T = ph[(g + 1) & (uint64_t)(M - 1)];
    steps += newton_target_f64(P.m, P.lcap, 1.0, zr, zi, T.x, T.y, 1e-2, 16, &h, true, Tp.x, Tp.y,
                               0.0, Li);
  }
  if (j == nchunks - 1) starts[g / every] = make_double2(zr, 0.0);  // t = 1/2, real
  const double2 zn = seeds[j + 1];
  const double er = zr - zn.x, ei = zi - zn.y;
  // the end of the chunk must be the next seed, not a neighbour one turn away
  return !(er * er + ei * ei <= 0.0625 * h * h + 1e-28);
}

}  // namespace mt
