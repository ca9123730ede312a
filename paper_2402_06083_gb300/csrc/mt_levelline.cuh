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

// Radii lambda0^(2 - i / shrink), i = 0 .. shrink, of the iso-angle shrink
// steps of the lift: the same at every level, so a seed computes them once
// (shrink + 1 binary64 pow calls instead of 2 shrink per level).  Larger
// shrink counts (late retries) evaluate them in place.
constexpr int LIFT_RADII = 65;

__device__ __forceinline__ bool shrink_radii(double lambda0, int shrink, double* R) {
  if (shrink >= LIFT_RADII) return false;
  for (int i = 0; i <= shrink; ++i) R[i] = pow(lambda0, 2.0 - (double)i / shrink);
  return true;
}

__device__ __forceinline__ double shrink_radius(const double* R, bool tab, double lambda0, int shrink,
                                                int i) {
  return tab ? R[i] : pow(lambda0, 2.0 - (double)i / shrink);
}

// a1 + a2: the seed at t = j / N0 (j = 0 .. N0/2), lifted through the
// nested family (Sec. 4.2): a point z on |p_k| = lambda0 at phase 2 pi d_k t
// satisfies p_{k+1}(z) = lambda0^2 e^{2 i pi d_{k+1} t} + z, i.e. it lies
// |z| away from the ray of phase 2 pi d_{k+1} t at radius lambda0^2.  The
// radius is brought back to lambda0 along that iso-angle ray in 'shrink'
// geometric steps, the first of which also removes the |z| offset (its
// log-space predictor corrects toward the exact previous target).  Solves
// below the last level stop at 1e-2 of their predictor, the last level at
// 1e-3 (the seed is a start of the walk).  For s_{l,n}, a final homotopy
// p_m + alpha p_{l-1}, alpha: 0 -> 1, at fixed target moves the point from
// |p_m| = lambda0 to |s_{l,n}| = lambda0 (p_m - alpha p_l for q_{l,n}).  A seed that lands on the wrong
// preimage makes the walk of its chunk miss the next seed (walk_fail).
__device__ __forceinline__ double2 lift_seed(const PolyDev& P, double lambda0, int64_t N0,
                                             int log2N0, int shrink, int64_t j,
                                             unsigned long long& steps) {
  double c, s;
  unit_phase((uint64_t)j, (uint64_t)N0, c, s);
  double zr = lambda0 * c, zi = lambda0 * s;  // |p_1| = |c| = lambda0 at angle t
  const double Lq = -log(lambda0) / shrink;  // log of the radius ratio per shrink step
  double R[LIFT_RADII];
  const bool tab = shrink_radii(lambda0, shrink, R);
  for (int k = 1; k < P.m; ++k) {
    // phase of level k+1: d_{k+1} t = 2^k j / N0 (exact in integers)
    const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
    unit_phase(num, (uint64_t)N0, c, s);
    const double rel = (k + 1 < P.m) ? 1e-2 : 1e-3;
    for (int q = 1; q <= shrink; ++q) {
      const double rp = shrink_radius(R, tab, lambda0, shrink, q - 1);
      const double r = shrink_radius(R, tab, lambda0, shrink, q);
      steps += newton_target_f64(k + 1, -1, 0.0, zr, zi, r * c, r * s, rel, 40, nullptr, true, rp * c,
                                 rp * s, Lq, 0.0);
    }
  }
  if (P.kind != 0) {
    // homotopy p_m -> p_m + p_{l-1} (s_{l,n}) or p_m - p_l (q_{l,n}) at target
    // lambda0 e^{2 i pi d t}, d = 2^(m-1)
    const int k = P.m - 1;
    const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
    unit_phase(num, (uint64_t)N0, c, s);
    const int A = 8;
    for (int a = 1; a <= A; ++a) {
      const double alpha = cap_sign(P) * a / A;
      steps += newton_target_f64(P.m, P.lcap, alpha, zr, zi, lambda0 * c, lambda0 * s, 1e-3, 40,
                                 nullptr);
    }
  }
  if (j == 0 || j == N0 / 2) zi = 0.0;  // the two real end points of the line
  return make_double2(zr, zi);
}

// One walk sub-step (Prop. computeLevelLine): from z near the previous
// target Tp to P(z) = T, T = Tp e^{L}, L = i 2 pi / M.  In w = log P the
// level line is straight and dz/dw = P / P'.  The predictor is a second-
// order Taylor step in w: dz = z' dw + z'' dw^2 / 2 with dw = L - (P - Tp)/P
// (the log of T / P to first order) and z'' estimated from z' at this and
// the previous sub-step (zp, zp_prev, one step dw ~ L apart).  Newton with
// target T then corrects until a step falls below rel * h (h = predictor
// length) or steps stop shrinking after the third.  Returns the number of
// Newton evaluations; zp receives z' at this sub-step's first point.
__device__ __forceinline__ int walk_substep_f64(int m, int lcap, double sgn, double& zr, double& zi, double tr,
                                                double ti, double tpr, double tpi, double Li,
                                                bool have_prev, double& zpr, double& zpi,
                                                double rel, int cap, double& h) {
  double thr2 = 0.0, prev2 = 0.0, h2 = 0.0;
  int it = 0;
  while (it < cap) {
    double vr, vi, dr, di;
    if (lcap < 0) orbit_pn_f64(m, zr, zi, vr, vi, dr, di);
    else orbit_f64(m, lcap, sgn, zr, zi, vr, vi, dr, di);
    double qr, qi;
    if (it == 0) {
      // z' = P / P' and dz = z' (L - (P - Tp) / P) + (z' - z'_prev) L / 2
      double wr, wi;
      cdiv_f64(vr, vi, dr, di, wr, wi);            // z'
      double er, ei;
      cdiv_f64(vr - tpr, vi - tpi, dr, di, er, ei);  // (P - Tp) / P'
      // -dz = (P - Tp)/P' - z' L - (z' - z'_prev) L / 2
      qr = er + wi * Li;
      qi = ei - wr * Li;
      if (have_prev) {
        qr += 0.5 * (wi - zpi) * Li;
        qi -= 0.5 * (wr - zpr) * Li;
      }
      zpr = wr;
      zpi = wi;
    } else {
      cdiv_f64(vr - tr, vi - ti, dr, di, qr, qi);
    }
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
  h = sqrt(h2);
  return it;
}

// a3: walk chunk j = [j/N0, (j+1)/N0] in L sub-steps of 1/M turn (sub-step
// g has P = lambda0 e^{2 i pi g / M}, ph[q] = lambda0 e^{2 i pi q / M});
// every 'every'-th point is a descent start with index g / every.  Returns
// true if the chunk did not end on the next seed (a skipped turn).
__device__ __forceinline__ bool walk_chunk_from(const PolyDev& P, const double2* ph, int M, int every,
                                                int64_t L, int64_t nchunks, int64_t j, double2 z0,
                                                double2 zn, double2* __restrict__ starts,
                                                unsigned long long& steps, int64_t sbase = 0) {
  double zr = z0.x, zi = z0.y;
  uint64_t g = (uint64_t)j * (uint64_t)L;
  double h = 0.0, zpr = 0.0, zpi = 0.0;
  const double Li = 6.283185307179586 / M;  // L = log(T / Tp) = i 2 pi / M
  for (int64_t i = 0; i < L; ++i, ++g) {
    if ((g & (uint64_t)(every - 1)) == 0) starts[(int64_t)(g / every) - sbase] = make_double2(zr, zi);
    const double2 Tp = ph[g & (uint64_t)(M - 1)];
    const double2 T = ph[(g + 1) & (uint64_t)(M - 1)];
    // a sub-step that ends on a start converges to 1e-2 of its predictor;
    // the others to 1e-1 (the next predictor corrects toward the exact
    // previous target, so their error does not carry over)
    const double rel = (((g + 1) & (uint64_t)(every - 1)) == 0) ? 1e-2 : 1e-1;
    steps += walk_substep_f64(P.m, P.lcap, cap_sign(P), zr, zi, T.x, T.y, Tp.x, Tp.y, Li, i > 0, zpr, zpi, rel,
                              16, h);
  }
  if (j == nchunks - 1) starts[(int64_t)(g / every) - sbase] = make_double2(zr, 0.0);  // t = 1/2, real
  const double er = zr - zn.x, ei = zi - zn.y;
  // the end of the chunk must be the next seed, not a neighbour one turn away
  return !(er * er + ei * ei <= 0.0625 * h * h + 1e-28);
}

__device__ __forceinline__ bool walk_chunk(const PolyDev& P, const double2* ph, int M, int every,
                                           int64_t L, int64_t nchunks, int64_t j,
                                           const double2* __restrict__ seeds,
                                           double2* __restrict__ starts,
                                           unsigned long long& steps) {
  return walk_chunk_from(P, ph, M, every, L, nchunks, j, seeds[j], seeds[j + 1], starts, steps);
}

}  // namespace mt
