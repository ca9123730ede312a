// mt_levelline.cu -- steps a1-a3 of the path: the discrete level line.
//
// Level line (Sec. 4.1): for |zeta0| above the critical values of P, the
// solution lambda(t) of lambda' = i P/P' satisfies P(lambda(t)) = e^{it}
// zeta0 (eq. LevelLinesFlowSol); the discrete level line L_{zeta0,N}(P)
// samples it at N equal phase steps (eq. defDiscreteLev), and
// P^{-1}(zeta0) = L_{zeta0, deg P}(P).  We index points by the external
// angle t in [0, 1): the point z(t) satisfies P(z(t)) = lambda0 e^{2 i pi d t}
// and t = 0 is the real end point c > 0 (Sec. 6.3.1).
//
// GB300 design.  The paper walks the fine line sequentially on one core
// (hypQuick) or splits it into jobs seeded from a coarse line lifted through
// the nested family p_k -> p_{k+1} (Sec. 4.2, "p_17(z_j) = lambda0^2 + z_j").
// Here every lane is one job: k_seed_lift computes the seed of chunk j at
// t = j / N0 by lifting the circle |p_1| = lambda0 level by level, and
// k_walk walks the chunk [j/N0, (j+1)/N0] with M Newton-with-target
// sub-steps per turn (Prop. computeLevelLine), writing every (M / c_L)-th
// point as a descent start, and checks that it ends on the next seed (a
// skip of a turn -- the failure named in Sec. 6.4.1 -- shows up there).
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

// a1 + a2: seeds at t = j / N0, j = 0 .. N0/2, lifted through the nested
// family (Sec. 4.2): from z on |p_k| = lambda0 at phase 2 pi d_k t, solve
// p_{k+1} = lambda0^2 e^{2 i pi d_{k+1} t} (valid start since
// p_{k+1}(z) = lambda0^2 e^{...} + z), then shrink the modulus back to
// lambda0 along the iso-angle ray in 'shrink' geometric steps.  For
// s_{l,n}, a final homotopy p_m + alpha p_{l-1}, alpha: 0 -> 1, at fixed
// target moves the point from |p_m| = lambda0 to |s_{l,n}| = lambda0.
__global__ void k_seed_lift(PolyDev P, double lambda0, int64_t N0, int log2N0, int shrink,
                            double2* seeds, DevCounters* ctr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0;
  if (j <= N0 / 2) {
    double c, s;
    unit_phase((uint64_t)j, (uint64_t)N0, c, s);
    double zr = lambda0 * c, zi = lambda0 * s;  // |p_1| = |c| = lambda0 at angle t
    const double lam2 = lambda0 * lambda0;
    for (int k = 1; k < P.m; ++k) {
      // phase of level k+1: d_{k+1} t = 2^k j / N0 (exact in integers)
      const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
      unit_phase(num, (uint64_t)N0, c, s);
      steps += newton_target_f64(k + 1, -1, 0.0, zr, zi, lam2 * c, lam2 * s, 1e-3, 40, nullptr);
      const double Lq = -log(lambda0) / shrink;  // log of the radius ratio per shrink step
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
    seeds[j] = make_double2(zr, zi);
  }
  warp_add_u64(&ctr->walk_newton, steps);
}

// a3: walk chunk j = [j/N0, (j+1)/N0] in L sub-steps of 1/M turn
// (sub-step g has P = lambda0 e^{2 i pi g / M}); every 'every'-th point is a
// descent start with index g / every.
__global__ void k_walk(PolyDev P, double lambda0, int M, int every, int64_t L, int64_t nchunks,
                       const double2* __restrict__ seeds, double2* __restrict__ starts,
                       DevCounters* ctr) {
  __shared__ double2 ph[64];
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double c, s;
    unit_phase((uint64_t)q, (uint64_t)M, c, s);
    ph[q] = make_double2(lambda0 * c, lambda0 * s);
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, fails = 0;
  if (j < nchunks) {
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
    if (!(er * er + ei * ei <= 0.0625 * h * h + 1e-28)) fails = 1;
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

cudaError_t launch_seed_lift(const PolyDev& P, double lambda0, int64_t N0, int shrink_steps,
                             double2* seeds, DevCounters* ctr, cudaStream_t s) {
  int log2N0 = 0;
  while ((int64_t(1) << log2N0) < N0) ++log2N0;
  const int64_t n = N0 / 2 + 1;
  const int bs = 128;
  const int64_t grid = (n + bs - 1) / bs;
  MT_COUNT_LAUNCH(1);
  k_seed_lift<<<(unsigned)grid, bs, 0, s>>>(P, lambda0, N0, log2N0, shrink_steps, seeds, ctr);
  return cudaGetLastError();
}

cudaError_t launch_walk(const PolyDev& P, double lambda0, int M, int every, int64_t L,
                        int64_t nchunks, const double2* seeds, double2* starts, DevCounters* ctr,
                        cudaStream_t s) {
  const int bs = 64;
  const int64_t grid = (nchunks + bs - 1) / bs;
  MT_COUNT_LAUNCH(1);
  k_walk<<<(unsigned)grid, bs, 0, s>>>(P, lambda0, M, every, L, nchunks, seeds, starts, ctr);
  return cudaGetLastError();
}

}  // namespace mt
