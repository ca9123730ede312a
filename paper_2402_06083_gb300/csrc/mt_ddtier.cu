// mt_ddtier.cu -- the double-double tier (MT_DD): roots clustered closer
// than binary64 can resolve (the two left-most real roots of p_28 lie
// 118.4 / 4^28 = 1.6e-15 apart, four ulps of 2; Sec. 6.3.2).
//
// The paper switches to MPFR "only when necessary" (Sec. 1.1) and refines
// the roots near the real axis left of -2 + 4^-16 in high precision (Sec.
// 6.3.2).  Here the need is detected, not assumed: a binary64 / mixed pass
// runs first; its root set merges candidates closer than the pixel eps, so
// two roots closer than that become one representative.  Such a
// representative either fails its disk certificate (Thm proofRoots: its
// disk holds two roots) or passes only with a disk smaller than ~eps (the
// radius retries of the certificate).  Every representative that failed,
// or whose proven radius is below 2 eps, becomes a zone centre f, and the
// disk D(f, R) is redone in double-double:
//   1. the pieces of the level line (Ls = 32 sub-steps each) whose descents
//      ended within R + margin of a zone centre are walked again in dd,
//      each from its own dd-lifted seed;
//   2. their starts descend in dd; main representatives within R + margin
//      are polished in dd;
//   3. a dd point belongs to the zone iff it lies within R of a centre (the
//      same test for both sources, on the same dd-accurate value, so a root
//      is never counted on both sides of a zone boundary); main
//      representatives whose polished value is in a zone are dropped;
//   4. the zone points form their own separated set (dd comparisons), get
//      dd types and a disk certificate with dd centres, checked disjoint
//      from the certified disks of the kept main representatives;
//   5. both sets are emitted as one list sorted by Re (hi parts), the low
//      parts going to the caller's lo buffer.
// "all" mode makes every root a zone member: the whole split is redone in dd.
#include "mt_dd.cuh"
#include "mt_pert.cuh"
#include "mt_levelline.cuh"

namespace mt {

// ---- zone membership -------------------------------------------------------------

// nbad < 0: every point is in the zone ("all" mode).  bad is sorted by Re.
__device__ __forceinline__ bool zone_hit(double x, double y, const double2* __restrict__ bad,
                                         int nbad, double R) {
  if (nbad < 0) return true;
  int lo = 0, hi = nbad;
  // first centre with Re >= x - R, searched on order-preserving integer keys
  // (GB300's binary64 pipe is the scarce one; the comparisons of the search
  // run on the integer pipe)
  const uint64_t kl = f64_key(x - R), kh = f64_key(x + R);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (f64_key(bad[mid].x) < kl) lo = mid + 1; else hi = mid;
  }
  const double R2 = R * R;
  for (int f = lo; f < nbad && f64_key(bad[f].x) <= kh; ++f) {
    const double dx = x - bad[f].x, dy = y - bad[f].y;
    if (fma(dx, dx, dy * dy) < R2) return true;
  }
  return false;
}

// zone_hit for the bulk tests (every start, every representative): the
// centres' windows [x_f - R', x_f + R'] (R' = R (1 + 2^-30), so the windows
// hold every point the exact test below accepts) as order-preserving integer
// keys from the host, klo and khi both sorted like the centres.  The first
// centre whose window reaches x is a binary search on khi, the last one the
// first klo above x; only the exact test runs in binary64.
__device__ __forceinline__ bool zone_hit_k(double x, double y, const double2* __restrict__ bad,
                                           const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi,
                                           int nbad, double R) {
  if (nbad < 0) return true;  // "all" mode
  const uint64_t kx = f64_key0(x);
  int lo = 0, hi = nbad;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (khi[mid] < kx) lo = mid + 1; else hi = mid;
  }
  const double R2 = R * R;
  for (int f = lo; f < nbad && klo[f] <= kx; ++f) {
    const double dx = x - bad[f].x, dy = y - bad[f].y;
    if (fma(dx, dx, dy * dy) < R2) return true;
  }
  return false;
}

// ulp(x) = 2^(e(x) - 52) for |x| in [2^e, 2^(e+1)); 2^-1074 below 2^-1022
__device__ __forceinline__ double ulp64(double x) {
  const double a = fabs(x);
  if (!(a >= 2.2250738585072014e-308)) return 4.9406564584124654e-324;
  return __longlong_as_double(__double_as_longlong(a) & 0x7ff0000000000000ll) * 2.220446049250313e-16;
}

// dd points are sorted by their hi parts only: within equal (or adjacent) hi
// the lo parts come in any order, so a scan away from a point may stop only
// once the hi parts alone are farther apart than w plus two ulps.
__device__ __forceinline__ bool hi_beyond(double a_hi, double b_hi, double w) {
  return fabs(a_hi - b_hi) > w + 2.0 * ulp64(fmax(fabs(a_hi), fabs(b_hi)));
}

// Representatives that failed, or whose proven radius is below thr.
__global__ void k_collect_bad(const double2* __restrict__ reps, const unsigned long long* n_reps,
                              int64_t cap, const uint8_t* __restrict__ pass,
                              const double* __restrict__ radius, double thr,
                              double2* __restrict__ bad, unsigned long long* nbad, int max_bad) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= cap || u >= (int64_t)*n_reps || (pass[u] && radius[u] >= thr)) return;
  const unsigned long long k = atomicAdd(nbad, 1ull);
  if (k < (unsigned long long)max_bad) bad[k] = reps[u];
}

// Piece G = [G Ls, (G+1) Ls) of the line's sub-steps is redone when a
// descent that started in it (converged or timed out) ended within R of a
// zone centre.
__global__ void k_mark_pieces(const double2* __restrict__ cand, const uint8_t* __restrict__ status,
                              int64_t S, int every, int64_t Ls, int64_t npieces,
                              const double2* __restrict__ bad, const uint64_t* __restrict__ klo,
                              const uint64_t* __restrict__ khi, int nbad, double R,
                              uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S || status[i] == 1) return;
  const double2 c = cand[i];
  if (!finite2(c.x, c.y) || !zone_hit_k(c.x, fabs(c.y), bad, klo, khi, nbad, R)) return;
  int64_t G = (i * (int64_t)every) / Ls;
  if (G >= npieces) G = npieces - 1;
  flag[G] = 1;
}

// Streamed splits: the same from the end points kept in 32-bit fixed point
// (2^-29 per unit, INT_MIN: divergent).  Rounding moved each coordinate by
// at most 2^-30, so the zone test takes a radius grown by 2^-29: a superset
// of the pieces the binary64 test marks.
__global__ void k_mark_pieces_fix(const int2* __restrict__ candq, int64_t S, int every, int64_t Ls,
                                  int64_t npieces, const double2* __restrict__ bad, int nbad, double R,
                                  uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S) return;
  const int2 c = candq[i];
  if (c.x == (int)0x80000000) return;
  const double x = c.x * 1.862645149230957e-09, y = fabs(c.y * 1.862645149230957e-09);  // * 2^-29
  if (!zone_hit(x, y, bad, nbad, R + 1.862645149230957e-09)) return;
  int64_t G = (i * (int64_t)every) / Ls;
  if (G >= npieces) G = npieces - 1;
  flag[G] = 1;
}

// ids[pos[G]] = G for the flagged pieces (pos = exclusive scan of flag);
// flag == nullptr: every piece ("all" mode).  Ids past ids_cap are dropped
// (the host compares the count with the capacity).
__global__ void k_piece_ids(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                            int64_t npieces, int64_t* __restrict__ ids, int64_t ids_cap) {
  const int64_t G = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (G >= npieces) return;
  if (!flag) {
    if (G < ids_cap) ids[G] = G;
  } else if (flag[G] && (int64_t)pos[G] < ids_cap) {
    ids[pos[G]] = G;
  }
}

// Main representatives within R of a centre -> polish list.
__global__ void k_near_reps(const double2* __restrict__ reps, const unsigned long long* n_reps,
                            int64_t cap, const double2* __restrict__ bad, const uint64_t* __restrict__ klo,
                            const uint64_t* __restrict__ khi, int nbad, double R,
                            uint32_t* __restrict__ near, unsigned long long* nnear, int64_t near_cap) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= cap || u >= (int64_t)*n_reps) return;
  const double2 c = reps[u];
  if (!zone_hit_k(c.x, c.y, bad, klo, khi, nbad, R)) return;
  const unsigned long long k = atomicAdd(nnear, 1ull);
  if ((int64_t)k < near_cap) near[k] = (uint32_t)u;
}

__device__ __forceinline__ void push_zone(dd zr, dd zi, dd* __restrict__ zx, dd* __restrict__ zy,
                                          unsigned long long* nz, int64_t zcap) {
  const unsigned long long k = atomicAdd(nz, 1ull);
  if ((int64_t)k < zcap) {
    zx[k] = zr;
    zy[k] = zi;
  }
}

// ---- dd level line of the redone chunks ----------------------------------------------


// The double-double pass's walk and descents in binary32 perturbation
// form (mt_pert.cuh) around double-double anchors.  Near the left tip the
// points of the level line lie closer than binary64 resolves, but the walk
// only has to follow |P| = lambda0 to 1e-2 of a sub-step, and a descent only
// has to reach its root's basin before the double-double finish: what needs
// the 106 bits is the position, which the anchor (double-double) carries,
// not the arithmetic of each step, which binary32 does relative to |delta|.
// The anchor's orbit Z_1 .. Z_{m-1} goes to shared memory in binary32
// (truncated on the integer pipe), P(anchor) as binary32 hi + lo; the
// binary64 pipe then issues one double-double orbit per anchor instead of
// one per Newton step.
template <bool CAP, int STRIDE>
__device__ __forceinline__ void dd_ref_orbit(const PolyDev& P, dd cr, dd ci, float2* zs, float4& v) {
  dd zr = dd_make(0.0), zi = dd_make(0.0), capr = dd_make(0.0), capi = dd_make(0.0);
  zs[0] = make_float2(0.f, 0.f);
  for (int k = 1; k <= P.m; ++k) {
    const dd xx = dd_mul(zr, zr), yy = dd_mul(zi, zi), xy = dd_mul(zr, zi);
    zr = dd_add(dd_sub(xx, yy), cr);
    zi = dd_add(dd_twice(xy), ci);
    if (k < P.m) zs[k * STRIDE] = make_float2(f32_trunc(zr.hi), f32_trunc(zi.hi));
    if (CAP && k == P.lcap) { capr = zr; capi = zi; }
  }
  const dd vr = CAP ? dd_add(zr, capr) : zr, vi = CAP ? dd_add(zi, capi) : zi;
  const float hx = f32_trunc(vr.hi), hy = f32_trunc(vi.hi);
  v = make_float4(hx, hy, f32_trunc((vr.hi - f64_of_f32(hx)) + vr.lo), f32_trunc((vi.hi - f64_of_f32(hy)) + vi.lo));
}

// Seeds of the redone pieces.  Piece k of the batch (line piece ids[k])
// needs the points at t = ids[k] / NQ and (ids[k] + 1) / NQ (NQ = pieces
// around the whole line).  Adjacent redone pieces share their boundary, so
// piece k contributes its start seed and, unless piece k + 1 starts where
// it ends, its end seed: cnt[k] = 1 or 2, off = exclusive scan of cnt, and
// the start seed of piece k is seed off[k], its end seed seed off[k] + 1
// in both cases.
__global__ void k_dd_seed_count(const int64_t* __restrict__ ids, int64_t nb,
                                uint32_t* __restrict__ cnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  cnt[k] = (k + 1 < nb && ids[k + 1] == ids[k] + 1) ? 1u : 2u;
}

// thread (k, e): e = 0 the start seed of piece k, e = 1 its own end seed.
// The lift of the seed through the nested family (Sec. 4.2: at level k a
// Newton solve of p_{k+1} from the level-k point, with the shrink steps back
// to lambda0, as lift_seed) with each level's solves in binary32
// perturbation form around the double-double point reached at the level
// below (dd_ref_orbit of p_{k+1}: one double-double orbit per level instead
// of one per Newton step); a level whose binary32 solves fail is redone by
// double-double solves.  Shared memory: m rows of 32
// binary32 pairs per warp.
__global__ void k_dd_seeds(PolyDev P, double lambda0, int64_t NQ, int log2NQ, int shrink,
                           const int64_t* __restrict__ ids, const uint32_t* __restrict__ cnt,
                           const uint32_t* __restrict__ off, int64_t nb, dd* __restrict__ sx,
                           dd* __restrict__ sy, DevCounters* ctr) {
  extern __shared__ float2 zsh[];
  float2* zs = zsh + (threadIdx.x >> 5) * 32 * P.m + (threadIdx.x & 31);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, s32 = 0;
  const int64_t k = g >> 1;
  const int e = (int)(g & 1);
  if (k < nb && (e == 0 || cnt[k] == 2)) {
    const int64_t jq = ids[k] + e;
    double c, s;
    unit_phase((uint64_t)jq, (uint64_t)NQ, c, s);
    dd zr = dd_make(lambda0 * c), zi = dd_make(lambda0 * s);
    const double Lq = -log(lambda0) / shrink;
    for (int lv = 1; lv < P.m; ++lv) {
      const uint64_t num = (lv >= log2NQ) ? 0 : (((uint64_t)jq << lv) & (uint64_t)(NQ - 1));
      unit_phase(num, (uint64_t)NQ, c, s);
      const double rel = (lv + 1 < P.m) ? 1e-2 : 1e-3;  // as lift_seed
      PolyDev Q;
      Q.kind = 0; Q.l = 0; Q.n = lv + 1; Q.m = lv + 1; Q.lcap = -1; Q.log2d = lv;
      float4 v;
      dd_ref_orbit<false, 32>(Q, zr, zi, zs, v);
      float dx = 0.f, dy = 0.f;
      bool bad = false;
      int it = 0;
      for (int q = 1; q <= shrink && !bad; ++q) {
        const double rp = pow(lambda0, 2.0 - (double)(q - 1) / shrink);
        const double r = pow(lambda0, 2.0 - (double)q / shrink);
        it += newton_target_walk<false, 0, 32, true>(Q, zs, v, dx, dy, (float)(r * c), (float)(r * s), (float)rel,
                                                     40, nullptr, (float)(rp * c), (float)(rp * s), 0.f, &bad,
                                                     (float)Lq, true);
      }
      s32 += it;
      if (!bad) {
        zr = dd_add_d(zr, f64_of_f32(dx));
        zi = dd_add_d(zi, f64_of_f32(dy));
      } else {  // double-double solves from the level's start
        for (int q = 1; q <= shrink; ++q) {
          const double rp = pow(lambda0, 2.0 - (double)(q - 1) / shrink);
          const double r = pow(lambda0, 2.0 - (double)q / shrink);
          steps += newton_target_dd(lv + 1, -1, 0.0, zr, zi, dd_make(r * c), dd_make(r * s), rel, 40, nullptr,
                                    true, rp * c, rp * s, Lq, 0.0);
        }
      }
    }
    if (P.kind == 1) {  // the homotopy p_m -> p_m + p_{l-1}, in double-double
      const int kk = P.m - 1;
      const uint64_t num = (kk >= log2NQ) ? 0 : (((uint64_t)jq << kk) & (uint64_t)(NQ - 1));
      unit_phase(num, (uint64_t)NQ, c, s);
      for (int a = 1; a <= 8; ++a)
        steps += newton_target_dd(P.m, P.lcap, a / 8.0, zr, zi, dd_make(lambda0 * c), dd_make(lambda0 * s), 1e-3,
                                  40, nullptr);
    }
    if (jq == 0 || jq == NQ / 2) zi = dd_make(0.0);
    sx[off[k] + e] = zr;
    sy[off[k] + e] = zi;
  }
  warp_add_u64(&ctr->steps_dd, steps);
  warp_add_u64(&ctr->steps_fp32, s32);
}

// The same walk with every Newton step in double-double (s_{l,n}: at order
// 26 the binary32 walk's starts, valid to the walk's tolerance, left 66 of
// the tip roots of s_{3,23} unfound, so the Misiurewicz family keeps the
// double-double walk).
__global__ void k_dd_walk(PolyDev P, double lambda0, int M, int every, int64_t Ls, int64_t npieces,
                          const int64_t* __restrict__ ids, const uint32_t* __restrict__ off, int64_t nb,
                          const dd* __restrict__ sx, const dd* __restrict__ sy, dd* __restrict__ stx,
                          dd* __restrict__ sty, uint8_t* __restrict__ st_ok, DevCounters* ctr) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, fails = 0;
  if (k < nb) {
    const int64_t G = ids[k];
    const int64_t s0 = off[k];
    dd zr = sx[s0], zi = sy[s0];
    uint64_t g = (uint64_t)G * (uint64_t)Ls;
    double h = 0.0;
    const double Li = 6.283185307179586 / M;
    for (int64_t i = 0; i < Ls; ++i, ++g) {
      if ((g & (uint64_t)(every - 1)) == 0) {
        const int64_t slot = (k * Ls + i) / every;
        stx[slot] = zr;
        sty[slot] = zi;
        st_ok[slot] = 1;
      }
      double c, s, cp, sp;
      unit_phase(g + 1, (uint64_t)M, c, s);
      unit_phase(g, (uint64_t)M, cp, sp);
      const double rel = (((g + 1) & (uint64_t)(every - 1)) == 0) ? 1e-2 : 1e-1;
      steps += newton_target_dd(P.m, P.lcap, 1.0, zr, zi, dd_make(lambda0 * c), dd_make(lambda0 * s), rel,
                                16, &h, true, lambda0 * cp, lambda0 * sp, 0.0, Li);
    }
    const double er = dd_to_d(dd_sub(zr, sx[s0 + 1])), ei = dd_to_d(dd_sub(zi, sy[s0 + 1]));
    if (!(er * er + ei * ei <= 0.0625 * h * h)) fails = 1;
    if (G == npieces - 1) {
      const int64_t slot = (nb * Ls) / every;
      stx[slot] = zr;
      sty[slot] = dd_make(0.0);
      st_ok[slot] = 1;
    }
  }
  warp_add_u64(&ctr->steps_dd, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

// a3 of the dd pass: one lane per piece of Ls sub-steps from its dd seed,
// re-anchored every K sub-steps.  The start of the line's sub-step g =
// ids[k] Ls + i with g % every == 0 goes to slot (k Ls + i) / every, the
// line's last point (t = 1/2, end of the last piece) to slot nb Ls / every.
// A piece whose end misses its end seed (a skipped turn) counts in
// walk_fail.  Shared memory: m rows of 32 binary32 pairs per warp.
template <bool CAP>
__global__ void k_dd_walk_pert(PolyDev P, double lambda0, int M, int every, int64_t Ls, int64_t npieces,
                               const int64_t* __restrict__ ids, const uint32_t* __restrict__ off, int64_t nb,
                               const dd* __restrict__ sx, const dd* __restrict__ sy, dd* __restrict__ stx,
                               dd* __restrict__ sty, uint8_t* __restrict__ st_ok, int K, DevCounters* ctr) {
  extern __shared__ float2 zsh[];
  __shared__ float2 ph[64];
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double c, s;
    unit_phase((uint64_t)q, (uint64_t)M, c, s);
    ph[q] = make_float2((float)(lambda0 * c), (float)(lambda0 * s));
  }
  __syncthreads();
  float2* zs = zsh + (threadIdx.x >> 5) * 32 * P.m + (threadIdx.x & 31);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, fails = 0;
  if (k < nb) {
    const int64_t G = ids[k];
    const int64_t s0 = off[k];
    dd ar = sx[s0], ai = sy[s0];
    float4 v;
    dd_ref_orbit<CAP, 32>(P, ar, ai, zs, v);
    float dx = 0.f, dy = 0.f, h = 0.f;
    bool bad = false;
    const float Li = 6.2831853f / M;
    uint64_t g = (uint64_t)G * (uint64_t)Ls;
    int kc = K;
    for (int64_t i = 0; i < Ls; ++i, ++g) {
      if ((g & (uint64_t)(every - 1)) == 0) {
        const int64_t slot = (k * Ls + i) / every;
        stx[slot] = dd_add_d(ar, f64_of_f32(dx));
        sty[slot] = dd_add_d(ai, f64_of_f32(dy));
        st_ok[slot] = 1;
      }
      const float2 Tp = ph[g & (uint64_t)(M - 1)];
      const float2 T = ph[(g + 1) & (uint64_t)(M - 1)];
      const float rel = (((g + 1) & (uint64_t)(every - 1)) == 0) ? 1e-2f : 1e-1f;
      steps += newton_target_walk<CAP, 0, 32, true>(P, zs, v, dx, dy, T.x, T.y, rel, 16, &h, Tp.x, Tp.y, Li, &bad);
      if (--kc == 0 && i + 1 < Ls) {  // re-anchor at the current point
        kc = K;
        ar = dd_add_d(ar, f64_of_f32(dx));
        ai = dd_add_d(ai, f64_of_f32(dy));
        dx = dy = 0.f;
        dd_ref_orbit<CAP, 32>(P, ar, ai, zs, v);
      }
    }
    const dd fr = dd_add_d(ar, f64_of_f32(dx)), fi = dd_add_d(ai, f64_of_f32(dy));
    const double er = dd_to_d(dd_sub(fr, sx[s0 + 1])), ei = dd_to_d(dd_sub(fi, sy[s0 + 1]));
    const double hh = (double)h;
    if (bad || !(er * er + ei * ei <= 0.0625 * hh * hh)) fails = 1;
    if (G == npieces - 1) {
      const int64_t slot = (nb * Ls) / every;
      stx[slot] = fr;
      sty[slot] = dd_make(0.0);
      st_ok[slot] = 1;
    }
  }
  warp_add_u64(&ctr->steps_fp32, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

// One dd Newton step of eq. Newton; false if the quotient is not finite.
__device__ __forceinline__ bool dd_newton_step(const PolyDev& P, dd& zr, dd& zi, double& s2) {
  dd vr, vi;
  double dr, di, qr, qi;
  orbit_dd(P.m, P.lcap, 1.0, zr, zi, vr, vi, dr, di);
  cdiv_f64(dd_to_d(vr), dd_to_d(vi), dr, di, qr, qi);
  if (!finite2(qr, qi)) return false;
  zr = dd_add_d(zr, -qr);
  zi = dd_add_d(zi, -qi);
  s2 = fma(qr, qr, qi * qi);
  return true;
}

// Stop rule of the dd descents: |step| < tol, or the steps stopped
// shrinking at the dd rounding floor (~1e-30 relative).
__device__ __forceinline__ bool dd_converged(double s2, double prev2, double tol2, const dd& zr,
                                             const dd& zi) {
  const double fl = 1e-30 * (1.0 + fabs(zr.hi) + fabs(zi.hi));
  return s2 < tol2 || (s2 >= 0.25 * prev2 && s2 < fl * fl);
}

// dd descents from the dd starts; converged roots in a zone (folded to the
// upper half, P having real coefficients) are appended to the zone list.
// a4 of the dd pass, one thread per start: double-double Newton steps (eq.
// Newton) from the start to the dd tolerance or the divergence bound.  (A
// binary32 perturbation phase ahead of them, handing over at 1e-2 of the
// descent's scale, measured slower: its divergent lanes cost more than the
// dd steps it saved.)  Converged descents that end in a zone are appended to
// the zone list.
__global__ void __launch_bounds__(64) k_dd_descend(PolyDev P, int64_t count, const dd* __restrict__ zx0,
                                                   const dd* __restrict__ zy0, const uint8_t* __restrict__ ok0,
                                                   double tol2, int cap, const double2* __restrict__ bad,
                                                   int nbad, double R, dd* __restrict__ ox, dd* __restrict__ oy,
                                                   unsigned long long* nout, int64_t out_cap, DevCounters* ctr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long sdd = 0;
  if (i < count && ok0[i]) {
    dd zr = zx0[i], zi = zy0[i];
    // long jump (as k_descend): |c| beyond max(4, 2 |start|)
    const double rdiv2 = fmax(16.0, 4.0 * fma(zr.hi, zr.hi, zi.hi * zi.hi));
    bool conv = false;
    double pv2 = 1e300;
    for (int t = 0; t < cap; ++t) {
      double q2;
      if (!dd_newton_step(P, zr, zi, q2)) break;
      ++sdd;
      if (!(fma(zr.hi, zr.hi, zi.hi * zi.hi) <= rdiv2)) break;
      if (dd_converged(q2, pv2, tol2, zr, zi)) {
        conv = true;
        break;
      }
      pv2 = q2;
    }
    if (conv) {
      if (zi.hi < 0.0) zi = dd_neg(zi);
      if (zone_hit(zr.hi, zi.hi, bad, nbad, R)) push_zone(zr, zi, ox, oy, nout, out_cap);
    }
  }
  warp_add_u64(&ctr->steps_dd, sdd);
}

// dd polish of the main representatives in the polish list.  drop[u] = 1
// when the polished value is in a zone; if the polish failed or jumped
// farther than 'margin' (to another root), the binary64 value decides and
// the polished value is not used.  Polished values in a zone join the zone
// list.
__global__ void k_dd_polish(PolyDev P, const double2* __restrict__ reps,
                            const uint32_t* __restrict__ near, const unsigned long long* nnear,
                            int64_t near_cap, double tol2, const double2* __restrict__ bad, int nbad,
                            double R, double margin, uint8_t* __restrict__ drop, dd* __restrict__ ox,
                            dd* __restrict__ oy, unsigned long long* nout, int64_t out_cap,
                            DevCounters* ctr) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0;
  int64_t nn = (int64_t)*nnear;
  if (nn > near_cap) nn = near_cap;
  if (k < nn) {
    const uint32_t u = near[k];
    const double2 c = reps[u];
    dd zr = dd_make(c.x), zi = dd_make(c.y);
    bool conv = false;
    double prev2 = 1e300;
    for (int it = 0; it < 8; ++it) {
      double s2;
      if (!dd_newton_step(P, zr, zi, s2)) break;
      ++steps;
      if (dd_converged(s2, prev2, tol2, zr, zi)) {
        conv = true;
        break;
      }
      prev2 = s2;
    }
    if (conv) {
      const double mx = zr.hi - c.x, my = zi.hi - c.y;
      conv = fma(mx, mx, my * my) < margin * margin;
    }
    if (conv && zi.hi < 0.0) zi = dd_neg(zi);
    const bool in = conv ? zone_hit(zr.hi, zi.hi, bad, nbad, R) : zone_hit(c.x, c.y, bad, nbad, R);
    drop[u] = in ? 1 : 0;
    if (in && conv) push_zone(zr, zi, ox, oy, nout, out_cap);
  }
  warp_add_u64(&ctr->steps_dd, steps);
}

// ---- the zone's root set ---------------------------------------------------------

__global__ void k_dd_keys(const dd* __restrict__ zx, dd* __restrict__ zy,
                          const unsigned long long* nz, int64_t zcap, double eps,
                          uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= zcap) return;
  if (i >= (int64_t)*nz) {  // padding sorts last
    keys[i] = ~0ull;
    vals[i] = (uint32_t)i;
    return;
  }
  if (fabs(dd_to_d(zy[i])) < 0.5 * eps) zy[i] = dd_make(0.0);  // a real root
  keys[i] = f64_key(zx[i].hi);
  vals[i] = (uint32_t)i;
}

// flag[p] = 1 if sorted zone point p has no earlier point within the
// Chebyshev pixel eps (compared in dd).
__global__ void k_dd_cluster(const dd* __restrict__ zx, const dd* __restrict__ zy,
                             const uint32_t* __restrict__ vals, const unsigned long long* nz,
                             int64_t zcap, double eps, uint32_t* __restrict__ flag) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= zcap) return;
  int64_t n = (int64_t)*nz;
  if (n > zcap) n = zcap;
  if (p >= n) {
    flag[p] = 0;
    return;
  }
  const uint32_t vp = vals[p];
  uint32_t rep = 1;
  for (int64_t q = p - 1; q >= 0 && p - q < 4096; --q) {
    const uint32_t vq = vals[q];
    if (hi_beyond(zx[vp].hi, zx[vq].hi, eps)) break;
    const double dx = dd_to_d(dd_sub(zx[vp], zx[vq]));
    const double dy = dd_to_d(dd_sub(zy[vp], zy[vq]));
    if (fabs(dx) < eps && fabs(dy) < eps) {
      rep = 0;
      break;
    }
  }
  flag[p] = rep;
}

__global__ void k_dd_compact(const dd* __restrict__ zx, const dd* __restrict__ zy,
                             const uint32_t* __restrict__ vals, const uint32_t* __restrict__ flag,
                             const uint32_t* __restrict__ pos, int64_t zcap, dd* __restrict__ rx,
                             dd* __restrict__ ry) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= zcap || !flag[p]) return;
  rx[pos[p]] = zx[vals[p]];
  ry[pos[p]] = zy[vals[p]];
}

// Exact type (as type_of of the binary64 path) with dd orbit values.
__device__ int type_of_dd(const PolyDev& P, dd cr, dd ci, double tau) {
  const int n = P.n;
  const int len = (P.kind == 0) ? n : P.l + n;
  int g = n;
  if (P.kind == 1) {
    int a = n, b = P.l - 1;
    while (b) {
      const int t = a % b;
      a = b;
      b = t;
    }
    g = a;
  }
  dd zr = dd_make(0.0), zi = dd_make(0.0), lr = dd_make(0.0), li = dd_make(0.0);
  double dzr = 0.0, dzi = 0.0, ldr = 0.0, ldi = 0.0;
  int hyp = 0, mis = 0;
  for (int k = 1; k <= len; ++k) {
    const double tzr = twice_f64(zr.hi), tzi = twice_f64(zi.hi);
    const double ndr = fma(tzr, dzr, fma(-tzi, dzi, 1.0));
    const double ndi = fma(tzr, dzi, tzi * dzr);
    const dd xx = dd_mul(zr, zr), yy = dd_mul(zi, zi), xy = dd_mul(zr, zi);
    zr = dd_add(dd_sub(xx, yy), cr);
    zi = dd_add(dd_twice(xy), ci);
    dzr = ndr;
    dzi = ndi;
    const double vr = dd_to_d(zr), vi = dd_to_d(zi);
    if (!hyp && k <= g && (g % k) == 0 &&
        fma(vr, vr, vi * vi) <= tau * tau * fma(dzr, dzr, dzi * dzi))
      hyp = k;
    if (P.kind == 1) {
      if (k == P.l) {
        lr = zr;
        li = zi;
        ldr = dzr;
        ldi = dzi;
      }
      const int kk = k - P.l;
      if (!mis && kk >= 1 && (n % kk) == 0) {
        const double er = dd_to_d(dd_sub(zr, lr)), ei = dd_to_d(dd_sub(zi, li));
        const double fr = dzr - ldr, fi = dzi - ldi;
        if (fma(er, er, ei * ei) <= tau * tau * fma(fr, fr, fi * fi)) mis = kk;
      }
    }
  }
  if (P.kind == 0) return hyp ? hyp : 255;
  if (hyp) return (32 + hyp < 64) ? 32 + hyp : 255;
  if (mis) return mis < 32 ? mis : 255;
  return 255;
}

// ---- disk certificate with dd centres ----------------------------------------------
//
// Thm proofRoots over disks whose centres are the dd values of the orbit
// (Thm diskArithmetic with a double-word centre arithmetic): every dd
// operation adds DD_REL_ERR |result| (above the published bounds of the
// algorithms used) to the radius of its result.  The derivative orbit has
// binary64 centres computed from the hi parts; its radius takes the half
// ulps of the binary64 roundings plus 2 |z_lo| |z'| for the dropped low part.
// Radii are binary64 rounded upward.

__device__ __forceinline__ double abs_ub64(double x, double y) {
  return __dsqrt_ru(__fma_ru(x, x, __dmul_ru(y, y)));
}
__device__ __forceinline__ double abs_lb64(double x, double y) {
  return __dsqrt_rd(__fma_rd(x, x, __dmul_rd(y, y)));
}
__device__ __forceinline__ double dd_abs_ub(const dd& x, const dd& y) {
  return __dadd_ru(abs_ub64(x.hi, y.hi), __dadd_ru(fabs(x.lo), fabs(y.lo)));
}

// Disk evaluation of P over D(c, rad) with dd centres: fz >= sup |P(c)|
// over the point orbit, the derivative disk B' = D(W, rw) encloses
// P'(D(c, rad)); returns fz, |W|_lb and rw.
__device__ void dd_disk_eval(const PolyDev& P, dd cr, dd ci, double rad, double& fz_out,
                             double& wabs_lb, double& rw_out) {
  const double E = DD_REL_ERR * 1.0001;
  dd zr = dd_make(0.0), zi = dd_make(0.0), czr = dd_make(0.0), czi = dd_make(0.0);
  double dx = 0.0, dy = 0.0, cdx = 0.0, cdy = 0.0;
  double rz0 = 0.0, rz = 0.0, rd = 0.0, crz0 = 0.0, crd = 0.0;
  for (int k = 1; k <= P.m; ++k) {
    const double mz = dd_abs_ub(zr, zi);
    const double md = abs_ub64(dx, dy);
    // z' = 2 z z' + 1 from the hi parts of z
    const double tzx = twice_f64(zr.hi), tzy = twice_f64(zi.hi);
    const double in_re = fma(-tzy, dy, 1.0);
    const double nd_x = fma(tzx, dx, in_re);
    const double p_im = tzy * dx;
    const double nd_y = fma(tzx, dy, p_im);
    double Rd = __dmul_ru(0.5, __dadd_ru(__dadd_ru(ulp64(in_re), ulp64(nd_x)),
                                         __dadd_ru(ulp64(p_im), ulp64(nd_y))));
    Rd = __fma_ru(__dmul_ru(2.0, __dadd_ru(fabs(zr.lo), fabs(zi.lo))), md, Rd);
    const double prod = __fma_ru(rz, rd, __fma_ru(rz, md, __dmul_ru(rd, mz)));
    const double nrd = __fma_ru(2.0, prod, Rd);
    // z = z^2 + c in dd: xx, yy, xy, xx - yy, + cr, 2 xy (exact), + ci
    const dd xx = dd_mul(zr, zr), yy = dd_mul(zi, zi), xy = dd_mul(zr, zi);
    const dd df = dd_sub(xx, yy);
    const dd nzr = dd_add(df, cr);
    const dd nzi = dd_add(dd_twice(xy), ci);
    double mag = __dadd_ru(__dadd_ru(fabs(xx.hi), fabs(yy.hi)), __dadd_ru(fabs(xy.hi), fabs(df.hi)));
    mag = __dadd_ru(mag, __dadd_ru(fabs(nzr.hi), fabs(nzi.hi)));
    const double Rz = __dmul_ru(E, mag);
    const double mz2 = __dmul_ru(2.0, mz);
    const double nrz0 = __fma_ru(rz0, rz0, __fma_ru(mz2, rz0, Rz));
    const double nrz = __dadd_ru(__fma_ru(rz, rz, __fma_ru(mz2, rz, Rz)), rad);
    zr = nzr;
    zi = nzi;
    dx = nd_x;
    dy = nd_y;
    rz0 = nrz0;
    rz = nrz;
    rd = nrd;
    if (k == P.lcap) {
      czr = zr;
      czi = zi;
      cdx = dx;
      cdy = dy;
      crz0 = rz0;
      crd = rd;
    }
  }
  if (P.lcap >= 0) {  // s_{l,n} = p_m + p_{l-1}
    const dd vr = dd_add(zr, czr), vi = dd_add(zi, czi);
    const double wx = dx + cdx, wy = dy + cdy;
    rz0 = __dadd_ru(__dadd_ru(rz0, crz0), __dmul_ru(E, __dadd_ru(fabs(vr.hi), fabs(vi.hi))));
    rd = __dadd_ru(__dadd_ru(rd, crd), __dmul_ru(0.5, __dadd_ru(ulp64(wx), ulp64(wy))));
    zr = vr;
    zi = vi;
    dx = wx;
    dy = wy;
  }
  fz_out = __dadd_ru(dd_abs_ub(zr, zi), rz0);
  wabs_lb = abs_lb64(dx, dy);
  rw_out = rd;
}

// Thm proofRoots with dd centres: one root in D(c, rad)
__device__ bool certify_dd(const PolyDev& P, dd cr, dd ci, double rad) {
  double fz, wl, rw;
  dd_disk_eval(P, cr, ci, rad, fz, wl, rw);
  const double dist = __dsub_rd(wl, rw);
  return isfinite(fz) && isfinite(dist) && dist > 0.0 && __dmul_rd(rad, dist) > fz;
}

// A zone root's disk must not meet the certified disk of a kept main
// representative (main reps sorted by Re, radii up to wmax).
__device__ bool meets_main(double x, double y, double rz, const double2* __restrict__ reps,
                           int64_t nmain, const uint8_t* __restrict__ drop,
                           const double* __restrict__ radius, double wmax) {
  if (!reps) return false;
  const double w = wmax + rz;
  int64_t lo = 0, hi = nmain;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (reps[mid].x < x - w) lo = mid + 1; else hi = mid;
  }
  for (int64_t q = lo; q < nmain && reps[q].x <= x + w && q - lo < 4096; ++q) {
    if (drop[q]) continue;
    const double ex = reps[q].x - x, ey = reps[q].y - y;
    const double lim = radius[q] + rz;
    if (fma(ex, ex, ey * ey) <= 1.0001 * lim * lim) return true;
  }
  return false;
}

// Type, multiplicity and certificate of each zone representative (sorted by
// hi Re), with the zone's share of the counters.
__global__ void k_dd_type_cert(PolyDev P, const dd* __restrict__ rx, const dd* __restrict__ ry,
                               const unsigned long long* nz_dev, double tau, double tol,
                               const double2* __restrict__ reps, const unsigned long long* n_main,
                               const uint8_t* __restrict__ drop, const double* __restrict__ radius,
                               double wmax, uint8_t* __restrict__ type, uint8_t* __restrict__ pass,
                               uint32_t* __restrict__ mult, int64_t zcap, DevCounters* ctr) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)*nz_dev;
  if (n > zcap) n = zcap;
  unsigned long long npass = 0, nreal = 0;
  double rad = 0.0;
  bool ok = false;
  if (u < zcap) {
    if (u >= n) {
      mult[u] = 0;
    } else {
      const dd cr = rx[u], ci = ry[u];
      const int t = type_of_dd(P, cr, ci, tau);
      const unsigned m = (ci.hi == 0.0) ? 1u : 2u;
      type[u] = (uint8_t)t;
      mult[u] = m;
      nreal = (m == 1);
      // nearest other zone root or conjugate within W = tol / 0.45
      const double W = tol / 0.45;
      double nn2 = W * W;
      if (m == 2) nn2 = fmin(nn2, 4.0 * ci.hi * ci.hi);
      for (int dir = -1; dir <= 1; dir += 2) {
        for (int64_t q = u + dir; q >= 0 && q < n && (q - u) * dir < 4096; q += dir) {
          if (hi_beyond(rx[q].hi, cr.hi, W)) break;
          const double ex = dd_to_d(dd_sub(rx[q], cr));
          const double ey = dd_to_d(dd_sub(ry[q], ci));
          const double ey2 = dd_to_d(dd_add(ry[q], ci));
          nn2 = fmin(nn2, fmin(fma(ex, ex, ey * ey), fma(ex, ex, ey2 * ey2)));
        }
      }
      rad = fmin(tol, 0.45 * sqrt(nn2));
      for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
        if (attempt) rad *= 0.25;
        ok = rad > 0.0 && certify_dd(P, cr, ci, rad);
      }
      if (ok && meets_main(cr.hi, ci.hi, rad, reps, (int64_t)*n_main, drop, radius, wmax)) ok = false;
      pass[u] = ok ? 1 : 0;
      npass = ok ? m : 0;
      if (t < 64) atomicAdd(&ctr->type_count[t], (unsigned long long)m);
    }
  }
  warp_add_u64(&ctr->n_cert_pass, npass);
  warp_add_u64(&ctr->n_reps_real, nreal);
  const unsigned long long rb = (unsigned long long)__double_as_longlong(rad);
  warp_min_u64(&ctr->min_radius_bits, (u < n && ok) ? rb : ~0ull);
  warp_max_u64(&ctr->max_radius_bits, (u < n && ok) ? rb : 0ull);
}

// Main representatives after the zone pass: kmult = mult of the kept ones;
// the counters lose the dropped ones (unsigned counters: adding the two's
// complement subtracts).
__global__ void k_dd_keep(const unsigned long long* n_reps, int64_t cap,
                          const uint32_t* __restrict__ mult, const uint8_t* __restrict__ drop,
                          const uint8_t* __restrict__ type, const uint8_t* __restrict__ pass,
                          uint32_t* __restrict__ kmult, DevCounters* ctr) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long dpass = 0, dreal = 0, drep = 0;
  if (u < cap) {
    if (u >= (int64_t)*n_reps) {
      kmult[u] = 0;
    } else if (drop[u]) {
      const unsigned m = mult[u];
      kmult[u] = 0;
      if (pass[u]) dpass = m;
      dreal = (m == 1);
      drep = 1;
      if (type[u] < 64) atomicAdd(&ctr->type_count[type[u]], 0ull - (unsigned long long)m);
    } else {
      kmult[u] = mult[u];
    }
  }
  warp_add_u64(&ctr->n_cert_pass, 0ull - dpass);
  warp_add_u64(&ctr->n_reps_real, 0ull - dreal);
  warp_add_u64(&ctr->n_reps, 0ull - drep);
}

// Emission of the merged list.  Kept main rep u goes to mpos[u] + (zone
// multiplicity before it); zone rep v to zmpos[v] + (kept main multiplicity
// up to it).  Equal Re: main before zone on both sides.
__global__ void k_dd_emit_main(const double2* __restrict__ reps, const unsigned long long* n_reps,
                               int64_t cap, const uint32_t* __restrict__ kmult,
                               const uint32_t* __restrict__ mpos, const uint8_t* __restrict__ type,
                               int mis_code, const dd* __restrict__ zrx,
                               const unsigned long long* nz_dev, int64_t zcap,
                               const uint32_t* __restrict__ zmpos, const unsigned long long* zt,
                               double2* __restrict__ out, uint8_t* __restrict__ is_mis,
                               int64_t cap_out) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= cap || u >= (int64_t)*n_reps || kmult[u] == 0) return;
  const double2 z = reps[u];
  int64_t nz = (int64_t)*nz_dev;
  if (nz > zcap) nz = zcap;
  int64_t lo = 0, hi = nz;  // zone reps with hi Re < z.x (compared as integer keys)
  const uint64_t kz = f64_key0(z.x);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (f64_key0(zrx[mid].hi) < kz) lo = mid + 1; else hi = mid;
  }
  const int64_t p = (int64_t)mpos[u] + (lo < nz ? (int64_t)zmpos[lo] : (int64_t)*zt);
  const uint8_t im = !type || mis_code < 0 ? 0
                     : mis_code == MIS_CODE_RAW ? type[u] : (uint8_t)(type[u] == mis_code);
  if (kmult[u] == 1) {
    if (p < cap_out) {
      out[p] = make_double2(z.x, 0.0);
      if (is_mis) is_mis[p] = im;
    }
  } else {
    if (p < cap_out) {
      out[p] = make_double2(z.x, -z.y);
      if (is_mis) is_mis[p] = im;
    }
    if (p + 1 < cap_out) {
      out[p + 1] = make_double2(z.x, z.y);
      if (is_mis) is_mis[p + 1] = im;
    }
  }
}

__global__ void k_dd_emit_zone(const dd* __restrict__ zrx, const dd* __restrict__ zry,
                               const unsigned long long* nz_dev, int64_t zcap,
                               const uint32_t* __restrict__ zmult, const uint32_t* __restrict__ zmpos,
                               const uint8_t* __restrict__ ztype, int mis_code,
                               const double2* __restrict__ reps, const unsigned long long* n_reps,
                               const uint32_t* __restrict__ mpos, const unsigned long long* mt,
                               double2* __restrict__ out, double2* __restrict__ out_lo,
                               uint8_t* __restrict__ is_mis, int64_t cap_out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nz = (int64_t)*nz_dev;
  if (nz > zcap) nz = zcap;
  if (v >= nz) return;
  const dd x = zrx[v], y = zry[v];
  const int64_t nm = (int64_t)*n_reps;
  int64_t lo = 0, hi = nm;  // main reps with Re <= x.hi
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (reps[mid].x <= x.hi) lo = mid + 1; else hi = mid;
  }
  const int64_t mb = (lo < nm) ? (int64_t)mpos[lo] : (int64_t)*mt;
  const int64_t p = (int64_t)zmpos[v] + mb;
  const uint8_t im = mis_code < 0 ? 0 : mis_code == MIS_CODE_RAW ? ztype[v] : (uint8_t)(ztype[v] == mis_code);
  if (zmult[v] == 1) {
    if (p < cap_out) {
      out[p] = make_double2(x.hi, 0.0);
      if (out_lo) out_lo[p] = make_double2(x.lo, 0.0);
      if (is_mis) is_mis[p] = im;
    }
  } else {
    if (p < cap_out) {
      out[p] = make_double2(x.hi, -y.hi);
      if (out_lo) out_lo[p] = make_double2(x.lo, -y.lo);
      if (is_mis) is_mis[p] = im;
    }
    if (p + 1 < cap_out) {
      out[p + 1] = make_double2(x.hi, y.hi);
      if (out_lo) out_lo[p + 1] = make_double2(x.lo, y.lo);
      if (is_mis) is_mis[p + 1] = im;
    }
  }
}

// Counters of the merged list: n_full and the zone's representatives.
__global__ void k_dd_totals(const unsigned long long* mt, const unsigned long long* zt,
                            const unsigned long long* nz, int64_t zcap, DevCounters* ctr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctr->n_full = *mt + *zt;
    ctr->n_reps += (*nz < (unsigned long long)zcap) ? *nz : (unsigned long long)zcap;
  }
}

// Certificate of a list with low parts (mt_certify with d_roots_lo), sorted
// by hi Re through 'order'.
__global__ void k_dd_certify_list(PolyDev P, const double2* __restrict__ hi,
                                  const double2* __restrict__ lo, const uint32_t* __restrict__ order,
                                  int64_t n, double tol, uint8_t* __restrict__ pass,
                                  double* __restrict__ radius, DevCounters* ctr) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long npass = 0;
  if (p < n) {
    const int64_t ip = order[p];
    const dd cr = dd{hi[ip].x, lo[ip].x}, ci = dd{hi[ip].y, lo[ip].y};
    const double W = tol / 0.45;
    double nn2 = W * W;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int64_t q = p + dir; q >= 0 && q < n && (q - p) * dir < 4096; q += dir) {
        const int64_t iq = order[q];
        if (hi_beyond(hi[iq].x, cr.hi, W)) break;
        const double ex = dd_to_d(dd_sub(dd{hi[iq].x, lo[iq].x}, cr));
        const double ey = dd_to_d(dd_sub(dd{hi[iq].y, lo[iq].y}, ci));
        nn2 = fmin(nn2, fma(ex, ex, ey * ey));
      }
    }
    double rad = fmin(tol, 0.45 * sqrt(nn2));
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
      if (attempt) rad *= 0.25;
      ok = rad > 0.0 && certify_dd(P, cr, ci, rad);
    }
    pass[ip] = ok ? 1 : 0;
    if (radius) radius[ip] = rad;
    npass = ok;
  }
  warp_add_u64(&ctr->n_cert_pass, npass);
}

// Newton-basin certificate (Thm proofContract) of a list with low parts, as
// k_basin with dd centres (sorted by hi Re through 'order').
__global__ void k_dd_basin(PolyDev P, const double2* __restrict__ hi, const double2* __restrict__ lo,
                           const uint32_t* __restrict__ order, int64_t n,
                           const double* __restrict__ rin, double eps_max,
                           double* __restrict__ basin, DevCounters* ctr) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long npass = 0;
  if (p < n) {
    const int64_t ip = order[p];
    const dd cr = dd{hi[ip].x, lo[ip].x}, ci = dd{hi[ip].y, lo[ip].y};
    const double Wn = 4.0 * eps_max;
    double nn2 = Wn * Wn;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int64_t q = p + dir; q >= 0 && q < n && (q - p) * dir < 4096; q += dir) {
        const int64_t iq = order[q];
        if (hi_beyond(hi[iq].x, cr.hi, Wn)) break;
        const double ex = dd_to_d(dd_sub(dd{hi[iq].x, lo[iq].x}, cr));
        const double ey = dd_to_d(dd_sub(dd{hi[iq].y, lo[iq].y}, ci));
        nn2 = fmin(nn2, fma(ex, ex, ey * ey));
      }
    }
    double out = 0.0;
    const double r = rin[ip];
    if (r > 0.0) {
      double fz, wl, rw;
      dd_disk_eval(P, cr, ci, r, fz, wl, rw);
      const double dist = __dsub_rd(wl, rw);
      if (isfinite(fz) && isfinite(dist) && dist > 0.0) {
        const double eta = fmin(__ddiv_ru(fz, dist), r);
        double eps = fmin(eps_max, 0.25 * sqrt(nn2));
        for (int k = 0; k < 24 && eps > 3.0 * eta; ++k, eps *= 0.25) {
          dd_disk_eval(P, cr, ci, eps, fz, wl, rw);
          if (isfinite(wl) && isfinite(rw) && __dsub_rd(wl, rw) > __dmul_ru(4.0, rw)) {
            out = eps;
            break;
          }
        }
      }
    }
    basin[ip] = out;
    npass = out > 0.0;
  }
  warp_add_u64(&ctr->n_cert_pass, npass);
}

// ---- launchers ---------------------------------------------------------------------

namespace {
inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }
}  // namespace

#define MT_DD_LAUNCH(kernel, n, bs, ...)                          \
  do {                                                            \
    if ((n) > 0) {                                                \
      MT_COUNT_LAUNCH(1);                                         \
      kernel<<<blocks_for((n), (bs)), (bs), 0, s>>>(__VA_ARGS__); \
    }                                                             \
  } while (0)

cudaError_t dd_collect_bad(const double2* reps, const unsigned long long* n_reps, int64_t cap,
                           const uint8_t* pass, const double* radius, double thr, double2* bad,
                           unsigned long long* nbad, int max_bad, cudaStream_t s) {
  MT_DD_LAUNCH(k_collect_bad, cap, 256, reps, n_reps, cap, pass, radius, thr, bad, nbad, max_bad);
  return cudaGetLastError();
}

cudaError_t dd_mark_pieces(const double2* cand, const uint8_t* status, int64_t S, int every,
                           int64_t Ls, int64_t npieces, const double2* bad, const uint64_t* klo,
                           const uint64_t* khi, int nbad, double R, uint32_t* flag, cudaStream_t s) {
  MT_DD_LAUNCH(k_mark_pieces, S, 256, cand, status, S, every, Ls, npieces, bad, klo, khi, nbad, R, flag);
  return cudaGetLastError();
}

cudaError_t dd_mark_pieces_fix(const int2* candq, int64_t S, int every, int64_t Ls, int64_t npieces,
                               const double2* bad, int nbad, double R, uint32_t* flag, cudaStream_t s) {
  MT_DD_LAUNCH(k_mark_pieces_fix, S, 256, candq, S, every, Ls, npieces, bad, nbad, R, flag);
  return cudaGetLastError();
}

cudaError_t dd_piece_ids(const uint32_t* flag, const uint32_t* pos, int64_t npieces, int64_t* ids,
                         int64_t ids_cap, cudaStream_t s) {
  MT_DD_LAUNCH(k_piece_ids, npieces, 256, flag, pos, npieces, ids, ids_cap);
  return cudaGetLastError();
}

cudaError_t dd_near_reps(const double2* reps, const unsigned long long* n_reps, int64_t cap,
                         const double2* bad, const uint64_t* klo, const uint64_t* khi, int nbad, double R,
                         uint32_t* near, unsigned long long* nnear, int64_t near_cap, cudaStream_t s) {
  MT_DD_LAUNCH(k_near_reps, cap, 256, reps, n_reps, cap, bad, klo, khi, nbad, R, near, nnear, near_cap);
  return cudaGetLastError();
}

cudaError_t dd_seeds(const PolyDev& P, double lambda0, int64_t NQ, int shrink, const int64_t* ids,
                     int64_t nb, uint32_t* cnt, uint32_t* off, void* scan_tmp, dd* sx, dd* sy,
                     DevCounters* ctr, cudaStream_t s) {
  int log2NQ = 0;
  while ((int64_t(1) << log2NQ) < NQ) ++log2NQ;
  MT_DD_LAUNCH(k_dd_seed_count, nb, 256, ids, nb, cnt);
  cudaError_t e = launch_exclusive_scan(cnt, off, nb, scan_tmp, nullptr, s);
  if (e != cudaSuccess) return e;
  {
    const int bs = 64;
    const size_t smem = (size_t)P.m * bs * sizeof(float2);
    MT_COUNT_LAUNCH(1);
    k_dd_seeds<<<blocks_for(2 * nb, bs), bs, smem, s>>>(P, lambda0, NQ, log2NQ, shrink, ids, cnt, off, nb, sx, sy,
                                                         ctr);
  }
  return cudaGetLastError();
}

cudaError_t dd_walk(const PolyDev& P, double lambda0, int M, int every, int64_t Ls, int64_t npieces,
                    const int64_t* ids, const uint32_t* off, int64_t nb, const dd* sx, const dd* sy,
                    dd* stx, dd* sty, uint8_t* st_ok, DevCounters* ctr, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (P.kind != 0) {  // s_{l,n}: the double-double walk
    MT_DD_LAUNCH(k_dd_walk, nb, 32, P, lambda0, M, every, Ls, npieces, ids, off, nb, sx, sy, stx, sty, st_ok, ctr);
    return cudaGetLastError();
  }
  const int bs = 32;  // one lane per piece: spread the few warps over the SMs
  const size_t smem = (size_t)P.m * bs * sizeof(float2);
  MT_COUNT_LAUNCH(1);
  if (P.lcap >= 0)
    k_dd_walk_pert<true><<<blocks_for(nb, bs), bs, smem, s>>>(P, lambda0, M, every, Ls, npieces, ids, off, nb, sx, sy,
                                                              stx, sty, st_ok, M, ctr);
  else
    k_dd_walk_pert<false><<<blocks_for(nb, bs), bs, smem, s>>>(P, lambda0, M, every, Ls, npieces, ids, off, nb, sx,
                                                               sy, stx, sty, st_ok, M, ctr);
  return cudaGetLastError();
}

cudaError_t dd_descend(const PolyDev& P, int64_t count, const dd* zx0, const dd* zy0,
                       const uint8_t* ok0, double tol, int cap, const double2* bad, int nbad,
                       double R, dd* ox, dd* oy, unsigned long long* nout, int64_t out_cap,
                       DevCounters* ctr, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_DD_LAUNCH(k_dd_descend, count, 64, P, count, zx0, zy0, ok0, tol * tol, cap, bad, nbad, R, ox, oy, nout,
               out_cap, ctr);
  return cudaGetLastError();
}

cudaError_t dd_polish(const PolyDev& P, const double2* reps, const uint32_t* near,
                      const unsigned long long* nnear, int64_t near_cap, int64_t launch_n, double tol,
                      const double2* bad, int nbad, double R, double margin, uint8_t* drop, dd* ox,
                      dd* oy, unsigned long long* nout, int64_t out_cap, DevCounters* ctr,
                      cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_polish, launch_n, 64, P, reps, near, nnear, near_cap, tol * tol, bad, nbad, R,
               margin, drop, ox, oy, nout, out_cap, ctr);
  return cudaGetLastError();
}

cudaError_t dd_keys(const dd* zx, dd* zy, const unsigned long long* nz, int64_t zcap, double eps,
                    uint64_t* keys, uint32_t* vals, cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_keys, zcap, 256, zx, zy, nz, zcap, eps, keys, vals);
  return cudaGetLastError();
}

cudaError_t dd_cluster(const dd* zx, const dd* zy, const uint32_t* vals, const unsigned long long* nz,
                       int64_t zcap, double eps, uint32_t* flag, cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_cluster, zcap, 256, zx, zy, vals, nz, zcap, eps, flag);
  return cudaGetLastError();
}

cudaError_t dd_compact(const dd* zx, const dd* zy, const uint32_t* vals, const uint32_t* flag,
                       const uint32_t* pos, int64_t zcap, dd* rx, dd* ry, cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_compact, zcap, 256, zx, zy, vals, flag, pos, zcap, rx, ry);
  return cudaGetLastError();
}

cudaError_t dd_type_cert(const PolyDev& P, const dd* rx, const dd* ry, const unsigned long long* nz,
                         double tau, double tol, const double2* reps, const unsigned long long* n_main,
                         const uint8_t* drop, const double* radius, double wmax, uint8_t* type,
                         uint8_t* pass, uint32_t* mult, int64_t zcap, DevCounters* ctr,
                         cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_type_cert, zcap, 64, P, rx, ry, nz, tau, tol, reps, n_main, drop, radius, wmax, type,
               pass, mult, zcap, ctr);
  return cudaGetLastError();
}

cudaError_t dd_keep(const unsigned long long* n_reps, int64_t cap, const uint32_t* mult,
                    const uint8_t* drop, const uint8_t* type, const uint8_t* pass, uint32_t* kmult,
                    DevCounters* ctr, cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_keep, cap, 256, n_reps, cap, mult, drop, type, pass, kmult, ctr);
  return cudaGetLastError();
}

cudaError_t dd_emit(const double2* reps, const unsigned long long* n_reps, int64_t cap,
                    const uint32_t* kmult, const uint32_t* mpos, const unsigned long long* mt,
                    const uint8_t* type, int mis_code, const dd* zrx, const dd* zry,
                    const unsigned long long* nz, int64_t zcap, const uint32_t* zmult,
                    const uint32_t* zmpos, const unsigned long long* zt, const uint8_t* ztype,
                    double2* out, double2* out_lo, uint8_t* is_mis, int64_t cap_out,
                    DevCounters* ctr, cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_emit_main, cap, 256, reps, n_reps, cap, kmult, mpos, type, mis_code, zrx, nz, zcap,
               zmpos, zt, out, is_mis, cap_out);
  MT_DD_LAUNCH(k_dd_emit_zone, zcap, 128, zrx, zry, nz, zcap, zmult, zmpos, ztype, mis_code, reps, n_reps,
               mpos, mt, out, out_lo, is_mis, cap_out);
  MT_COUNT_LAUNCH(1);
  k_dd_totals<<<1, 32, 0, s>>>(mt, zt, nz, zcap, ctr);
  return cudaGetLastError();
}

cudaError_t dd_certify_list(const PolyDev& P, const double2* hi, const double2* lo,
                            const uint32_t* order, int64_t n, double tol, uint8_t* pass,
                            double* radius, DevCounters* ctr, cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_certify_list, n, 64, P, hi, lo, order, n, tol, pass, radius, ctr);
  return cudaGetLastError();
}

cudaError_t dd_basin(const PolyDev& P, const double2* hi, const double2* lo, const uint32_t* order,
                     int64_t n, const double* radius, double eps_max, double* basin, DevCounters* ctr,
                     cudaStream_t s) {
  MT_DD_LAUNCH(k_dd_basin, n, 64, P, hi, lo, order, n, radius, eps_max, basin, ctr);
  return cudaGetLastError();
}

}  // namespace mt
