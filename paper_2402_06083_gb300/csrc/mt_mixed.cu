// mt_mixed.cu -- the mixed-precision tier (MT_MIXED): binary32 level-line
// tracking and early Newton steps around float-float anchors (binary64 ones
// in the seed lift), and a binary64 finish.
//
// Why.  The paper runs everything in FP80 (Sec. 6.1) and notes that GPUs
// offer little beyond FP64 (Sec. 6.4.5).  On a GB300 the binary64 pipe is
// the bottleneck (about 1.2 TFLOP/s) while binary32 runs ~60x faster, so the
// bulk of the Newton steps -- which only need to stay in the right basin --
// move to binary32, and binary64 is spent where precision is decided.
//
// How.  Absolute binary32 coordinates cannot resolve the level line at the
// periods of interest (sub-step spacings reach 1e-11 near c = -2 at n = 20),
// so the binary32 work is done in perturbation form around an anchor c0
// (the published perturbation technique of deep-zoom Mandelbrot
// renderers): with Z_k = p_k(c0) (float-float, ~1e-14; binary64 in the seed
// lift) and c = c0 + delta,
//   e_{k+1} = (2 Z_k + e_k) e_k + delta,   p_k(c) = Z_k + e_k,
//   p'_{k+1}(c) = 2 (Z_k + e_k) p'_k(c) + 1            (binary32),
// so binary32 carries only the difference from the anchor and its relative
// precision applies to |delta|, not to |c|.  The residual P(c) - T is
// (Z_m - T) + e_m with Z_m split into binary32 hi + lo.
//   - Walk: the anchor is re-taken every K sub-steps (a few turns of the
//     phase) from the current point, so |delta| stays a few turns' length.
//   - Descent: the anchor is the start point; binary32 Newton steps run to
//     the binary32 floor, then binary64 Newton steps (1.08 a root at p_28),
//     once per group of end points on the same root, finish to the binary64
//     tolerance (eq. Newton).
// The anchors only steer the binary32 steps; every root's digits come from
// its binary64 finishing steps.  The chunk-end check of the walk and the
// count check catch any tracking failure, and the host then repeats the
// split in plain binary64.
#include "mt_levelline.cuh"
#include "mt_pert.cuh"

namespace mt {

constexpr int MIX_MAXM = 41;
constexpr int64_t MIX_BATCH = int64_t(1) << 23;  // starts per launch of the binary32 descent

// Float-float (binary32 pair) arithmetic from the published error-free
// transforms: Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based TwoProd.
// ~48-bit accurate; used where a binary64 result is not needed but binary32
// is not enough (the descents' anchor orbits).
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_from(double x) {
  ff r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ ff ff_norm(float s, float e) {  // FastTwoSum, |s| >= |e|
  ff r;
  r.hi = s + e;
  r.lo = e - (r.hi - s);
  return r;
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.hi + b.hi;  // TwoSum
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
  return ff_norm(s, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;  // TwoProd
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_twice(ff a) { return ff{a.hi + a.hi, a.lo + a.lo}; }

// binary64 reference orbit at c0: zs[k * stride] = Z_k in binary32 for
// k = 0 .. m-1 (truncated on the integer pipe: the binary64 pipe keeps the
// orbit itself), and v = P(c0) = Z_m (+ Z_lcap) as binary32 hi (x, y) + lo (z, w).
__device__ __forceinline__ void ref_orbit(const PolyDev& P, double c0x, double c0y, float2* zs,
                                          int stride, float4& v) {
  double zx = 0.0, zy = 0.0, capx = 0.0, capy = 0.0;
  zs[0] = make_float2(0.f, 0.f);
  for (int k = 1; k <= P.m; ++k) {
    const double nx = fma(zx, zx, fma(-zy, zy, c0x));
    const double ny = fma(twice_f64(zx), zy, c0y);
    zx = nx;
    zy = ny;
    if (k < P.m) zs[k * stride] = make_float2(f32_trunc(zx), f32_trunc(zy));  // integer pipe
    if (k == P.lcap) { capx = zx; capy = zy; }
  }
  const double vx = zx + capx, vy = zy + capy;
  const float hx = (float)vx, hy = (float)vy;
  v = make_float4(hx, hy, (float)(vx - (double)hx), (float)(vy - (double)hy));
}

// binary32 perturbation orbit: e = P(c0 + delta) - P(c0), D = P'(c0 + delta).
// The derivative is carried as g_k = p'_k / 2^k (g_{k+1} = p_k g_k +
// 2^-(k+1)): the same binary32 roundings as p'_{k+1} = 2 p_k p'_k + 1 up to
// powers of two, without doubling p_k (12 binary32 operations a step, not 14).
__device__ __forceinline__ void pert_eval(const PolyDev& P, const float2* zs, int stride, float dx,
                                          float dy, float& ex, float& ey, float& Dx, float& Dy) {
  float e_x = 0.f, e_y = 0.f, g_x = 0.f, g_y = 0.f;
  float ce_x = 0.f, ce_y = 0.f, cg_x = 0.f, cg_y = 0.f;
  int hexp = (127 - 1) << 23;  // exponent field of 2^-(k+1), k = 0
#pragma unroll 2
  for (int k = 0; k < P.m; ++k) {
    const float2 Z = zs[k * stride];
    const float zx = Z.x + e_x, zy = Z.y + e_y;  // p_k(c)
    const float h = __int_as_float(hexp);
    hexp -= 1 << 23;
    const float ng_x = fmaf(zx, g_x, fmaf(-zy, g_y, h));
    const float ng_y = fmaf(zx, g_y, zy * g_x);
    const float sx = Z.x + zx, sy = Z.y + zy;  // 2 Z_k + e_k
    const float ne_x = fmaf(sx, e_x, fmaf(-sy, e_y, dx));
    const float ne_y = fmaf(sx, e_y, fmaf(sy, e_x, dy));
    e_x = ne_x; e_y = ne_y; g_x = ng_x; g_y = ng_y;
    if (k + 1 == P.lcap) { ce_x = e_x; ce_y = e_y; cg_x = g_x; cg_y = g_y; }
  }
  ex = e_x + ce_x;
  ey = e_y + ce_y;
  // p'_m + p'_lcap = 2^m (g_m + 2^(lcap-m) g_lcap), exact scalings
  const float a = P.lcap > 0 ? __int_as_float((127 + P.lcap - P.m) << 23) : 0.f;
  const float s = __int_as_float((127 + P.m) << 23);
  Dx = fmaf(a, cg_x, g_x) * s;
  Dy = fmaf(a, cg_y, g_y) * s;
}

// Newton with target in perturbation form: the binary32 twin of the walk's
// newton_target_f64, with the same predictor (pred: first step solves
// log P = log T from the previous target Tp, L = log(T / Tp)) and stop rule.
__device__ __forceinline__ int newton_target_pert(const PolyDev& P, const float2* zs, int stride,
                                                  const float4& v, float& dx, float& dy, float tx,
                                                  float ty, float rel, int cap, float* first,
                                                  bool pred, float tpx, float tpy, float Lr,
                                                  float Li, bool* bad) {
  float thr2 = 0.f, prev2 = 0.f, h2 = 0.f;
  int it = 0;
  while (it < cap) {
    float ex, ey, Dx, Dy;
    pert_eval(P, zs, stride, dx, dy, ex, ey, Dx, Dy);
    float nr, ni;
    if (it == 0 && pred) {  // P - Tp - L P
      const float Pr = v.x + (v.z + ex), Pi = v.y + (v.w + ey);
      nr = (Pr - tpx) - fmaf(Lr, Pr, -Li * Pi);
      ni = (Pi - tpy) - fmaf(Lr, Pi, Li * Pr);
    } else {
      nr = ((v.x - tx) + v.z) + ex;
      ni = ((v.y - ty) + v.w) + ey;
    }
    float qr, qi;
    if (!cdiv_f32(nr, ni, Dx, Dy, qr, qi)) { *bad = true; break; }
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

// a1 + a2 in the mixed tier: the lift of k_seed_lift (Sec. 4.2) with each
// level's solves in perturbation form around the point reached at the
// previous level (one binary64 reference orbit of p_{k+1} per level instead
// of ~(1 + shrink) x 3 binary64 Newton steps).  The s_{l,n} homotopy at the
// last level stays binary64.
__global__ void k_seed_lift_mixed(PolyDev P, double lambda0, int64_t N0, int log2N0, int shrink,
                                  double2* seeds, uint8_t* __restrict__ seed_bad, DevCounters* ctr) {
  extern __shared__ float2 zsh[];
  float2* zs = zsh + threadIdx.x;
  const int stride = blockDim.x;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, s32 = 0, fails = 0;
  if (j <= N0 / 2) {
    double c, s;
    unit_phase((uint64_t)j, (uint64_t)N0, c, s);
    double zr = lambda0 * c, zi = lambda0 * s;
    const float lam2 = (float)(lambda0 * lambda0);
    const float Lq = (float)(-log(lambda0) / shrink);
    double R[LIFT_RADII];
    const bool tab = shrink_radii(lambda0, shrink, R);
    bool bad = false;
    for (int k = 1; k < P.m; ++k) {
      const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
      unit_phase(num, (uint64_t)N0, c, s);
      PolyDev Q;
      Q.kind = 0; Q.l = 0; Q.n = k + 1; Q.m = k + 1; Q.lcap = -1; Q.log2d = k;
      float4 v;
      ref_orbit(Q, zr, zi, zs, stride, v);
      float dx = 0.f, dy = 0.f;
      const float ec = (float)c, es = (float)s;
      int it = newton_target_pert(Q, zs, stride, v, dx, dy, lam2 * ec, lam2 * es, 1e-3f, 40, nullptr,
                                  false, 0.f, 0.f, 0.f, 0.f, &bad);
      for (int q = 1; q <= shrink; ++q) {
        const float rp = (float)shrink_radius(R, tab, lambda0, shrink, q - 1);
        const float r = (float)shrink_radius(R, tab, lambda0, shrink, q);
        it += newton_target_pert(Q, zs, stride, v, dx, dy, r * ec, r * es, 1e-3f, 40, nullptr, true,
                                 rp * ec, rp * es, Lq, 0.f, &bad);
      }
      steps += it;
      s32 += it;
      zr += (double)dx;
      zi += (double)dy;
    }
    if (P.kind == 1) {
      // binary64 homotopy p_m -> p_m + p_{l-1} (as in k_seed_lift)
      const int k = P.m - 1;
      const uint64_t num = (k >= log2N0) ? 0 : (((uint64_t)j << k) & (uint64_t)(N0 - 1));
      unit_phase(num, (uint64_t)N0, c, s);
      for (int a = 1; a <= 8; ++a) {
        const double alpha = a / 8.0;
        for (int t = 0; t < 40; ++t) {
          double vr, vi, dr, di, qr, qi;
          orbit_f64(P.m, P.lcap, alpha, zr, zi, vr, vi, dr, di);
          cdiv_f64(vr - lambda0 * c, vi - lambda0 * s, dr, di, qr, qi);
          if (!finite2(qr, qi)) break;
          zr -= qr;
          zi -= qi;
          ++steps;
          if (fma(qr, qr, qi * qi) <= 1e-24 * fma(zr, zr, zi * zi) + 1e-300) break;
        }
      }
    }
    if (j == 0 || j == N0 / 2) zi = 0.0;
    seeds[j] = make_double2(zr, zi);
    fails = bad ? 1 : 0;
    seed_bad[j] = bad ? 1 : 0;  // lifted again in binary64 by k_seed_repair
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->seed_newton, steps);
  warp_add_u64(&ctr->steps_fp32, s32);
  warp_add_u64(&ctr->walk_fail, fails);
}

// Float-float reference orbit of the walk, anchored at c0' = the float-float
// value of c0 (hi + lo, exactly a binary64), so that no bit of the anchor is
// lost: the caller carries c0 - c0' (below 2^-47 |c0|) in delta.  Z_k
// (k < m) to shared memory in binary32, P(c0') as binary32 hi + lo.  Its
// ~1e-14 relative accuracy moves P by far less than the walk's tolerance
// (1e-2 of a sub-step) and keeps the walk off the binary64 pipe, where one
// binary64 anchor cost as much as the binary32 sub-steps it served.
template <bool CAP, int MC, int STRIDE>
__device__ __forceinline__ void ref_orbit_ff(const PolyDev& P, double c0x, double c0y, float2* zs, float4& v,
                                             double& ax, double& ay) {
  const ff cx = ff_from(c0x), cy = ff_from(c0y);
  ax = (double)cx.hi + (double)cx.lo;
  ay = (double)cy.hi + (double)cy.lo;
  ff zx{0.f, 0.f}, zy{0.f, 0.f}, capx{0.f, 0.f}, capy{0.f, 0.f};
  zs[0] = make_float2(0.f, 0.f);
  const int m = MC > 0 ? MC : P.m;
#pragma unroll 2
  for (int k = 1; k <= m; ++k) {
    const ff nx = ff_add(ff_add(ff_mul(zx, zx), ff_neg(ff_mul(zy, zy))), cx);
    const ff ny = ff_add(ff_twice(ff_mul(zx, zy)), cy);
    zx = nx;
    zy = ny;
    if (k < m) zs[k * STRIDE] = make_float2(zx.hi, zy.hi);
    if (CAP && k == P.lcap) { capx = zx; capy = zy; }
  }
  const ff vx = CAP ? ff_add(zx, capx) : zx, vy = CAP ? ff_add(zy, capy) : zy;
  v = make_float4(vx.hi, vy.hi, vx.lo, vy.lo);
}

// a3 in the mixed tier: one lane per chunk of L sub-steps, binary32
// perturbation around a float-float anchor re-taken every K sub-steps.
// Shared memory: each warp owns m rows of 32 binary32 pairs (row stride 32,
// a compile-time constant).  j0 / nch / sbase: chunks [j0, j0 + nch) only,
// start g / every written at g / every - sbase (a streamed split's piece;
// 0 / nchunks / 0 for the whole line).  MC as in k_descend_mixed.
template <bool CAP, int MC>
__global__ void k_walk_mixed(PolyDev P, double lambda0, int M, int every, int64_t L, int64_t nchunks,
                             int K, const double2* __restrict__ seeds, double2* __restrict__ starts,
                             uint8_t* __restrict__ chunk_fail, DevCounters* ctr, int64_t j0, int64_t nch,
                             int64_t sbase) {
  extern __shared__ float2 zsh[];
  __shared__ float2 ph[64];
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double c, s;
    unit_phase((uint64_t)q, (uint64_t)M, c, s);
    ph[q] = make_float2((float)(lambda0 * c), (float)(lambda0 * s));
  }
  __syncthreads();
  const int m = MC > 0 ? MC : P.m;
  float2* zs = zsh + (threadIdx.x >> 5) * 32 * m + (threadIdx.x & 31);
  const int64_t jl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = j0 + jl;
  unsigned long long steps = 0, fails = 0;
  if (jl < nch && j < nchunks) {
    const double2 s0 = seeds[j];
    double c0x, c0y;
    float4 v;
    ref_orbit_ff<CAP, MC, 32>(P, s0.x, s0.y, zs, v, c0x, c0y);
    float dx = (float)(s0.x - c0x), dy = (float)(s0.y - c0y), h = 0.f;
    bool bad = false;
    const float Li = 6.2831853f / M;
    const int esh = __ffs(every) - 1;  // every is a power of two
    uint64_t g = (uint64_t)j * (uint64_t)L;
    int kc = K;  // sub-steps to the next anchor
    for (int64_t i = 0; i < L; ++i, ++g) {
      if ((g & (uint64_t)(every - 1)) == 0)
        starts[(int64_t)(g >> esh) - sbase] = make_double2(c0x + (double)dx, c0y + (double)dy);
      const float2 Tp = ph[g & (uint64_t)(M - 1)];
      const float2 T = ph[(g + 1) & (uint64_t)(M - 1)];
      // tight (1e-2) only on the sub-steps that end on a start, as in walk_chunk
      const float rel = (((g + 1) & (uint64_t)(every - 1)) == 0) ? 1e-2f : 1e-1f;
      steps += newton_target_walk<CAP, MC, 32>(P, zs, v, dx, dy, T.x, T.y, rel, 16, &h, Tp.x, Tp.y, Li, &bad);
      if (--kc == 0 && i + 1 < L) {  // re-anchor at the current point
        kc = K;
        const double px = c0x + (double)dx, py = c0y + (double)dy;
        ref_orbit_ff<CAP, MC, 32>(P, px, py, zs, v, c0x, c0y);
        dx = (float)(px - c0x);
        dy = (float)(py - c0y);
      }
    }
    const double cx = c0x + (double)dx, cy = c0y + (double)dy;
    if (j == nchunks - 1) starts[(int64_t)(g >> esh) - sbase] = make_double2(cx, 0.0);
    const double2 zn = seeds[j + 1];
    const double er = cx - zn.x, ei = cy - zn.y;
    const double hh = (double)h;
    if (bad || !(er * er + ei * ei <= 0.0625 * hh * hh + 1e-28)) fails = 1;
    chunk_fail[j] = (uint8_t)fails;  // walked again in binary64 by k_walk_repair
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->steps_fp32, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

using WalkMixedFn = void (*)(PolyDev, double, int, int, int64_t, int64_t, int, const double2*, double2*, uint8_t*,
                             DevCounters*, int64_t, int64_t, int64_t);
template <int MC>
WalkMixedFn walk_mixed_fixed(int m) {
  if constexpr (MC < 16) {
    (void)m;
    return nullptr;
  } else {
    return m == MC ? &k_walk_mixed<false, MC> : walk_mixed_fixed<MC - 1>(m);
  }
}
WalkMixedFn walk_mixed_kernel(const PolyDev& P) {
  if (P.lcap >= 0) return &k_walk_mixed<true, 0>;
  WalkMixedFn f = walk_mixed_fixed<33>(P.m);
  return f ? f : &k_walk_mixed<false, 0>;
}

// a4 in the mixed tier, anchors: the reference orbit of a start c0 in
// float-float, rounded to binary32 (Z_k, k = 1 .. m-1), plus P(c0) as
// binary32 hi + lo and the long-jump bound on |delta|.  The anchor only
// steers the binary32 descent into the basin of its root (the binary64
// finish sets the digits), so float-float's ~1e-14 suffices and keeps this
// off the binary64 pipe.  A warp computes the orbits of the 32 starts of a
// queue range together, lane j the orbit of start g + j, into its own slot
// of the buffer: Z_k of lane j at za[(k - 1) * 32 + j] (each store
// instruction writes 256 contiguous bytes), P(c0) at zv[j], the bound at
// zr[j].  The slots are small (32 orbits per warp) and are read back by the
// same warp moments later, so they stay in L2.
struct WarpSlot {
  float2* za;  // [m - 1][32]
  float4* zv;  // [32]
  float* zr;   // [32]
};
__device__ __forceinline__ WarpSlot warp_slot(float2* wbuf, int m1, unsigned warp) {
  const size_t per = (size_t)32 * m1 + 80;  // float2 units: anchors, 32 float4, 32 float
  float2* b = wbuf + per * warp;
  WarpSlot w;
  w.za = b;
  w.zv = (float4*)(b + (size_t)32 * m1);
  w.zr = (float*)(b + (size_t)32 * m1 + 64);
  return w;
}
template <bool CAP, int MC>
__device__ __forceinline__ void anchor_orbit(const PolyDev& P, double2 c0, const WarpSlot& w, unsigned j) {
  const int m = MC > 0 ? MC : P.m;
  const ff cx = ff_from(c0.x), cy = ff_from(c0.y);
  ff zx{0.f, 0.f}, zy{0.f, 0.f}, capx{0.f, 0.f}, capy{0.f, 0.f};
#pragma unroll 4
  for (int k = 1; k <= m; ++k) {
    const ff nx = ff_add(ff_add(ff_mul(zx, zx), ff_neg(ff_mul(zy, zy))), cx);
    const ff ny = ff_add(ff_twice(ff_mul(zx, zy)), cy);
    zx = nx;
    zy = ny;
    if (k < m) w.za[(k - 1) * 32 + j] = make_float2(zx.hi, zy.hi);
    if (CAP && k == P.lcap) { capx = zx; capy = zy; }
  }
  const ff vx = ff_add(zx, capx), vy = ff_add(zy, capy);
  w.zv[j] = make_float4(vx.hi, vy.hi, vx.lo, vy.lo);
  // long jump (as in k_descend: |c| > max(4, 2|c0|)); |delta| beyond rdel implies it
  const float r0 = sqrtf(fmaf(cx.hi, cx.hi, cy.hi * cy.hi)) * 1.0001f;
  w.zr[j] = fmaxf(4.f, 2.f * r0) + r0;
}

// a4 in the mixed tier, binary32 phase (persistent, per-lane refill as in
// k_descend) over starts [base, base + cnt), cnt < 2^31.  Each lane keeps
// the anchor orbit of its descent (Z_1 .. Z_{m-1}) in its own column of
// shared memory (row k - 1 holds Z_k of every lane; the row stride DM_BS + 1
// is odd, so the rows of one column fall in different banks).  Lanes that
// finished are refilled together once DM_REFILL of them wait (or none is
// running): they take the next start indices of the warp's range of the
// work queue, and a refilled lane copies its orbit from the warp's slot
// into its column (m - 1 independent loads, L2 hits).  When the range runs
// out the warp takes the next one (one atomic per 32 starts) and computes
// its 32 anchor orbits with every lane (anchor_orbit): the orbits cost one
// full-width pass per 32 starts and never travel through HBM.  The Newton
// loop is binary32 only.  Each descent runs binary32 Newton steps to the
// binary32 floor and leaves (delta, its largest squared step) in pack[]
// with status 3 ("finish in binary64"), or stops as divergent (1) / timed
// out (2).  The binary64 finish runs in k_finish_f64, a separate uniform
// launch, once per root.  MC: the orbit length when fixed at compile time
// (p_n), else 0.
constexpr int DESC_POOL = 32;  // work indices taken per queue atomic (one per lane of a range)
constexpr int DM_BS = 128;     // threads per block of the binary32 descent
constexpr int DM_REFILL = 4;   // idle lanes that trigger a refill
constexpr int DM_MAX_WARPS = 16384;  // warp slots of the anchor buffer (grids are capped to fit)

template <bool CAP, int MC>
__global__ void __launch_bounds__(DM_BS) k_descend_mixed(PolyDev P, const double2* __restrict__ starts,
                                                         int64_t base, int64_t cnt, float2* wbuf, int cap,
                                                         float4* __restrict__ pack,
                                                         uint8_t* __restrict__ status,
                                                         unsigned* queue, DevCounters* ctr) {
  extern __shared__ float2 zsh[];
  constexpr int stride = DM_BS + 1;
  const float2* zs = zsh + threadIdx.x;  // row 0 (Z_1) of this lane's column
  const unsigned lane = threadIdx.x & 31;
  const int m1 = (MC > 0 ? MC : P.m) - 1;
  const unsigned n = (unsigned)cnt;
  const WarpSlot ws = warp_slot(wbuf, m1, (blockIdx.x * DM_BS + threadIdx.x) >> 5);
  unsigned idx = ~0u;  // this lane's start (~0u: none)
  float dx = 0.f, dy = 0.f, h1 = 0.f, prev2 = 0.f, rdelta = 0.f;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  int it = 0;
  unsigned long long s32 = 0, ndiv = 0, nto = 0;
  // the warp's range [pool_base, pool_base + 32) and its next unused index
  // (warp-uniform; none taken yet: pool_next at the range's end)
  unsigned pool_base = 0, pool_next = DESC_POOL;
  bool drained = false;                   // the queue is empty (warp-uniform)
  // a refilled lane with start i of the range in the slot: its orbit into
  // its column, and the state of a new descent
  auto take_orbit = [&](unsigned i) {
    const unsigned j = i - pool_base;
    float2* dst = zsh + threadIdx.x;
    if (MC > 0) {
#pragma unroll
      for (int k = 0; k < (MC > 0 ? MC - 1 : 1); ++k) dst[k * stride] = ws.za[k * 32 + j];
    } else {
      for (int k = 0; k < m1; ++k) dst[k * stride] = ws.za[k * 32 + j];
    }
    v = ws.zv[j];
    rdelta = ws.zr[j];
    dx = dy = 0.f;
    it = 0;
    prev2 = 0.f;
    h1 = 0.f;
  };
  for (;;) {
    const unsigned need = drained ? 0u : __ballot_sync(0xffffffffu, idx == ~0u);
    const unsigned R = __popc(need);
    if (R >= DM_REFILL || (R == 32u && need)) {
      // the r-th lane that needs a start takes the r-th unused index of the
      // range, then of the next range
      const bool mine = (need >> lane) & 1u;
      const unsigned r_me = __popc(need & lanemask_lt());
      const unsigned rem = pool_base + DESC_POOL - pool_next;
      if (mine && r_me < rem) {
        idx = pool_next + r_me;
        if (idx < n) take_orbit(idx);
      }
      if (rem >= R) {
        pool_next += R;
      } else {
        __syncwarp();  // the copies above have read the slot
        unsigned g = 0;
        if (lane == 0) g = atomicAdd(queue, (unsigned)DESC_POOL);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g + lane < n) anchor_orbit<CAP, MC>(P, starts[base + g + lane], ws, lane);
        __syncwarp();  // the slot is written before any lane reads it
        pool_base = g;
        pool_next = g + (R - rem);
        if (mine && r_me >= rem) {
          idx = g + (r_me - rem);
          if (idx < n) take_orbit(idx);
        }
      }
      if (mine && idx >= n) idx = n;  // the queue is drained: never refilled again
      if (__any_sync(0xffffffffu, mine && idx == n)) drained = true;
    }
    const bool active = idx < n;
    if (!__any_sync(0xffffffffu, active)) {
      if (drained) break;
      continue;  // every lane idle: the next pass refills all 32
    }
    if (active) {
      int outcome = -1;
      float ex, ey, Dx, Dy, qr, qi;
      pert_eval_t<CAP, MC, stride>(P, zs, dx, dy, ex, ey, Dx, Dy);
      const float nr = (v.x + v.z) + ex, ni = (v.y + v.w) + ey;
      if (!cdiv_f32(nr, ni, Dx, Dy, qr, qi)) {
        outcome = 3;  // out of binary32 range: binary64 decides
      } else {
        dx -= qr;
        dy -= qi;
        ++it;
        ++s32;
        const float s2 = fmaf(qr, qr, qi * qi);
        h1 = fmaxf(h1, s2);  // largest step so far
        if (!(fmaf(dx, dx, dy * dy) <= rdelta * rdelta)) outcome = 1;
        // binary32 floor: the step is 1e-5 of the descent's scale, or it
        // stopped shrinking once already below 1e-3 of it
        else if (s2 <= 1e-10f * h1 || (s2 <= 1e-6f * h1 && s2 > 0.25f * prev2)) outcome = 3;
        else if (it >= cap) outcome = 2;
        prev2 = s2;
      }
      if (outcome >= 0) {
        pack[base + idx] = make_float4(dx, dy, h1, 0.f);
        status[base + idx] = (uint8_t)outcome;
        ndiv += outcome == 1;
        nto += outcome == 2;
        idx = ~0u;
      }
    }
  }
  warp_add_u64(&ctr->desc_newton, s32);
  warp_add_u64(&ctr->desc_fp32, s32);
  warp_add_u64(&ctr->steps_fp32, s32);
  warp_add_u64(&ctr->n_diverge, ndiv);
  warp_add_u64(&ctr->n_timeout, nto);
}

using DescMixedFn = void (*)(PolyDev, const double2*, int64_t, int64_t, float2*, int, float4*, uint8_t*,
                             unsigned*, DevCounters*);

// The instantiation for a polynomial: p_n with 16 <= n <= 33 has its orbit
// length fixed at compile time; everything else runs the general loop.
template <int MC>
DescMixedFn desc_mixed_fixed(int m) {
  if constexpr (MC < 16) {
    (void)m;
    return nullptr;
  } else {
    return m == MC ? &k_descend_mixed<false, MC> : desc_mixed_fixed<MC - 1>(m);
  }
}
DescMixedFn desc_mixed_kernel(const PolyDev& P) {
  if (P.lcap >= 0) return &k_descend_mixed<true, 0>;
  DescMixedFn f = desc_mixed_fixed<33>(P.m);
  return f ? f : &k_descend_mixed<false, 0>;
}

// a4 in the mixed tier, binary64 finish, once per root.
//
// About three in four descents repeat a root (Table newtonSteps), and the
// repeats come from starts anywhere along the line, not only from the
// neighbouring ones.  The binary32 end points of two descents that reached
// the same root agree to the binary32 floor (~1e-5 of the descent's
// largest step), while distinct roots sit at distances comparable to that
// step.  So the end points, conjugate-folded, are sorted by Re, and an end
// point that lies within FINISH_SAME (1e-4) of the smaller of the two
// descent scales from one of its FINISH_SCAN sorted predecessors follows
// that predecessor: only the head of each group gets the binary64 Newton
// steps, and followers take the head's result (the root set would merge
// them anyway).  A wrong merge can only drop one of the c_L descents of a
// root; the count check then reports it and the tier falls back to
// binary64 (measured: 3e-3 instead of 1e-4 already merges distinct roots
// at p_24).  A group whose scan would run past FINISH_SCAN predecessors
// gets a head of its own: one more finish, never a wrong merge.
constexpr float FINISH_SAME2 = 1e-8f;  // (1e-4)^2 of the squared scale h1
constexpr int FINISH_SCAN = 32;

// The left tip c = -2 (Sec. 6.3.2): the real roots there close in on one
// another faster than the binary32 descents resolve (at p_30 two real roots
// 1.4e-12 apart near -2 + 3.9e-4, one of them reached by no binary32
// descent).  Descents that end within tip_box of -2 are redone in binary64
// from their start (status 4).  Near -2 the real roots of a degree-d
// polynomial of the family are spaced as sqrt(c + 2) / d, so the region of
// spacings below a fixed threshold shrinks as 1 / d^2: tip_box =
// 1e-3 (d / 2^29)^2, 2.5 times the p_30 case (0.8 % of the descents there).
inline double tip_box(const PolyDev& P) { return 1e-3 * exp2(2.0 * (P.log2d - 29)); }
// Sort keys of the binary32 end points: Re in fixed point, 2^-37 per unit
// over [-2.25, 1.75) (every root of the family lies in Re in [-2, 1/4]),
// FINISH_KEY_BITS = 40 bits, so that five radix passes order them.  The map
// c -> floor((c + 2.25) 2^37) is monotone (non-decreasing), so the sort
// orders the end points by Re up to one bucket, FINISH_BUCKET wide.
constexpr int FINISH_KEY_BITS = 40;
constexpr double FINISH_BUCKET = 7.275957614183426e-12;  // 2^-37
constexpr uint64_t TIP_KEY = (1ull << FINISH_KEY_BITS) - 2;  // above every finite key, below the rest
constexpr uint64_t REST_KEY = (1ull << FINISH_KEY_BITS) - 1;
// The key's bits above FINISH_KEY_BITS carry the descent's squared scale
// h1 (binary32, its low 8 bits dropped: rounded down, so the grouping test
// only tightens) through the sort, which orders the low 40 bits only: the
// group scan reads it from the sorted keys instead of gathering it.
__device__ __forceinline__ uint64_t with_scale(uint64_t key, float h1) {
  return key | ((uint64_t)(__float_as_uint(fmaxf(h1, 0.f)) >> 8) << FINISH_KEY_BITS);
}
__device__ __forceinline__ float key_scale(uint64_t key) {
  return __uint_as_float((unsigned)(key >> FINISH_KEY_BITS) << 8);
}
__device__ __forceinline__ uint64_t finish_key(double re) {
  // floor((re + 2.25) 2^37) = floor(re 2^37) + 2.25 2^37, the first term an
  // arithmetic shift of re's significand (integer pipe only: on GB300 the
  // binary64 pipe issues at 1/64 of the binary32 rate)
  const long long b = __double_as_longlong(re);
  const int E = (int)((b >> 52) & 0x7ff);
  const long long M = (b & 0x000fffffffffffffll) | (E ? 0x0010000000000000ll : 0ll);
  const int sh = min(63, 1038 - max(E, 1));  // re 2^37 = M 2^(E' - 1038), E' = max(E, 1)
  long long k;
  if (sh <= 0) k = b < 0 ? -0x7fffffffffffll : 0x7fffffffffffll;  // |re| >= 2^14: clamped below
  else if (b >= 0) k = M >> sh;
  else k = -(long long)(((unsigned long long)M + ((1ull << sh) - 1ull)) >> sh);
  k += 309237645312ll;  // 2.25 2^37
  const long long top = (long long)(1ull << (FINISH_KEY_BITS - 1)) - 1;
  return (uint64_t)(k < 0 ? 0 : k > top ? top : k);
}

// c32 = start + delta in binary64, folded into the upper half for the
// descents to finish (status 3), whose Re is their sort key; the others
// keep their end point and sort after them.  Descents that end in the tip
// box keep their start instead (status 4, key TIP_KEY, so that the stable
// sort lists them in index order between the two).  Counts both.
__global__ void k_c32_keys(int64_t count, double box, double2* __restrict__ starts, const float4* __restrict__ pack,
                           uint8_t* __restrict__ status, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, DevCounters* ctr) {
  // grid-stride over a bounded grid: the counts reach the two counters in a
  // few thousand atomics, not one per warp of the 2^28 descents.  Four
  // elements a round, all loaded before any is stored (the loads of a round
  // are in flight together; a load of starts cannot pass an earlier store
  // to it).
  constexpr int U = 4;
  unsigned long long n3 = 0, n4 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint64_t kx = f64_key(-2.0 + box), ky = f64_key(box);
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < count; i0 += U * stride) {
    float4 q[U];
    double2 c0[U];
    uint8_t st[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < count) {
        q[u] = pack[i];
        c0[u] = starts[i];
        st[u] = status[i];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= count) break;
      // the binary32 deltas widen on the integer pipe (f64_of_f32: a
      // subnormal delta, far below half an ulp of the start, becomes 0)
      double2 c = make_double2(c0[u].x + f64_of_f32(q[u].x), c0[u].y + f64_of_f32(q[u].y));
      const bool fin = st[u] == 3;
      // Im c < 0 (sign bit set, not -0): fold into the upper half
      const long long by = __double_as_longlong(c.y);
      if (fin && by < 0 && (by << 1) != 0) c.y = __longlong_as_double(by & 0x7fffffffffffffffll);
      uint64_t key = REST_KEY;
      // the tip box, compared on order-preserving integer keys
      if (fin && f64_key(c.x) < kx && f64_key(c.y) < ky) {
        status[i] = 4;  // redone in binary64 from c0
        key = TIP_KEY;
        ++n4;
      } else {
        starts[i] = c;
        if (fin) {
          key = with_scale(finish_key(c.x), q[u].z);
          ++n3;
        }
      }
      keys[i] = key;
      vals[i] = (uint32_t)i;
    }
  }
  warp_add_u64(&ctr->n_c32_fin, n3);
  warp_add_u64(&ctr->n_tip64, n4);
}

// list2 of the descents to redo in binary64: sorted positions n3 .. n3+n4
// (status 4, in index order)
__global__ void k_tip_list(const uint32_t* __restrict__ vals, const unsigned long long* __restrict__ n3,
                           const unsigned long long* __restrict__ n4, uint32_t* __restrict__ list2) {
  const int64_t a = (int64_t)*n3, m = (int64_t)*n4;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    list2[t] = vals[a + t];
}

// The descents redone in binary64 join the list of finished heads
// (list[*nlist ..]) and are counted; k_finish_count then moves *nlist.
// Grid-stride: the list is about 1 % of the descents.
__global__ void k_finish_append(const uint32_t* __restrict__ list2, const unsigned long long* __restrict__ n2,
                                uint32_t* __restrict__ list, const unsigned long long* __restrict__ nlist,
                                int64_t cap, const uint8_t* __restrict__ status, DevCounters* ctr) {
  const int64_t m = (int64_t)*n2, base = (int64_t)*nlist;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long nconv = 0, ndiv = 0, nto = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m && base + t < cap; t += stride) {
    const uint32_t i = list2[t];
    list[base + t] = i;
    const uint8_t st = status[i];
    nconv += st == 0;
    ndiv += st == 1;
    nto += st == 2;
  }
  warp_add_u64(&ctr->n_conv, nconv);
  warp_add_u64(&ctr->n_diverge, ndiv);
  warp_add_u64(&ctr->n_timeout, nto);
}
__global__ void k_finish_count(unsigned long long* nlist, const unsigned long long* n2, int64_t cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const unsigned long long t = *nlist + *n2;
    *nlist = t < (unsigned long long)cap ? t : (unsigned long long)cap;
  }
}

// head[p] = 1 for a sorted position p whose end point starts a group;
// link[p] = p - q for a follower of the sorted position q (0 otherwise)
__global__ void k_finish_heads(int64_t count, const uint32_t* __restrict__ vals,
                               const uint64_t* __restrict__ skeys, const double2* __restrict__ c32,
                               const unsigned long long* __restrict__ n3, uint32_t* __restrict__ head,
                               uint8_t* __restrict__ link) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  uint32_t h = 0;
  uint8_t lk = 0;
  // the n3 end points to finish (status 3) sort first: their keys lie below TIP_KEY
  if (p < (int64_t)*n3) {
    const uint32_t i = vals[p];
    h = 1;
    const double2 a = c32[i];
    const float ha = key_scale(skeys[p]);
    const float reach2 = FINISH_SAME2 * ha;  // min(ha, hb) <= ha
    for (int k = 1; k <= FINISH_SCAN && k <= p; ++k) {
      const uint32_t j = vals[p - k];
      const double2 b = c32[j];
      // the differences in binary64, the tests in binary32 (the differences
      // truncated on the integer pipe: never larger, so the scan never stops
      // early)
      const float ex = f32_trunc(a.x - b.x), ey = f32_trunc(a.y - b.y);
      // sorted by Re up to one bucket: every earlier entry lies below
      // b.x + FINISH_BUCKET, so none is within reach once ex - bucket is
      const float eb = ex - (float)FINISH_BUCKET;
      if (eb > 0.f && eb * eb > reach2) break;
      const float sc = fminf(ha, key_scale(skeys[p - k]));
      if (fmaf(ex, ex, ey * ey) <= FINISH_SAME2 * sc) {
        h = 0;
        lk = (uint8_t)k;
        break;
      }
    }
  }
  head[p] = h;
  link[p] = lk;
}

// list[pos[p]] = original index of the head at sorted position p
__global__ void k_finish_list(int64_t count, const uint32_t* __restrict__ head, const uint32_t* __restrict__ pos,
                              const uint32_t* __restrict__ vals, uint32_t* __restrict__ list) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count && head[p]) list[pos[p]] = vals[p];
}

// Binary64 Newton steps (eq. Newton) from each head's binary32 end point
// until |step| < tol (normally two steps) or the rounding floor.
// Persistent, with per-lane refill by warp vote (as k_descend): a lane that
// finished takes the next head of the list at once, so the warp never waits
// for its slowest finish (one to six steps) before starting new ones.
__global__ void __launch_bounds__(128) k_finish_f64(PolyDev P, const uint32_t* __restrict__ list,
                                                    const unsigned long long* __restrict__ nlist,
                                                    int64_t cap_list, double tol2, int cap,
                                                    const double2* __restrict__ c32,
                                                    double2* __restrict__ cand,
                                                    uint8_t* __restrict__ status,
                                                    unsigned long long* queue, DevCounters* ctr) {
  const unsigned lane = threadIdx.x & 31;
  const int64_t nl = (int64_t)*nlist < cap_list ? (int64_t)*nlist : cap_list;
  const float tol2f = f32_trunc(tol2), tol2q = 0.0625f * tol2f;  // tol^2, (tol / 4)^2
  int64_t t = -1;  // position in the list of this lane's finish
  double zx = 0.0, zy = 0.0;
  float prev2 = 3.0e38f;
  int it = 0;
  bool drained = false;  // warp-uniform: the list is handed out
  unsigned long long s64 = 0;
  for (;;) {
    const unsigned need = drained ? 0u : __ballot_sync(0xffffffffu, t < 0);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long b0 = 0;
      if ((int)lane == leader) b0 = atomicAdd(queue, (unsigned long long)__popc(need));
      b0 = __shfl_sync(0xffffffffu, b0, leader);
      if (t < 0) {
        t = (int64_t)(b0 + __popc(need & lanemask_lt()));
        if (t < nl) {
          const double2 z = c32[list[t]];
          zx = z.x;
          zy = z.y;
          it = 0;
          prev2 = 3.0e38f;
        }
      }
      if ((int64_t)(b0 + __popc(need)) >= nl) drained = true;
    }
    const bool active = t >= 0 && t < nl;
    if (!__any_sync(0xffffffffu, active)) break;
    if (active) {
      double vr, vi;
      float dr, di, kr, ki;
      orbit_f64_d32_k(P.m, P.lcap, zx, zy, vr, vi, dr, di, kr, ki);
      // the quotient in binary32: the derivative is binary32 already, and a
      // step accurate to 1e-7 of itself leaves ~1e-7 q besides the quadratic
      // K q^2 -- far below tol for the q ~ 1e-5 of a descent's scale that
      // the binary32 phase leaves; binary64 only for the value and z - q
      float qr, qi;
      if (!cdiv_f32s(f32_trunc(vr), f32_trunc(vi), dr, di, qr, qi)) {
        double qd, qe;  // a derivative out of binary32's scaled range: binary64
        cdiv_f64(vr, vi, (double)dr, (double)di, qd, qe);
        qr = f32_trunc(qd);
        qi = f32_trunc(qe);
      }
      zx -= f64_of_f32(qr);
      zy -= f64_of_f32(qi);
      ++it;
      ++s64;
      const float s2 = fmaf(qr, qr, qi * qi);
      // the next step, predicted: q^2 P''/(2P') (binary32); NaN or inf never accepts
      const float q2r = fmaf(qr, qr, -qi * qi), q2i = 2.f * qr * qi;
      const float pr = fmaf(q2r, kr, -q2i * ki), pi = fmaf(q2r, ki, q2i * kr);
      const float pred2 = fmaf(pr, pr, pi * pi);
      const float fzx = f32_trunc(zx), fzy = f32_trunc(zy);
      // binary64 rounding floor (16 ulp of the larger of 1 and |z|), in binary32
      const float fl = (1.f + fabsf(fzx) + fabsf(fzy)) * 3.552713678800501e-15f;
      int outcome = -1;
      if (!finite2(zx, zy) || fmaf(fzx, fzx, fzy * fzy) > 1e4f) outcome = 1;
      else if (s2 < tol2f) outcome = 0;
      // quadratic regime (the next step under a quarter of this one) and the
      // next step under tol / 4: c - q is the root to within tol / 4
      else if (pred2 <= tol2q && pred2 <= 0.0625f * s2) outcome = 0;
      else if (s2 >= 0.25f * prev2 && s2 < fl * fl) outcome = 0;  // rounding floor
      else if (it >= cap) outcome = 2;
      prev2 = s2;
      if (outcome >= 0) {
        const uint32_t i = list[t];
        cand[i] = make_double2(zx, zy);
        status[i] = (uint8_t)outcome;
        t = -1;
      }
    }
  }
  warp_add_u64(&ctr->desc_newton, s64);
  warp_add_u64(&ctr->finish_newton, s64);
}

// Followers take their head's result (following the links back in sorted
// order, each at most FINISH_SCAN positions); descents discarded by the
// binary32 phase (status 1, 2, already counted there) keep their binary32
// end point.  The outcomes of the finished groups are counted here.
__global__ void k_finish_followers(int64_t count, const uint32_t* __restrict__ vals,
                                   const uint32_t* __restrict__ head, const uint8_t* __restrict__ link,
                                   const double2* __restrict__ c32, double2* __restrict__ cand,
                                   uint8_t* __restrict__ status, DevCounters* ctr) {
  unsigned long long nconv = 0, ndiv = 0, nto = 0;
  // sorted positions below n3 hold the end points that were to finish (status 3)
  const int64_t n3 = (int64_t)ctr->n_c32_fin;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count;
       p += (int64_t)gridDim.x * blockDim.x) {  // grid-stride: few counter atomics
    const uint32_t i = vals[p];
    bool finished = head[p] != 0;
    uint8_t st = finished ? status[i] : (p < n3 ? 3 : 0);  // a head's outcome of the finish
    if (p < n3 && !finished) {
      int64_t q = p - link[p];
      for (int g = 0; g < 4096 && !head[q] && link[q]; ++g) q -= link[q];
      if (head[q]) {
        const uint32_t j = vals[q];
        cand[i] = cand[j];
        st = status[j];
      } else {  // unresolved (never seen): no root from this descent
        cand[i] = c32[i];
        st = 2;
      }
      status[i] = st;
      finished = true;
    } else if (!finished) {
      cand[i] = c32[i];
    }
    if (finished) {
      nconv += st == 0;
      ndiv += st == 1;
      nto += st == 2;
    }
  }
  warp_add_u64(&ctr->n_conv, nconv);
  warp_add_u64(&ctr->n_diverge, ndiv);
  warp_add_u64(&ctr->n_timeout, nto);
}

cudaError_t launch_seed_lift_mixed(const PolyDev& P, double lambda0, int64_t N0, int shrink_steps,
                                   double2* seeds, uint8_t* seed_bad, DevCounters* ctr, cudaStream_t s) {
  if (P.m > MIX_MAXM) return cudaErrorInvalidValue;
  int log2N0 = 0;
  while ((int64_t(1) << log2N0) < N0) ++log2N0;
  const int64_t n = N0 / 2 + 1;
  const int bs = 128;
  const size_t smem = (size_t)P.m * bs * sizeof(float2);
  MT_COUNT_LAUNCH(1);
  k_seed_lift_mixed<<<(unsigned)((n + bs - 1) / bs), bs, smem, s>>>(P, lambda0, N0, log2N0,
                                                                    shrink_steps, seeds, seed_bad, ctr);
  return cudaGetLastError();
}

cudaError_t launch_walk_mixed(const PolyDev& P, double lambda0, int M, int every, int64_t L,
                              int64_t nchunks, int K, const double2* seeds, double2* starts,
                              uint8_t* chunk_fail, DevCounters* ctr, cudaStream_t s, int block, int64_t j0,
                              int64_t nch) {
  if (P.m > MIX_MAXM) return cudaErrorInvalidValue;
  if (nch < 0) nch = nchunks - j0;
  if (nch <= 0) return cudaSuccess;
  const int bs = (block >= 32 && block <= 256 && block % 32 == 0) ? block : 64;
  const size_t smem = (size_t)P.m * bs * sizeof(float2);
  const int64_t grid = (nch + bs - 1) / bs;
  const WalkMixedFn kwalk = walk_mixed_kernel(P);
  MT_COUNT_LAUNCH(1);
  cudaError_t e = ktimer_begin(KS_WALK, s);
  if (e != cudaSuccess) return e;
  kwalk<<<(unsigned)grid, bs, smem, s>>>(P, lambda0, M, every, L, nchunks, K, seeds, starts, chunk_fail, ctr, j0,
                                         nch, j0 * L / every);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return ktimer_end(s);
}

// The anchor buffer: one slot of 32 orbits per warp of the descent's grid
// (at most DM_MAX_WARPS warps).
size_t mixed_anchor_bytes(const PolyDev& P, int64_t count) {
  (void)count;
  const int m1 = P.m > 1 ? P.m - 1 : 1;
  return (size_t)DM_MAX_WARPS * ((size_t)32 * m1 + 80) * sizeof(float2) + 256;
}

cudaError_t launch_descend_mixed(const PolyDev& P, double2* starts, int64_t count, double tol, int cap,
                                 double2* cand, uint8_t* status, void* anchors, const FinishScratch& fin,
                                 DevCounters* ctr, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (P.m > MIX_MAXM) return cudaErrorInvalidValue;
  const int bs = DM_BS;
  const size_t smem = (size_t)(P.m > 1 ? P.m - 1 : 1) * (bs + 1) * sizeof(float2);
  const DescMixedFn kdesc = desc_mixed_kernel(P);
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024 &&  // long orbits: opt in to more than 48 KB
      (e = cudaFuncSetAttribute(kdesc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kdesc, bs, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  float2* wbuf = (float2*)anchors;
  float4* pack = (float4*)cand;  // (delta, scale) until the finish writes the roots
  for (int64_t base = 0; base < count; base += MIX_BATCH) {
    const int64_t cnt = (count - base < MIX_BATCH) ? count - base : MIX_BATCH;
    int64_t grid = (int64_t)device_sm_count() * per_sm;
    const int64_t need = (cnt + bs - 1) / bs;
    if (grid > need) grid = need;
    if (grid > DM_MAX_WARPS / (bs / 32)) grid = DM_MAX_WARPS / (bs / 32);
    // the work queue (32-bit: a batch holds fewer than 2^31 starts) restarts
    // at 0 for every batch
    unsigned* q = (unsigned*)&ctr->queue_head;
    if ((e = cudaMemsetAsync(q, 0, sizeof(*q), s)) != cudaSuccess) return e;
    MT_COUNT_LAUNCH(1);
    if ((e = ktimer_begin(KS_DESC32, s)) != cudaSuccess) return e;
    kdesc<<<(unsigned)grid, bs, smem, s>>>(P, starts, base, cnt, wbuf, cap, pack, status, q, ctr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = ktimer_end(s)) != cudaSuccess) return e;
  }
  // binary64 finish, once per group of end points on the same root
  const unsigned nb = (unsigned)((count + bs - 1) / bs);
  unsigned long long* n2 = &ctr->n_tip64;
  if ((e = cudaMemsetAsync(n2, 0, sizeof(*n2), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(&ctr->n_c32_fin, 0, sizeof(*n2), s)) != cudaSuccess) return e;
  MT_COUNT_LAUNCH(1);
  const unsigned egrid = std::min<unsigned>(nb, (unsigned)device_sm_count() * 16);  // grid-stride kernels
  k_c32_keys<<<egrid, bs, 0, s>>>(count, tip_box(P), starts, pack, status, fin.keys, fin.vals, ctr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const uint64_t* skeys = nullptr;  // the sorted keys
  {
    bool in_alt = false;
    if ((e = radix_sort_bits(fin.keys, fin.vals, fin.keys_alt, fin.vals_alt, count, fin.radix_tmp, 0,
                             FINISH_KEY_BITS, &in_alt, s)) != cudaSuccess)
      return e;
    // the permutation is read from vals (vals_alt becomes the head list)
    if (in_alt && (e = cudaMemcpyAsync(fin.vals, fin.vals_alt, (size_t)count * sizeof(uint32_t),
                                       cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    skeys = in_alt ? fin.keys_alt : fin.keys;
  }
  MT_COUNT_LAUNCH(1);
  k_finish_heads<<<nb, bs, 0, s>>>(count, fin.vals, skeys, starts, &ctr->n_c32_fin, fin.head, fin.link);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_exclusive_scan(fin.head, fin.pos, count, fin.scan_tmp, fin.nheads, s)) != cudaSuccess) return e;
  MT_COUNT_LAUNCH(1);
  k_finish_list<<<nb, bs, 0, s>>>(count, fin.head, fin.pos, fin.vals, fin.list);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    // persistent: 8 warps per SM keep the binary64 pipe busy (as k_descend)
    int fin_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fin_sm, k_finish_f64, bs, 0)) != cudaSuccess) return e;
    if (fin_sm > 2) fin_sm = 2;
    if (fin_sm < 1) fin_sm = 1;
    int64_t fgrid = (int64_t)device_sm_count() * fin_sm;
    if (fgrid > (int64_t)nb) fgrid = (int64_t)nb;
    unsigned long long* q = &ctr->queue_head;
    if ((e = cudaMemsetAsync(q, 0, sizeof(*q), s)) != cudaSuccess) return e;
    MT_COUNT_LAUNCH(1);
    if ((e = ktimer_begin(KS_FINISH, s)) != cudaSuccess) return e;
    k_finish_f64<<<(unsigned)fgrid, bs, 0, s>>>(P, fin.list, fin.nheads, count, tol * tol, 6, starts, cand, status,
                                                q, ctr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = ktimer_end(s)) != cudaSuccess) return e;
  }
  MT_COUNT_LAUNCH(1);
  k_finish_followers<<<egrid, bs, 0, s>>>(count, fin.vals, fin.head, fin.link, starts, cand, status, ctr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the tip box: binary64 descents from the starts (list in fin.pos, free
  // once the heads are listed), then counted with the heads
  const unsigned sgrid = (unsigned)device_sm_count() * 4;
  MT_COUNT_LAUNCH(1);
  k_tip_list<<<sgrid, bs, 0, s>>>(fin.vals, &ctr->n_c32_fin, n2, fin.pos);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_descend_list(P, starts, fin.pos, n2, count, tol, cap, cand, status, ctr, s)) != cudaSuccess)
    return e;
  MT_COUNT_LAUNCH(2);
  k_finish_append<<<sgrid, bs, 0, s>>>(fin.pos, n2, fin.list, fin.nheads, count, status, ctr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_finish_count<<<1, 32, 0, s>>>(fin.nheads, n2, count);
  return cudaGetLastError();
}

}  // namespace mt
