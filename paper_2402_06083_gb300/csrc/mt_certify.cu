// mt_certify.cu -- steps a6 (type of each root) and a7 (disk certificate).
//
// a6, exact type (eq. def:hyp, def:mis).  For a root c of p_n the exact
// period is the smallest k | n with p_k(c) = 0; for a root of s_{l,n}
// (eq. polyMisSimple) it is either a centre of period k | gcd(n, l-1) or a
// Misiurewicz point of type (l, k), k | n, with q_{l,k}(c) = p_{l+k}(c) -
// p_l(c) = 0.  "= 0" is decided by the Newton size |f/f'| < tau.  One orbit
// pass of length l + n gives every p_k and p'_k needed.
//
// a7, certificate.  Thm proofRoots: if f'(D(z0,R)) lies in a disk B' and
// R dist(0,B') > |f(z0)|, then f has exactly one root in D(z0,R).  The
// enclosures come from disk arithmetic (Thm diskArithmetic): centres rounded
// to nearest, radii rounded upward, each operation adding half an ulp of its
// rounded result plus half an ulp of each rounded real product.  ulp(x) is
// the paper's 2^(e(x)-N) (eq. defULP) with IEEE subnormals kept (the remark
// after Prop. rounding); the complex ulp sqrt(ulp(x)^2 + ulp(y)^2) is bounded
// above by ulp(x) + ulp(y).  The radius of root j is
// r_j = min(tol, 0.45 * distance to its nearest other root or conjugate),
// so passing disks are pairwise disjoint and, with count == degree, pair
// bijectively with the roots (proof of Thm certif).
#include "mt_common.cuh"

#include <cmath>
#include <cstring>
#include <limits>

namespace mt {

// ---------------------------------------------------------------------------
// a6

// Type code: p_n -> k (1..63); s_{l,n} -> k for Mis(l,k), 32 + k for Hyp(k);
// 255 if nothing matched.  The test |f| <= tau |f'| compares magnitudes, so
// it runs in binary32: the derivatives are binary32 (from rn32 of the
// binary64 orbit values), the value is truncated to binary32 on the integer
// pipe, and tau2 is tau^2 rounded to binary32 on the host.  A value whose
// square underflows binary32 passes (its Newton size is below tau unless
// |f'| is as small), and so does a derivative whose square overflows (a
// bounded orbit value over it has a Newton size far below tau).
__device__ __forceinline__ bool newton_small_f(double vr, double vi, float dr, float di, float tau2) {
  const float ar = f32_trunc(vr), ai = f32_trunc(vi);
  return fmaf(ar, ar, ai * ai) <= tau2 * fmaf(dr, dr, di * di);
}

// q_{l,n} (kind 2): 32 + k for Hyp(k), k | n (multiplicity eta_l(k)); k for
// Mis(l, k); 0 for Mis(j, k) with j < l (a root of q_{l-1,n} too).
__device__ __forceinline__ int type_of(const PolyDev& P, double cr, double ci, float tau2) {
  const int n = P.n;
  const int len = (P.kind == 0) ? n : P.l + n;
  const int g = (P.kind != 1) ? n : [&] {
    int a = n, b = P.l - 1;
    while (b) { int t = a % b; a = b; b = t; }
    return a;
  }();
  double zr = 0.0, zi = 0.0, lr = 0.0, li = 0.0;  // p_l
  float dzr = 0.f, dzi = 0.f, ldr = 0.f, ldi = 0.f;  // p'_l
  double l1r = 0.0, l1i = 0.0;                       // p_{l-1} (q_{l,n})
  float l1dr = 0.f, l1di = 0.f;
  int hyp = 0, mis = 0, earlier = 0;
  for (int k = 1; k <= len; ++k) {
    const float fr = __double2float_rn(zr), fi = __double2float_rn(zi);
    const float tfr = fr + fr, tfi = fi + fi;
    const float ndr = fmaf(tfr, dzr, fmaf(-tfi, dzi, 1.f));
    const float ndi = fmaf(tfr, dzi, tfi * dzr);
    const double tzr = twice_f64(zr);
    const double nzr = fma(zr, zr, fma(-zi, zi, cr));
    const double nzi = fma(tzr, zi, ci);
    zr = nzr; zi = nzi; dzr = ndr; dzi = ndi;
    if (!hyp && k <= g && (g % k) == 0 && newton_small_f(zr, zi, dzr, dzi, tau2)) hyp = k;
    if (P.kind != 0) {
      if (k == P.l) { lr = zr; li = zi; ldr = dzr; ldi = dzi; }
      const int kk = k - P.l;
      if (!mis && kk >= 1 && (n % kk) == 0 &&
          newton_small_f(zr - lr, zi - li, dzr - ldr, dzi - ldi, tau2))
        mis = kk;
    }
    if (P.kind == 2 && P.l >= 2) {  // q_{l-1,k}(c) = 0 for a k | n: preperiod below l
      if (k == P.l - 1) { l1r = zr; l1i = zi; l1dr = dzr; l1di = dzi; }
      const int kk = k - (P.l - 1);
      if (!earlier && kk >= 1 && (n % kk) == 0 &&
          newton_small_f(zr - l1r, zi - l1i, dzr - l1dr, dzi - l1di, tau2))
        earlier = 1;
    }
  }
  if (P.kind == 0) return hyp ? hyp : 255;
  if (P.kind == 2) {
    if (hyp) return (32 + hyp < 64) ? 32 + hyp : 255;
    if (earlier) return 0;
    return (mis && mis < 32) ? mis : 255;
  }
  if (hyp) return (32 + hyp < 64) ? 32 + hyp : 255;
  if (mis) return mis < 32 ? mis : 255;
  return 255;
}

// tau^2 for newton_small_f, rounded to binary32 on the host
static float tau2_of(double tau) { return (float)(tau * tau); }

__global__ void k_classify(PolyDev P0, double2* __restrict__ reps,
                           const unsigned long long* __restrict__ n_reps, int64_t cap, float tau2,
                           int polish, uint8_t* __restrict__ type, uint32_t* __restrict__ mult,
                           DevCounters* ctr, SegView sv) {
  __shared__ unsigned int hist[64];
  for (int q = threadIdx.x; q < 64; q += blockDim.x) hist[q] = 0;
  __syncthreads();
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nr = (int64_t)*n_reps;
  unsigned long long nreal = 0, nmult = 0;
  if (u < cap) {
    if (u < nr) {
      const uint16_t sg = sv.rep_seg ? sv.rep_seg[u] : 0;
      const PolyDev P = sv.tab ? sv.tab[sg] : P0;
      double2 z = reps[u];
      if (polish) {
        double vr, vi, dr, di, qr, qi;
        eval_P(P, z.x, z.y, vr, vi, dr, di);
        cdiv_f64(vr, vi, dr, di, qr, qi);
        if (finite2(qr, qi)) {
          z.x -= qr;
          if (z.y != 0.0) z.y -= qi;
          reps[u] = z;
        }
      }
      const int t = type_of(P, z.x, z.y, tau2);
      const unsigned m = (z.y == 0.0) ? 1u : 2u;
      type[u] = (uint8_t)t;
      mult[u] = m;
      nreal += (m == 1);
      // q_{l,n}: Hyp(k) counts eta_l(k) = floor((l-1)/k) + 2 times (Thm fact_mis)
      nmult += (P.kind == 2 && t > 32 && t < 64) ? (unsigned long long)m * ((P.l - 1) / (t - 32) + 2) : m;
      if (t < 64) atomicAdd(&hist[t], m);
      if (sv.pstat) {
        unsigned long long* ps = sv.pstat + (size_t)sg * PSTAT_W;
        atomicAdd(&ps[0], 1ull);
        if (m == 1) atomicAdd(&ps[1], 1ull);
        atomicAdd(&ps[2], (unsigned long long)m);
        if (t < 64) atomicAdd(&ps[4 + t], (unsigned long long)m);
      }
    } else {
      mult[u] = 0;
    }
  }
  warp_add_u64(&ctr->n_reps_real, nreal);
  warp_add_u64(&ctr->n_mult_full, nmult);
  __syncthreads();
  for (int q = threadIdx.x; q < 64; q += blockDim.x)
    if (hist[q]) atomicAdd(&ctr->type_count[q], (unsigned long long)hist[q]);
}

cudaError_t launch_classify(const PolyDev& P, double2* reps, const unsigned long long* n_reps,
                            int64_t cap, double tau, int polish, uint8_t* type, uint32_t* mult,
                            DevCounters* ctr, cudaStream_t s, SegView sv) {
  if (cap <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_classify<<<(unsigned)((cap + 127) / 128), 128, 0, s>>>(P, reps, n_reps, cap, tau2_of(tau), polish,
                                                           type, mult, ctr, sv);
  return cudaGetLastError();
}

__global__ void k_type_only(PolyDev P, const double2* __restrict__ roots, int64_t count, float tau2,
                            uint8_t* __restrict__ type) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double2 z = roots[i];
  type[i] = (uint8_t)type_of(P, z.x, z.y, tau2);
}

// q_{l,n}: per output root the exact type (eq. def:mis) and its multiplicity
// (Thm fact_mis).  Hyp(k): the smallest k | n with p_k(c) = 0, preperiod 0,
// multiplicity eta_l(k) = floor((l-1)/k) + 2.  Otherwise Mis(j, k): k the
// smallest divisor of n with q_{l,k}(c) = 0, then j the smallest preperiod
// with q_{j,k}(c) = 0 (q_{j,k} vanishes on Mis(j0,k0) exactly when j >= j0 and
// k0 | k); multiplicity 1.  255 / 0 where nothing matched.  The orbit (at
// most 40 steps) is kept whole, in local memory: one pass per root.
__global__ void k_type_q(PolyDev P, const double2* __restrict__ roots, int64_t count, float tau2,
                         uint8_t* __restrict__ pre, uint8_t* __restrict__ per, uint8_t* __restrict__ mult) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double2 c = roots[i];
  const int l = P.l, n = P.n, L = P.l + P.n;
  double zr[41], zi[41];
  float dr[41], di[41];
  zr[0] = zi[0] = 0.0;
  dr[0] = di[0] = 0.f;
  for (int k = 1; k <= L; ++k) {
    const float fr = __double2float_rn(zr[k - 1]), fi = __double2float_rn(zi[k - 1]);
    dr[k] = fmaf(fr + fr, dr[k - 1], fmaf(-(fi + fi), di[k - 1], 1.f));
    di[k] = fmaf(fr + fr, di[k - 1], (fi + fi) * dr[k - 1]);
    zr[k] = fma(zr[k - 1], zr[k - 1], fma(-zi[k - 1], zi[k - 1], c.x));
    zi[k] = fma(zr[k - 1] + zr[k - 1], zi[k - 1], c.y);
  }
  int a = -1, b = -1;
  for (int k = 1; k <= n && a < 0; ++k)
    if (n % k == 0 && newton_small_f(zr[k], zi[k], dr[k], di[k], tau2)) { a = 0; b = k; }
  for (int k = 1; k <= n && a < 0; ++k) {
    if (n % k || !newton_small_f(zr[l + k] - zr[l], zi[l + k] - zi[l], dr[l + k] - dr[l], di[l + k] - di[l], tau2))
      continue;
    for (int j = 2; j <= l; ++j)
      if (newton_small_f(zr[j + k] - zr[j], zi[j + k] - zi[j], dr[j + k] - dr[j], di[j + k] - di[j], tau2)) {
        a = j;
        b = k;
        break;
      }
  }
  if (pre) pre[i] = a < 0 ? 255 : (uint8_t)a;
  if (per) per[i] = b < 0 ? 255 : (uint8_t)b;
  if (mult) mult[i] = a < 0 ? 0 : (uint8_t)(a == 0 ? (l - 1) / b + 2 : 1);
}

cudaError_t launch_type_q(const PolyDev& P, const double2* roots, int64_t count, double tau, uint8_t* pre,
                          uint8_t* per, uint8_t* mult, cudaStream_t s) {
  if (count <= 0 || P.l + P.n > 40) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_type_q<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(P, roots, count, tau2_of(tau), pre, per, mult);
  return cudaGetLastError();
}

cudaError_t launch_type_only(const PolyDev& P, const double2* roots, int64_t count, double tau,
                             uint8_t* type, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_type_only<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(P, roots, count, tau2_of(tau), type);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a7: disk arithmetic (Thm diskArithmetic) with binary64 centres for the
// value and binary32 centres for the derivative.
//
// The value centres follow exactly the FMA sequence of the binary64 point
// orbit;
// each rounding adds half an ulp of its rounded result to the radius (Prop.
// rounding).  With FMA only the products that are rounded separately
// contribute an ulp term -- a refinement of the theorem's R_*, whose four
// product terms assume every product is rounded.  Radii are upper bounds
// kept in binary32 with every operation rounded upward (__f*_ru): a radius
// only needs a few correct bits, and this keeps the binary64 pipe for the
// centres.  Along the orbit the ulp terms are bounded through the moduli
// of the rounded results (below); the two sums of s_{l,n} and q_{l,n} take
// them from the binary64 exponent bits as binary32 powers of two rounded
// upward (2^-149 when the true ulp is smaller).

// upper bound, in binary32, of the paper's ulp(x) = 2^(e(x) - 53) for a
// binary64 x (2^-1074 for subnormals and zero)
__device__ __forceinline__ float ulp_ub(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  const int p = (e == 0) ? -1074 : e - 1075;
  if (p < -149) return 1.40129846e-45f;  // 2^-149 >= 2^p
  if (p > 127) return __int_as_float(0x7f800000);
  if (p >= -126) return __int_as_float((p + 127) << 23);
  return __int_as_float(1 << (p + 149));
}

// upper bound of |x + iy| in binary32 (the components bounded on the
// integer pipe, f32_abs_up)
__device__ __forceinline__ float abs_ub(double x, double y) {
  const float ax = f32_abs_up(x), ay = f32_abs_up(y);
  return __fsqrt_ru(__fmaf_ru(ax, ax, __fmul_ru(ay, ay)));
}
__device__ __forceinline__ float hsum_ru(float a, float b) {
  return __fmul_ru(0.5f, __fadd_ru(a, b));
}

// upper bound, in binary32, of ulp(x) for a binary32 x (2^-149 for
// subnormals and zero): ulp(x) = 2^(e(x) - 23)
__device__ __forceinline__ float ulp32_ub(float x) {
  const int e = (__float_as_int(x) >> 23) & 0xff;
  if (e == 0) return 1.40129846e-45f;
  if (e == 0xff) return __int_as_float(0x7f800000);
  const int p = e - 127 - 23;
  if (p >= -126) return __int_as_float((p + 127) << 23);
  return __int_as_float(1 << (p + 149));
}
__device__ __forceinline__ float abs_lb_f(float x, float y) {
  return __fsqrt_rd(__fmaf_rd(fabsf(x), fabsf(x), __fmul_rd(fabsf(y), fabsf(y))));
}

// Per-step bounds on the binary32 pipe.  Half an ulp of a rounded result x
// is at most 2^-53 |x| in binary64 and 2^-24 |x| in binary32 (x normal;
// below the normal range a floor of 2^-149, resp. 2^-150, per rounding
// covers it), so the rounding terms come from upper bounds of the results'
// moduli by binary32 operations rounded upward, instead of from their
// exponent bits.  |x| for a binary64 x is bounded by the next binary32 above
// |f32_trunc(x)| (trunc_abs_up), which also bounds |x - f32_trunc(x)| by
// the exact difference of the two.
__device__ __forceinline__ float trunc_abs_up(float t) {  // t = f32_trunc(x): >= |x|
  const int b = (__float_as_int(t) & 0x7fffffff) + 1;      // 2^-126 for t = 0, inf from the largest on
  return __int_as_float(min(max(b, 0x00800000), 0x7f800000));
}
// Upper bound of sqrt(x), x >= 0: sqrt.approx.f32 times 1 + 2^-19 rounded
// up; the argument is raised to 2^-126 first.  The approximation's relative
// error, measured on GB300 over every normal binary32, is below 2^-23.2;
// mt_check_sqrt_up repeats that check on the GPU at hand.
__device__ __forceinline__ float sqrt_up(float x) {
  float s;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(fmaxf(x, 1.17549435e-38f)));
  return __fmul_ru(s, 1.0000019073486328f);
}
// the Newton-size test of newton_small_f on the truncated value
__device__ __forceinline__ bool newton_small_ff(float ar, float ai, float dr, float di, float tau2) {
  return fmaf(ar, ar, ai * ai) <= tau2 * fmaf(dr, dr, di * di);
}

// One orbit over the disk D(c, rc) and over the point c at once (shared
// centres): returns the value centre V (binary64) with its point radius rv0,
// and the derivative centre W with its disk radius rw (W encloses
// P'(D(c, rc))).  The derivative only has to keep 0 out of B', so its
// centres run in binary32: z enters it as zf = f32_trunc(Z) (integer pipe),
// and the disk of z around zf is widened by |Z - zf| <= ulp(zf.x) +
// ulp(zf.y) (2^-126 for a component truncated to zero).
// TYPE: also the exact period of c as a root of p_n (kind 0), by the test
// of type_of (|p_k| <= tau |p'_k| for the smallest k | n) on these centres.
template <bool TYPE = false>
__device__ __forceinline__ void disk_orbit2(const PolyDev& P, double cx, double cy, float rc,
                                            double& Vx, double& Vy, float& rv0, float& Wx,
                                            float& Wy, float& rw, float tau2 = 0.f, int* hyp = nullptr) {
  constexpr float kU53 = 1.1102240834163406e-16f;  // 2^-53 (1 + 2^-20): covers |in_z|'s own rounding
  constexpr float kU24 = 5.9604644775390625e-08f;  // 2^-24
  const float kFloor64 = __int_as_float(3), kFloor32 = __int_as_float(2);  // 3 2^-149, 4 2^-150
  double zx = 0.0, zy = 0.0, czx = 0.0, czy = 0.0;
  float fx = 0.f, fy = 0.f;                      // f32_trunc(Z)
  float ax = 1.17549435e-38f, ay = 1.17549435e-38f;  // trunc_abs_up(fx), (fy): >= |Re Z|, |Im Z|
  float dx = 0.f, dy = 0.f, cdx = 0.f, cdy = 0.f;
  float rz0 = 0.f, rz = 0.f, rd = 0.f;  // radii: z (point), z (disk), z' (disk)
  float crz0 = 0.f, crd = 0.f;
  const float cxu = trunc_abs_up(f32_trunc(cx));  // >= |Re c|
  for (int k = 1; k <= P.m; ++k) {
    const float mz = sqrt_up(__fmaf_ru(ax, ax, __fmul_ru(ay, ay)));  // >= |Z| >= |zf|
    // z' = 2 z z' + 1 in binary32 around zf; |Z - zf| <= (ax - |fx|) + (ay - |fy|), both exact
    const float ez = __fadd_ru(ax - fabsf(fx), ay - fabsf(fy));
    const float rzz = __fadd_ru(rz, ez);
    const float md = sqrt_up(__fmaf_ru(dx, dx, __fmul_ru(dy, dy)));
    const float tfx = fx + fx, tfy = fy + fy;  // exact
    const float in_re = fmaf(-tfy, dy, 1.f);
    const float nd_x = fmaf(tfx, dx, in_re);
    const float p_im = tfy * dx;
    const float nd_y = fmaf(tfx, dy, p_im);
    const float sd = __fadd_ru(__fadd_ru(fabsf(in_re), fabsf(nd_x)), __fadd_ru(fabsf(p_im), fabsf(nd_y)));
    const float Rd = __fmaf_ru(kU24, sd, kFloor32);
    // radius of 2 (z z'): 2 (rzz rd + rzz |z'| + rd |zf|)
    const float prod = __fmaf_ru(rzz, rd, __fmaf_ru(rzz, md, __fmul_ru(rd, mz)));
    const float nrd = __fmaf_ru(2.f, prod, Rd);
    // z = z^2 + c in binary64: re = fma(zx, zx, fma(-zy, zy, cx)), im = fma(2zx, zy, cy)
    const double tzx = twice_f64(zx);
    const double in_z = fma(-zy, zy, cx);
    const double nz_x = fma(zx, zx, in_z);
    const double nz_y = fma(tzx, zy, cy);
    const float nfx = f32_trunc(nz_x), nfy = f32_trunc(nz_y);
    const float nax = trunc_abs_up(nfx), nay = trunc_abs_up(nfy);
    // |in_z| <= (|Re c| + |Im z|^2)(1 + 2^-53), |nz_x| <= nax, |nz_y| <= nay
    const float inb = __fmaf_ru(ay, ay, cxu);
    const float Rz = __fmaf_ru(kU53, __fadd_ru(__fadd_ru(inb, nax), nay), kFloor64);
    // radii of z^2 + C: 2 r |z| + r^2 (+ rc for the disk) + Rz
    const float mz2 = __fmul_ru(2.f, mz);
    const float nrz0 = __fmaf_ru(rz0, rz0, __fmaf_ru(mz2, rz0, Rz));
    const float nrz = __fadd_ru(__fmaf_ru(rz, rz, __fmaf_ru(mz2, rz, Rz)), rc);
    zx = nz_x; zy = nz_y; fx = nfx; fy = nfy; ax = nax; ay = nay; dx = nd_x; dy = nd_y;
    rz0 = nrz0; rz = nrz; rd = nrd;
    if (TYPE && !*hyp && (P.n % k) == 0 && newton_small_ff(fx, fy, dx, dy, tau2)) *hyp = k;
    if (k == P.lcap) { czx = zx; czy = zy; cdx = dx; cdy = dy; crz0 = rz0; crd = rd; }
  }
  if (P.lcap >= 0) {  // s_{l,n} = p_m + p_{l-1}, q_{l,n} = p_m - p_l: one disk sum each
    const double sg = (P.kind == 2) ? -1.0 : 1.0;
    const float sgf = (float)sg;
    const double vx = fma(sg, czx, zx), vy = fma(sg, czy, zy);
    const float wx = fmaf(sgf, cdx, dx), wy = fmaf(sgf, cdy, dy);
    rz0 = __fadd_ru(__fadd_ru(rz0, crz0), hsum_ru(ulp_ub(vx), ulp_ub(vy)));
    rd = __fadd_ru(__fadd_ru(rd, crd), hsum_ru(ulp32_ub(wx), ulp32_ub(wy)));
    zx = vx; zy = vy; dx = wx; dy = wy;
  }
  Vx = zx; Vy = zy; rv0 = rz0;
  Wx = dx; Wy = dy; rw = rd;
}

// The radius r = min(tol, 0.45 nn), nn the distance to the nearest other
// root or conjugate, kept as a binary32 lower bound: tol32 is the largest
// binary32 <= tol (host), the binary32 literals 0.45f and 0.9f lie below
// 0.45 and 0.9, and every step rounds down.  Two neighbours' radii then add
// to at most 0.9 of their binary64 distance, whose rounding (relative
// 2^-51) cannot close the gap, so passing disks stay disjoint.  The scan
// over the Re-sorted list stops at the first point with |Re dv| >= W, W >=
// tol / 0.45 (host, rounded up); |dx| >= W is an integer compare of the
// binary64 bit patterns (both non-negative), and only the rare points inside
// the window reach the binary64 distance.
__device__ __forceinline__ float rad_conj(double cy) {  // 0.45 |c - conj(c)| = 0.9 |Im c|
  return __fmul_rd(0.9f, fabsf(f32_trunc(cy)));
}
__device__ __forceinline__ float rad_near(double d2) {  // 0.45 sqrt(d2)
  return __fmul_rd(0.45f, __fsqrt_rd(f32_trunc(d2)));
}
__device__ __forceinline__ bool outside_window(double dx, long long Wbits) {
  return (__double_as_longlong(dx) & 0x7fffffffffffffffll) >= Wbits;
}
struct RadCap {
  float tol32;     // largest binary32 <= tol
  long long Wbits; // bits of W >= tol / 0.45
};
static RadCap rad_cap_of(double tol) {
  RadCap r;
  float t = (float)tol;
  if ((double)t > tol) t = std::nextafter(t, 0.f);
  r.tol32 = t;
  const double W = std::nextafter(tol / 0.45, std::numeric_limits<double>::infinity());
  std::memcpy(&r.Wbits, &W, sizeof W);
  return r;
}
// radii at least 2^-126 (normal binary32) are reported exactly in binary64
#define MT_RAD_MIN 1.17549435e-38f

// Certify the points of 'pts' (sorted by Re through 'order', or already
// sorted when order == nullptr).  upper: the list holds one representative
// per conjugate pair, so conjugates count as neighbours too.
// q_{l,n}: a root typed Hyp(k) (type 33..63) is a multiple root of q but a
// simple root of p_n, and is proven as a root of p_n; the others as roots of q.
__global__ void k_certify(PolyDev P0, const double2* __restrict__ pts,
                          const uint32_t* __restrict__ order, const unsigned long long* n_pts_dev,
                          int64_t n_pts_host, RadCap rc, int upper, const uint32_t* __restrict__ mult,
                          uint8_t* __restrict__ pass, double* __restrict__ radius,
                          DevCounters* ctr, SegView sv, const uint8_t* __restrict__ type) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = n_pts_dev ? (int64_t)*n_pts_dev : n_pts_host;
  unsigned long long npass = 0, overflow = 0;
  double radd = 0.0;
  bool ok = false, valid = p < n;
  if (valid) {
    const int64_t ip = order ? (int64_t)order[p] : p;
    const double2 c = pts[ip];
    const uint16_t sg = sv.rep_seg ? sv.rep_seg[p] : 0;  // (batch mode: pts are reps, no order)
    PolyDev P = sv.tab ? sv.tab[sg] : P0;
    if (P.kind == 2 && type && type[ip] > 32 && type[ip] < 64) {
      P.kind = 0;  // p_n
      P.m = P.n;
      P.lcap = -1;
    }
    // nearest neighbour (and conjugates) within the window W
    float rad = rc.tol32;
    if (upper && c.y != 0.0) rad = fminf(rad, rad_conj(c.y));
    int scanned = 0;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int64_t q = p + dir; q >= 0 && q < n; q += dir) {
        if (sv.rep_seg && sv.rep_seg[q] != sg) break;  // another polynomial of the batch
        const double2 v = pts[order ? (int64_t)order[q] : q];
        const double dx = v.x - c.x;
        if (outside_window(dx, rc.Wbits)) break;
        const double dy = v.y - c.y;
        double d2 = fma(dx, dx, dy * dy);
        if (upper) {
          const double ey = v.y + c.y;
          d2 = fmin(d2, fma(dx, dx, ey * ey));
        }
        rad = fminf(rad, rad_near(d2));
        if (++scanned >= 4096) { overflow = 1; break; }
      }
    }
    // sup |P(c)| from the point orbit, B' = D(W, rw) encloses P'(D(c, rad)).
    // Between two close roots the critical point sits about half-way, so a
    // disk of 0.45 nn may bring 0 into B'; then retry with rad / 4, / 16, / 64
    // (any passing radius proves the root; the disks stay disjoint).
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
      if (attempt) rad = __fmul_rd(rad, 0.25f);
      double Vx, Vy;
      float rv0, Wx, Wy, rw;
      disk_orbit2(P, c.x, c.y, rad, Vx, Vy, rv0, Wx, Wy, rw);
      const float fz = __fadd_ru(abs_ub(Vx, Vy), rv0);
      const float dist = __fsub_rd(abs_lb_f(Wx, Wy), rw);
      ok = isfinite(fz) && isfinite(dist) && dist > 0.f && rad >= MT_RAD_MIN && __fmul_rd(rad, dist) > fz;
    }
    radd = f64_of_f32(rad);
    pass[ip] = ok ? 1 : 0;
    if (radius) radius[ip] = radd;
    npass = ok ? (mult ? mult[p] : 1u) : 0u;
    if (sv.pstat && npass) atomicAdd(&sv.pstat[(size_t)sg * PSTAT_W + 3], npass);
  }
  warp_add_u64(&ctr->n_cert_pass, npass);
  if (overflow) atomicAdd(&ctr->cluster_overflow, 1ull);
  // radii are >= 0: their bit patterns order like the values
  const unsigned long long rb = (unsigned long long)__double_as_longlong(radd);
  warp_min_u64(&ctr->min_radius_bits, (valid && ok) ? rb : ~0ull);
  warp_max_u64(&ctr->max_radius_bits, (valid && ok) ? rb : 0ull);
}

// a6 + a7 fused for p_n (kind 0, one polynomial): the exact period of
// each representative comes from the centres of the certificate's first
// disk orbit (type_of's test on the binary64 point orbit, whose derivative
// centres differ from type_of's only by binary32 rounding), and
// its conjugate multiplicity (1 real, 2 otherwise) from Im = 0, which the
// root set made exact.  Writes what k_classify and k_certify write: type,
// mult, pass, radius and the counters; one orbit pass per root fewer.
__global__ void k_certify_typed(PolyDev P, const double2* __restrict__ pts, const unsigned long long* n_pts_dev,
                                int64_t cap, RadCap rc, float tau2, uint8_t* __restrict__ type,
                                uint32_t* __restrict__ mult, uint8_t* __restrict__ pass,
                                double* __restrict__ radius, DevCounters* ctr) {
  __shared__ unsigned int hist[64];
  for (int q = threadIdx.x; q < 64; q += blockDim.x) hist[q] = 0;
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)*n_pts_dev;
  unsigned long long npass = 0, overflow = 0, nreal = 0, nmult = 0;
  double radd = 0.0;
  bool ok = false;
  const bool valid = p < n && p < cap;
  if (valid) {
    const double2 c = pts[p];
    // Im c = 0 tested on the bits (+0 or -0)
    const bool real = (__double_as_longlong(c.y) << 1) == 0;
    const unsigned m = real ? 1u : 2u;
    float rad = rc.tol32;
    if (!real) rad = fminf(rad, rad_conj(c.y));
    int scanned = 0;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int64_t q = p + dir; q >= 0 && q < n; q += dir) {
        const double2 v = pts[q];
        const double dx = v.x - c.x;
        if (outside_window(dx, rc.Wbits)) break;
        const double dy = v.y - c.y, ey = v.y + c.y;
        rad = fminf(rad, rad_near(fmin(fma(dx, dx, dy * dy), fma(dx, dx, ey * ey))));
        if (++scanned >= 4096) { overflow = 1; break; }
      }
    }
    int hyp = 0;
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
      if (attempt) rad = __fmul_rd(rad, 0.25f);
      double Vx, Vy;
      float rv0, Wx, Wy, rw;
      if (attempt == 0) disk_orbit2<true>(P, c.x, c.y, rad, Vx, Vy, rv0, Wx, Wy, rw, tau2, &hyp);
      else disk_orbit2<false>(P, c.x, c.y, rad, Vx, Vy, rv0, Wx, Wy, rw);
      const float fz = __fadd_ru(abs_ub(Vx, Vy), rv0);
      const float dist = __fsub_rd(abs_lb_f(Wx, Wy), rw);
      ok = isfinite(fz) && isfinite(dist) && dist > 0.f && rad >= MT_RAD_MIN && __fmul_rd(rad, dist) > fz;
    }
    radd = f64_of_f32(rad);
    const int t = hyp ? hyp : 255;
    type[p] = (uint8_t)t;
    mult[p] = m;
    nreal += (m == 1);
    nmult += m;
    if (t < 64) atomicAdd(&hist[t], m);
    pass[p] = ok ? 1 : 0;
    if (radius) radius[p] = radd;
    npass = ok ? m : 0u;
  } else if (p < cap) {
    mult[p] = 0;
  }
  warp_add_u64(&ctr->n_cert_pass, npass);
  warp_add_u64(&ctr->n_reps_real, nreal);
  warp_add_u64(&ctr->n_mult_full, nmult);
  if (overflow) atomicAdd(&ctr->cluster_overflow, 1ull);
  const unsigned long long rb = (unsigned long long)__double_as_longlong(radd);
  warp_min_u64(&ctr->min_radius_bits, (valid && ok) ? rb : ~0ull);
  warp_max_u64(&ctr->max_radius_bits, (valid && ok) ? rb : 0ull);
  __syncthreads();
  for (int q = threadIdx.x; q < 64; q += blockDim.x)
    if (hist[q]) atomicAdd(&ctr->type_count[q], (unsigned long long)hist[q]);
}

cudaError_t launch_certify_typed(const PolyDev& P, const double2* reps, const unsigned long long* n_reps,
                                 int64_t cap, double tol, double tau, uint8_t* type, uint32_t* mult,
                                 uint8_t* pass, double* radius, DevCounters* ctr, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  if (P.kind != 0) return cudaErrorInvalidValue;
  MT_COUNT_LAUNCH(1);
  k_certify_typed<<<(unsigned)((cap + 127) / 128), 128, 0, s>>>(P, reps, n_reps, cap, rad_cap_of(tol),
                                                                 tau2_of(tau), type, mult, pass, radius, ctr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Newton-basin certificate (Thm proofContract): z* a simple root with
// |z0 - z*| < eta; if eps > 3 eta and P'(D(z0, eps)) lies in a disk B' with
// dist(0, B') > 2 diam(B'), then D(z0, eps) lies in the basin of attraction
// of z* for the Newton map.  eta comes from the localisation test itself:
// with B'_r enclosing P'(D(z0, r)) and r dist(0, B'_r) > |P(z0)|, the proof
// of Thm proofRoots places the root in D(z0, |P(z0)| / dist(0, B'_r)), so
// eta = |P(z0)|_ub / dist_lb (<= r).  eps runs over 0.25 nn, / 4, / 16, ...
// while eps > 3 eta; the first that passes is reported (0 if none).
__global__ void k_basin(PolyDev P, const double2* __restrict__ pts, const uint32_t* __restrict__ order,
                        int64_t n, const double* __restrict__ rin, double eps_max,
                        double* __restrict__ basin, DevCounters* ctr) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long npass = 0;
  if (p < n) {
    const int64_t ip = order[p];
    const double2 c = pts[ip];
    // nearest other root within 4 eps_max (the window of eps <= 0.25 nn)
    const double Wn = 4.0 * eps_max;
    double nn2 = Wn * Wn;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int64_t q = p + dir; q >= 0 && q < n && (q - p) * dir < 4096; q += dir) {
        const double2 v = pts[order[q]];
        const double dx = v.x - c.x;
        if (fabs(dx) >= Wn) break;
        const double dy = v.y - c.y;
        nn2 = fmin(nn2, fma(dx, dx, dy * dy));
      }
    }
    double out = 0.0;
    const double r = rin[ip];
    if (r > 0.0) {
      const float ru = __double2float_ru(r);
      double Vx, Vy;
      float rv0, Wx, Wy, rw;
      disk_orbit2(P, c.x, c.y, ru, Vx, Vy, rv0, Wx, Wy, rw);
      const float fz = __fadd_ru(abs_ub(Vx, Vy), rv0);
      const float dist = __fsub_rd(abs_lb_f(Wx, Wy), rw);
      if (isfinite(fz) && isfinite(dist) && dist > 0.f) {
        const float eta = fminf(__fdiv_ru(fz, dist), ru);
        double eps = fmin(eps_max, 0.25 * sqrt(nn2));
        for (int k = 0; k < 24 && eps > 3.0 * (double)eta; ++k, eps *= 0.25) {
          const float eu = __double2float_ru(eps);
          disk_orbit2(P, c.x, c.y, eu, Vx, Vy, rv0, Wx, Wy, rw);
          const float wl = abs_lb_f(Wx, Wy);
          // dist(0, B') = |W| - rw > 2 diam(B') = 4 rw
          if (isfinite(wl) && isfinite(rw) && __fsub_rd(wl, rw) > __fmul_ru(4.f, rw)) {
            out = (double)__double2float_rd(eps);
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

cudaError_t launch_basin(const PolyDev& P, const double2* pts, const uint32_t* order, int64_t count,
                         const double* radius, double eps_max, double* basin, DevCounters* ctr,
                         cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_basin<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(P, pts, order, count, radius, eps_max, basin,
                                                          ctr);
  return cudaGetLastError();
}

cudaError_t launch_certify(const PolyDev& P, const double2* reps, const unsigned long long* n_reps,
                           int64_t cap, double tol, const uint32_t* mult, uint8_t* pass,
                           double* radius, DevCounters* ctr, cudaStream_t s, SegView sv,
                           const uint8_t* type) {
  if (cap <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_certify<<<(unsigned)((cap + 127) / 128), 128, 0, s>>>(P, reps, nullptr, n_reps, cap, rad_cap_of(tol),
                                                          1, mult, pass, radius, ctr, sv, type);
  return cudaGetLastError();
}

// standalone certificate of an arbitrary list (sorted through 'order')
cudaError_t launch_certify_list(const PolyDev& P, const double2* pts, const uint32_t* order,
                                int64_t count, double tol, uint8_t* pass, double* radius,
                                DevCounters* ctr, cudaStream_t s, const uint8_t* type) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_certify<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(P, pts, order, nullptr, count,
                                                            rad_cap_of(tol), 0, nullptr, pass, radius, ctr,
                                                            SegView(), type);
  return cudaGetLastError();
}

// Every normal binary32 x: sqrt_up(x)^2 >= x (exact in binary64), and the
// largest relative error of the approximation itself.
__device__ unsigned long long g_sqrt_fail;
__device__ unsigned g_sqrt_maxrel;
__global__ void k_check_sqrt_up(unsigned long long count) {
  unsigned long long nf = 0;
  unsigned mr = 0;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float x = __uint_as_float(0x00800000u + (unsigned)i);
    const float su = sqrt_up(x);
    nf += !((double)su * (double)su >= (double)x);
    float s;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(s) : "f"(x));
    const double ex = sqrt((double)x);
    mr = max(mr, __float_as_uint((float)(fabs((double)s - ex) / ex)));
  }
  if (nf) atomicAdd(&g_sqrt_fail, nf);
  atomicMax(&g_sqrt_maxrel, mr);
}

cudaError_t check_sqrt_up(unsigned long long* n_fail, double* max_rel, cudaStream_t s) {
  const unsigned long long zero = 0;
  const unsigned zu = 0;
  cudaError_t e;
  if ((e = cudaMemcpyToSymbolAsync(g_sqrt_fail, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyToSymbolAsync(g_sqrt_maxrel, &zu, sizeof zu, 0, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  MT_COUNT_LAUNCH(1);
  k_check_sqrt_up<<<(unsigned)device_sm_count() * 16, 256, 0, s>>>(0x7f7fffffull - 0x00800000ull + 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  unsigned mr = 0;
  if ((e = cudaMemcpyFromSymbolAsync(n_fail, g_sqrt_fail, sizeof *n_fail, 0, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemcpyFromSymbolAsync(&mr, g_sqrt_maxrel, sizeof mr, 0, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  float f;
  std::memcpy(&f, &mr, sizeof f);
  *max_rel = f;
  return cudaSuccess;
}

}  // namespace mt
