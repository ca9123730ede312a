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

namespace mt {

// ---------------------------------------------------------------------------
// a6
__device__ __forceinline__ bool newton_small(double vr, double vi, double dr, double di,
                                             double tau) {
  // |v| <= tau |dv|, compared squared
  return fma(vr, vr, vi * vi) <= tau * tau * fma(dr, dr, di * di);
}

// Type code: p_n -> k (1..63); s_{l,n} -> k for Mis(l,k), 32 + k for Hyp(k);
// 255 if nothing matched.
__device__ __forceinline__ int type_of(const PolyDev& P, double cr, double ci, double tau) {
  const int n = P.n;
  const int len = (P.kind == 0) ? n : P.l + n;
  const int g = (P.kind == 0) ? n : [&] {
    int a = n, b = P.l - 1;
    while (b) { int t = a % b; a = b; b = t; }
    return a;
  }();
  double zr = 0.0, zi = 0.0, dzr = 0.0, dzi = 0.0;
  double lr = 0.0, li = 0.0, ldr = 0.0, ldi = 0.0;  // p_l, p'_l
  int hyp = 0, mis = 0;
  for (int k = 1; k <= len; ++k) {
    const double tzr = zr + zr, tzi = zi + zi;
    const double ndr = fma(tzr, dzr, fma(-tzi, dzi, 1.0));
    const double ndi = fma(tzr, dzi, tzi * dzr);
    const double nzr = fma(zr, zr, fma(-zi, zi, cr));
    const double nzi = fma(tzr, zi, ci);
    zr = nzr; zi = nzi; dzr = ndr; dzi = ndi;
    if (!hyp && k <= g && (g % k) == 0 && newton_small(zr, zi, dzr, dzi, tau)) hyp = k;
    if (P.kind == 1) {
      if (k == P.l) { lr = zr; li = zi; ldr = dzr; ldi = dzi; }
      const int kk = k - P.l;
      if (!mis && kk >= 1 && (n % kk) == 0 &&
          newton_small(zr - lr, zi - li, dzr - ldr, dzi - ldi, tau))
        mis = kk;
    }
  }
  if (P.kind == 0) return hyp ? hyp : 255;
  if (hyp) return (32 + hyp < 64) ? 32 + hyp : 255;
  if (mis) return mis < 32 ? mis : 255;
  return 255;
}

__global__ void k_classify(PolyDev P, double2* __restrict__ reps,
                           const unsigned long long* __restrict__ n_reps, int64_t cap, double tau,
                           int polish, uint8_t* __restrict__ type, uint32_t* __restrict__ mult,
                           DevCounters* ctr) {
  __shared__ unsigned int hist[64];
  for (int q = threadIdx.x; q < 64; q += blockDim.x) hist[q] = 0;
  __syncthreads();
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nr = (int64_t)*n_reps;
  unsigned long long nreal = 0;
  if (u < cap) {
    if (u < nr) {
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
      const int t = type_of(P, z.x, z.y, tau);
      const unsigned m = (z.y == 0.0) ? 1u : 2u;
      type[u] = (uint8_t)t;
      mult[u] = m;
      nreal += (m == 1);
      if (t < 64) atomicAdd(&hist[t], m);
    } else {
      mult[u] = 0;
    }
  }
  warp_add_u64(&ctr->n_reps_real, nreal);
  __syncthreads();
  for (int q = threadIdx.x; q < 64; q += blockDim.x)
    if (hist[q]) atomicAdd(&ctr->type_count[q], (unsigned long long)hist[q]);
}

cudaError_t launch_classify(const PolyDev& P, double2* reps, const unsigned long long* n_reps,
                            int64_t cap, double tau, int polish, uint8_t* type, uint32_t* mult,
                            DevCounters* ctr, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_classify<<<(unsigned)((cap + 127) / 128), 128, 0, s>>>(P, reps, n_reps, cap, tau, polish, type,
                                                           mult, ctr);
  return cudaGetLastError();
}

__global__ void k_type_only(PolyDev P, const double2* __restrict__ roots, int64_t count, double tau,
                            uint8_t* __restrict__ type) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double2 z = roots[i];
  type[i] = (uint8_t)type_of(P, z.x, z.y, tau);
}

cudaError_t launch_type_only(const PolyDev& P, const double2* roots, int64_t count, double tau,
                             uint8_t* type, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_type_only<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(P, roots, count, tau, type);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a7: disk arithmetic in binary64 (Thm diskArithmetic).
struct Disk {
  double x, y;  // centre, exact binary64 values
  double r;     // radius, an upper bound
};

// the paper's ulp(x) = 2^(e(x) - 53) for normal x, 2^-1074 for subnormals and 0
__device__ __forceinline__ double ulp64(double x) {
  const double a = fabs(x);
  if (!(a >= 2.2250738585072014e-308)) return 4.9406564584124654e-324;
  const double p2 = __longlong_as_double(__double_as_longlong(a) & 0x7ff0000000000000ll);
  return p2 * 2.220446049250313e-16;  // exact: product of powers of two above 2^-1074
}

__device__ __forceinline__ double abs_ru(double x, double y) {
  return __dsqrt_ru(__fma_ru(x, x, __dmul_ru(y, y)));
}
__device__ __forceinline__ double abs_rd(double x, double y) {
  return __dsqrt_rd(__fma_rd(x, x, __dmul_rd(y, y)));
}

// D(a) + D(b)
__device__ __forceinline__ Disk d_add(const Disk& a, const Disk& b) {
  Disk o;
  o.x = a.x + b.x;
  o.y = a.y + b.y;
  const double half_ulp = __dmul_ru(0.5, __dadd_ru(ulp64(o.x), ulp64(o.y)));
  o.r = __dadd_ru(__dadd_ru(a.r, b.r), half_ulp);
  return o;
}

// D(a) + exact point (cx, cy)
__device__ __forceinline__ Disk d_add_pt(const Disk& a, double cx, double cy) {
  Disk o;
  o.x = a.x + cx;
  o.y = a.y + cy;
  o.r = __dadd_ru(a.r, __dmul_ru(0.5, __dadd_ru(ulp64(o.x), ulp64(o.y))));
  return o;
}

// D(a) x D(b): centre by two FMAs, R* = 1/2 (ulp Re + ulp Im) + 1/2 sum of the
// ulps of the four real products, radius ra rb + ra |b| + rb |a| + R*.
__device__ __forceinline__ Disk d_mul(const Disk& a, const Disk& b) {
  const double yy = a.y * b.y, yx = a.y * b.x, xx = a.x * b.x, xy = a.x * b.y;
  Disk o;
  o.x = fma(a.x, b.x, -yy);
  o.y = fma(a.x, b.y, yx);
  double rs = __dadd_ru(__dadd_ru(ulp64(o.x), ulp64(o.y)),
                        __dadd_ru(__dadd_ru(ulp64(xx), ulp64(yy)), __dadd_ru(ulp64(xy), ulp64(yx))));
  rs = __dmul_ru(0.5, rs);  // exact unless subnormal; rounded up then
  const double ma = abs_ru(a.x, a.y), mb = abs_ru(b.x, b.y);
  double r = __fma_ru(a.r, b.r, rs);
  r = __fma_ru(a.r, mb, r);
  r = __fma_ru(b.r, ma, r);
  o.r = r;
  return o;
}

// D(a)^2
__device__ __forceinline__ Disk d_sqr(const Disk& a) { return d_mul(a, a); }

// Disk orbit of P over D(c, rc): value disk V and derivative disk W.
__device__ __forceinline__ void disk_orbit(const PolyDev& P, double cx, double cy, double rc,
                                           Disk& V, Disk& W) {
  Disk C;
  C.x = cx;
  C.y = cy;
  C.r = rc;
  Disk z = {0.0, 0.0, 0.0}, dz = {0.0, 0.0, 0.0};
  Disk zc = {0.0, 0.0, 0.0}, dzc = {0.0, 0.0, 0.0};
  for (int k = 1; k <= P.m; ++k) {
    Disk t = d_mul(z, dz);  // z_{k-1} z'_{k-1}
    t.x *= 2.0;             // exact scaling by 2
    t.y *= 2.0;
    t.r = __dmul_ru(t.r, 2.0);
    dz = d_add_pt(t, 1.0, 0.0);  // z'_k = 2 z_{k-1} z'_{k-1} + 1
    z = d_add(d_sqr(z), C);      // z_k = z_{k-1}^2 + C
    if (k == P.lcap) { zc = z; dzc = dz; }
  }
  if (P.lcap >= 0) {
    z = d_add(z, zc);
    dz = d_add(dz, dzc);
  }
  V = z;
  W = dz;
}

// Certify the points of 'pts' (sorted by Re through 'order', or already
// sorted when order == nullptr).  upper: the list holds one representative
// per conjugate pair, so conjugates count as neighbours too.
__global__ void k_certify(PolyDev P, const double2* __restrict__ pts,
                          const uint32_t* __restrict__ order, const unsigned long long* n_pts_dev,
                          int64_t n_pts_host, double tol, int upper, const uint32_t* __restrict__ mult,
                          uint8_t* __restrict__ pass, double* __restrict__ radius,
                          DevCounters* ctr) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = n_pts_dev ? (int64_t)*n_pts_dev : n_pts_host;
  unsigned long long npass = 0, overflow = 0;
  double rad = 0.0;
  bool ok = false, valid = p < n;
  if (valid) {
    const int64_t ip = order ? (int64_t)order[p] : p;
    const double2 c = pts[ip];
    // nearest neighbour (and conjugates) within the window W = tol / 0.45
    const double W = tol / 0.45;
    double nn2 = W * W;
    if (upper && c.y != 0.0) nn2 = fmin(nn2, 4.0 * c.y * c.y);
    int scanned = 0;
    for (int dir = -1; dir <= 1; dir += 2) {
      for (int64_t q = p + dir; q >= 0 && q < n; q += dir) {
        const double2 v = pts[order ? (int64_t)order[q] : q];
        const double dx = v.x - c.x;
        if (fabs(dx) >= W) break;
        const double dy = v.y - c.y;
        nn2 = fmin(nn2, fma(dx, dx, dy * dy));
        if (upper) {
          const double ey = v.y + c.y;
          nn2 = fmin(nn2, fma(dx, dx, ey * ey));
        }
        if (++scanned >= 4096) { overflow = 1; break; }
      }
    }
    rad = fmin(tol, 0.45 * sqrt(nn2));
    // |P(c)| bound: point disk orbit (radius = accumulated rounding)
    Disk V0, W0, V, Wd;
    disk_orbit(P, c.x, c.y, 0.0, V0, W0);
    const double fz = __dadd_ru(abs_ru(V0.x, V0.y), V0.r);
    // P'(D(c, rad)) inside B' = Wd
    disk_orbit(P, c.x, c.y, rad, V, Wd);
    const double dist = __dsub_rd(abs_rd(Wd.x, Wd.y), Wd.r);
    ok = isfinite(fz) && isfinite(dist) && dist > 0.0 && rad > 0.0 && __dmul_rd(rad, dist) > fz;
    pass[ip] = ok ? 1 : 0;
    if (radius) radius[ip] = rad;
    npass = ok ? (mult ? mult[p] : 1u) : 0u;
  }
  warp_add_u64(&ctr->n_cert_pass, npass);
  if (overflow) atomicAdd(&ctr->cluster_overflow, 1ull);
  if (valid && ok) {
    atomicMin(&ctr->min_radius_bits, (unsigned long long)__double_as_longlong(rad));
    atomicMax(&ctr->max_radius_bits, (unsigned long long)__double_as_longlong(rad));
  }
}

cudaError_t launch_certify(const PolyDev& P, const double2* reps, const unsigned long long* n_reps,
                           int64_t cap, double tol, const uint32_t* mult, uint8_t* pass,
                           double* radius, DevCounters* ctr, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_certify<<<(unsigned)((cap + 127) / 128), 128, 0, s>>>(P, reps, nullptr, n_reps, cap, tol, 1,
                                                          mult, pass, radius, ctr);
  return cudaGetLastError();
}

// standalone certificate of an arbitrary list (sorted through 'order')
cudaError_t launch_certify_list(const PolyDev& P, const double2* pts, const uint32_t* order,
                                int64_t count, double tol, uint8_t* pass, double* radius,
                                DevCounters* ctr, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_certify<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(P, pts, order, nullptr, count, tol, 0,
                                                            nullptr, pass, radius, ctr);
  return cudaGetLastError();
}

}  // namespace mt
