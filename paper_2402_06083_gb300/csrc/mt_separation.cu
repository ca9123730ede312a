// mt_separation.cu -- separation statistics of a root list (Sec. 6.3.2:
// the minimal distance among Hyp(n) follows 118.4 / 4^n, attained by the two
// left-most real roots; Fig. separationHistogram bins it over the geometric
// bands I_k = (-2 + 4^-(k+1), -2 + 4^-k] x R).
//
// For every root of the list (optionally only those with mask[i] != 0) the
// exact distance to its nearest other root of the same (masked) list, in
// three tiers:
//   1. Re window.  The list is sorted by Re; a thread scans away from its
//      root in both directions and stops once the real parts alone are
//      farther apart than the best distance so far.  This settles the roots
//      whose neighbours are near in Re (the antenna near -2, where real
//      roots differ only in Re).  With low parts the scan compares in
//      double-double and stops only when the hi parts are farther apart
//      than the best distance plus two ulps.  A root whose scan passes
//      SEP_WINDOW_CAP entries goes on with its best so far as a bound.
//   2. Strips, one thread per root.  The list is re-sorted by (Re strip,
//      Im), with about 16 roots per strip on average (2^10 .. 2^20 strips
//      over [-2.25, 2.25]); a table gives each strip's range.  The thread
//      visits the strips outward from its own and, in each, walks up and
//      down from its own Im while the keys stay inside [y - best, y + best];
//      the walk ends at the first strip farther than best.
//   3. Strips, one block per root, for roots whose tier-2 walk passed its
//      caps (isolated roots, far from everything): each thread of the block
//      binary-searches one strip, the block scans the hits together.
// Every comparison is the exact pair distance: the tiers only decide which
// pairs are looked at.
// Per-band minima are kept as the bit patterns of non-negative doubles,
// which order like the values (atomicMin on unsigned 64-bit).
#include "mt_common.cuh"

namespace mt {

namespace {

__device__ __forceinline__ double ulp_of(double x) {
  const double a = fabs(x);
  if (!(a >= 2.2250738585072014e-308)) return 4.9406564584124654e-324;
  return __longlong_as_double(__double_as_longlong(a) & 0x7ff0000000000000ll) * 2.220446049250313e-16;
}

// two-sum difference a - b of (hi, lo) pairs, rounded to binary64 at the end
__device__ __forceinline__ double dd_diff(double ah, double al, double bh, double bl) {
  const double s = ah - bh;
  const double bb = s - ah;
  const double e = (ah - (s - bb)) + (-bh - bb);
  return s + (e + (al - bl));
}

constexpr int SEP_WINDOW_CAP = 64;      // tier 1: entries of the Re window a thread scans
constexpr int SEP_THREAD_STRIPS = 64;   // tier 2: strips and points a thread walks
constexpr int SEP_THREAD_POINTS = 4096;
constexpr int SEP_STRIP_SHIFT = 44;     // strip index above bit 44 of a key (at most 2^20 strips)
constexpr double SEP_X0 = -2.25;        // strips cover [-2.25, 2.25]
constexpr double SEP_WIDTH = 4.5;
constexpr int SEP_BS = 256;

__device__ __forceinline__ double pos_inf() { return __longlong_as_double(0x7ff0000000000000ll); }

// Coordinate differences of roots a and b (double-double when lo is given).
__device__ __forceinline__ void pair_diff(const double2* hi, const double2* lo, int64_t a, int64_t b,
                                          double& dx, double& dy) {
  const double2 u = hi[a], v = hi[b];
  if (lo) {
    const double2 ul = lo[a], vl = lo[b];
    dx = dd_diff(v.x, vl.x, u.x, ul.x);
    dy = dd_diff(v.y, vl.y, u.y, ul.y);
  } else {
    dx = v.x - u.x;
    dy = v.y - u.y;
  }
}

// The binary64 pipe is the scarce one on this part: a pair is first tested
// on its squared distance (two FMA-class operations), and hypot -- the
// reported value -- is taken only for pairs within thr of the best so far.
// thr = best^2 (1 + 1e-15) covers the rounding of both squares; below
// 1e-140 the squares lose digits to underflow and every pair takes hypot.
__device__ __forceinline__ double sq_threshold(double best) {
  return best < 1e-140 ? pos_inf() : best * best * (1.0 + 1e-15);
}
__device__ __forceinline__ bool consider(double dx, double dy, double& best, double& thr) {
  if (!(fma(dx, dx, dy * dy) <= thr)) return false;
  const double h = hypot(dx, dy);
  if (!(h < best)) return false;
  best = h;
  thr = sq_threshold(best);
  return true;
}

// band of a root: the k >= 0 with Re c + 2 in (4^-(k+1), 4^-k]; roots with
// Re c + 2 > 1 fall in band 0, Re c + 2 <= 4^-64 in band 63
__device__ __forceinline__ int sep_band(double x) {
  const double t = x + 2.0;
  if (!(t > 0.0)) return 63;
  int k = 0;
  double up = 1.0;
  while (k < 63 && t <= 0.25 * up) {
    up *= 0.25;
    ++k;
  }
  return k;
}

__device__ __forceinline__ void record(double best, double x, unsigned long long* band_min) {
  if (best < pos_inf()) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(best);
    atomicMin(&band_min[sep_band(x)], bits);
    atomicMin(&band_min[64], bits);  // the whole list
  }
}

// The same for a whole warp (all 32 lanes call; has = the lane has a value):
// one atomic for the list minimum, and one for the band minimum when the
// warp's values share a band (roots sorted by Re mostly do), else per lane.
__device__ __forceinline__ void record_warp(bool has, double best, double x, unsigned long long* band_min) {
  has = has && best < pos_inf();
  const unsigned long long bits = has ? (unsigned long long)__double_as_longlong(best) : ~0ull;
  const int band = has ? sep_band(x) : -1;
  warp_min_u64(&band_min[64], bits);
  const int lead = __ffs(__ballot_sync(0xffffffffu, has)) - 1;
  if (lead < 0) return;
  const int band0 = __shfl_sync(0xffffffffu, band, lead);
  if (__all_sync(0xffffffffu, !has || band == band0)) {
    unsigned long long v = bits;
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&band_min[band0], v);
  } else if (has) {
    atomicMin(&band_min[band], bits);
  }
}

// Strip of a real part: monotone non-decreasing in x (a subtraction and a
// multiplication by a positive constant, both correctly rounded, then a
// clamp), which is all the strip walk relies on.  Points outside [-2.25,
// 2.25] land in the end strips.
__device__ __forceinline__ int strip_of(double x, int S, double scale) {
  const double t = (x - SEP_X0) * scale;
  if (!(t >= 0.0)) return 0;
  if (t >= (double)S) return S - 1;
  return (int)t;
}

// (strip, Im) order: the strip above bit 44, then the order-preserving image
// of Im truncated to 44 bits (truncation keeps <=, so y <= Y implies
// key(y) <= key(Y), and a key above key(Y) means y > Y)
__device__ __forceinline__ uint64_t strip_key(int s, double y) {
  return ((uint64_t)s << SEP_STRIP_SHIFT) | (f64_key(y) >> (64 - SEP_STRIP_SHIFT));
}

// first index in [lo, hi) with a[i] >= v (resp. a[i] > v)
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t lo, int64_t hi,
                                                   uint64_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t* __restrict__ a, int64_t lo, int64_t hi,
                                                   uint64_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// hi parts can differ from the values compared by half an ulp each, and the
// window ends are rounded: windows are widened by a few ulps of the magnitudes
__device__ __forceinline__ double window_margin(double2 c, double best) {
  return 4.0 * ulp_of(fabs(c.x) + fabs(c.y) + best) + 1e-300;
}

// strip order 0, -1, +1, -2, +2, ... around the root's own strip
__device__ __forceinline__ int64_t strip_offset(int64_t j) { return (j & 1) ? -((j + 1) / 2) : j / 2; }

}  // namespace

__global__ void k_separation_init(unsigned long long* band_min) {
  const int i = threadIdx.x;
  if (i < 65) band_min[i] = 0x7ff0000000000000ull;  // +inf
  if (i == 65 || i == 66) band_min[i] = 0ull;        // roots left by tier 1, by tier 2
}

// pass 1: Re-window scan, one thread per root
__global__ void k_separation(const double2* __restrict__ hi, const double2* __restrict__ lo,
                             const uint32_t* __restrict__ order, int64_t n,
                             const uint8_t* __restrict__ mask, double* __restrict__ nn_out,
                             unsigned long long* __restrict__ band_min,
                             unsigned long long* __restrict__ nisolated,
                             uint32_t* __restrict__ iso_idx, double* __restrict__ iso_best) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool has = false;
  double best = pos_inf(), cx = 0.0;
  if (p < n) {
  const int64_t ip = order[p];
  if (mask && !mask[ip]) {
    if (nn_out) nn_out[ip] = 0.0;
  } else {
  const double2 c = hi[ip];
  cx = c.x;
  double thr = pos_inf();
  int scanned = 0;
  bool cut = false;
  for (int dir = -1; dir <= 1 && !cut; dir += 2) {
    for (int64_t q = p + dir; q >= 0 && q < n; q += dir) {
      const int64_t iq = order[q];
      const double2 v = hi[iq];
      const double gap = fabs(v.x - c.x);
      if (gap > best + (lo ? 2.0 * ulp_of(fmax(fabs(v.x), fabs(c.x))) : 0.0)) break;
      if (++scanned > SEP_WINDOW_CAP) {
        cut = true;
        break;
      }
      if (mask && !mask[iq]) continue;
      double dx, dy;
      pair_diff(hi, lo, ip, iq, dx, dy);
      consider(dx, dy, best, thr);
    }
  }
  if (cut) {  // left to the strip pass, with best as an upper bound
    const unsigned long long k = atomicAdd(nisolated, 1ull);
    iso_idx[k] = (uint32_t)ip;  // k < n: each root is added at most once
    iso_best[k] = best;
  } else {
    if (nn_out) nn_out[ip] = best;
    has = true;
  }
  }
  }
  record_warp(has, best, cx, band_min);
}

__global__ void k_strip_keys(const double2* __restrict__ hi, int64_t n, int S, double scale,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 c = hi[i];
  keys[i] = strip_key(strip_of(c.x, S, scale), c.y);
  vals[i] = (uint32_t)i;
}

// offs[s] = first sorted entry of strip s, offs[S] = n
__global__ void k_strip_offsets(const uint64_t* __restrict__ skeys, int64_t n, int S,
                                uint32_t* __restrict__ offs) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > S) return;
  offs[s] = (uint32_t)(s == S ? n : lower_bound_u64(skeys, 0, n, (uint64_t)s << SEP_STRIP_SHIFT));
}

// tier 2: one thread per root left by tier 1.  In each strip the walk starts
// at the root's own Im and moves up and down while the keys stay inside the
// window [y - best, y + best] (the window shrinking with best).  A root
// that needs more than SEP_THREAD_STRIPS strips or SEP_THREAD_POINTS
// points goes on to tier 3 with its best so far.
__global__ void k_separation_strip_thread(const double2* __restrict__ hi, const double2* __restrict__ lo,
                                          const uint8_t* __restrict__ mask, const uint64_t* __restrict__ skeys,
                                          const uint32_t* __restrict__ sidx, const uint32_t* __restrict__ offs,
                                          int S, double scale, const uint32_t* __restrict__ iso_idx,
                                          const double* __restrict__ iso_best,
                                          const unsigned long long* __restrict__ niso,
                                          double* __restrict__ nn_out, unsigned long long* __restrict__ band_min,
                                          uint32_t* __restrict__ iso2_idx, double* __restrict__ iso2_best,
                                          unsigned long long* __restrict__ niso2) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool has = false;
  double best = pos_inf(), cx = 0.0;
  if (r < (int64_t)*niso) {
  const int64_t ip = iso_idx[r];
  const double2 c = hi[ip];
  cx = c.x;
  best = iso_best[r];
  double thr = sq_threshold(best);
  const int sq = strip_of(c.x, S, scale);
  int strips = 0, points = 0;
  bool defer = false;
  for (int64_t j = 0; !defer; ++j) {
    double m = window_margin(c, best);
    const int slo = strip_of(c.x - best - m, S, scale), shi = strip_of(c.x + best + m, S, scale);
    if ((j + 1) / 2 > max(sq - slo, shi - sq)) break;  // every strip left lies beyond best
    const int64_t s = sq + strip_offset(j);
    if (s < slo || s > shi) continue;
    if (++strips > SEP_THREAD_STRIPS) {
      defer = true;
      break;
    }
    const int64_t b0 = offs[s], b1 = offs[s + 1];
    if (b0 == b1) continue;
    const int64_t p0 = lower_bound_u64(skeys, b0, b1, strip_key((int)s, c.y));
    uint64_t kup = strip_key((int)s, c.y + best + m), kdn = strip_key((int)s, c.y - best - m);
    for (int dir = 1; dir >= -1 && !defer; dir -= 2) {
      for (int64_t pos = dir > 0 ? p0 : p0 - 1; pos >= b0 && pos < b1; pos += dir) {
        const uint64_t k = skeys[pos];
        if (dir > 0 ? k > kup : k < kdn) break;
        if (++points > SEP_THREAD_POINTS) {
          defer = true;
          break;
        }
        const int64_t q = sidx[pos];
        if (q == ip || (mask && !mask[q])) continue;
        double dx, dy;
        pair_diff(hi, lo, ip, q, dx, dy);
        if (consider(dx, dy, best, thr)) {
          m = window_margin(c, best);
          kup = strip_key((int)s, c.y + best + m);
          kdn = strip_key((int)s, c.y - best - m);
        }
      }
    }
  }
  if (defer) {
    const unsigned long long k = atomicAdd(niso2, 1ull);  // k < *niso
    iso2_idx[k] = (uint32_t)ip;
    iso2_best[k] = best;
  } else {
    if (nn_out) nn_out[ip] = best;
    has = true;
  }
  }
  record_warp(has, best, cx, band_min);
}

// tier 3: one block per root left by tier 2 walks the strips outward from
// its own, a chunk of SEP_BS strips at a time: each thread binary-searches
// one strip for the Im window, then the block scans the hits together
__global__ void __launch_bounds__(SEP_BS)
k_separation_strip_block(const double2* __restrict__ hi, const double2* __restrict__ lo,
                         const uint8_t* __restrict__ mask, const uint64_t* __restrict__ skeys,
                         const uint32_t* __restrict__ sidx, const uint32_t* __restrict__ offs, int S,
                         double scale, const uint32_t* __restrict__ iso_idx, const double* __restrict__ iso_best,
                         const unsigned long long* __restrict__ niso, double* __restrict__ nn_out,
                         unsigned long long* __restrict__ band_min) {
  __shared__ int64_t beg[SEP_BS];
  __shared__ int64_t incl[SEP_BS];  // inclusive prefix sums of the hit counts
  __shared__ double red[SEP_BS];
  const int t = threadIdx.x;
  const int64_t nr = (int64_t)*niso;
  for (int64_t r = blockIdx.x; r < nr; r += gridDim.x) {
    const int64_t ip = iso_idx[r];
    const double2 c = hi[ip];
    double best = iso_best[r];  // the same value in every thread throughout
    const int sq = strip_of(c.x, S, scale);
    for (int64_t base = 0;; base += SEP_BS) {
      const double m = window_margin(c, best);
      const int slo = strip_of(c.x - best - m, S, scale), shi = strip_of(c.x + best + m, S, scale);
      if ((base + 1) / 2 > max(sq - slo, shi - sq)) break;  // every strip of this chunk lies beyond best
      const int64_t s = sq + strip_offset(base + t);
      int64_t b = 0, k = 0;
      if (s >= slo && s <= shi) {
        const int64_t b0 = offs[s], b1 = offs[s + 1];
        b = lower_bound_u64(skeys, b0, b1, strip_key((int)s, c.y - best - m));
        k = upper_bound_u64(skeys, b, b1, strip_key((int)s, c.y + best + m)) - b;
      }
      beg[t] = b;
      incl[t] = k;
      __syncthreads();
      for (int off = 1; off < SEP_BS; off <<= 1) {
        const int64_t v = (t >= off) ? incl[t - off] : 0;
        __syncthreads();
        incl[t] += v;
        __syncthreads();
      }
      const int64_t total = incl[SEP_BS - 1];
      double mine = best, thr = sq_threshold(best);
      for (int64_t g = t; g < total; g += SEP_BS) {
        int u0 = 0, u1 = SEP_BS - 1;  // first slot with incl > g
        while (u0 < u1) {
          const int mid = (u0 + u1) >> 1;
          if (incl[mid] > g) u1 = mid; else u0 = mid + 1;
        }
        const int64_t pos = beg[u0] + g - (u0 ? incl[u0 - 1] : 0);
        const int64_t q = sidx[pos];
        if (q == ip || (mask && !mask[q])) continue;
        double dx, dy;
        pair_diff(hi, lo, ip, q, dx, dy);
        consider(dx, dy, mine, thr);
      }
      red[t] = mine;
      __syncthreads();
      for (int w = SEP_BS / 2; w > 0; w >>= 1) {
        if (t < w) red[t] = fmin(red[t], red[t + w]);
        __syncthreads();
      }
      best = fmin(best, red[0]);
      __syncthreads();  // red and incl are rewritten by the next chunk
    }
    if (t == 0) {
      if (nn_out) nn_out[ip] = best;
      record(best, c.x, band_min);
    }
    __syncthreads();
  }
}

cudaError_t launch_separation(const double2* hi, const double2* lo, const uint32_t* order, int64_t n,
                              const uint8_t* mask, double* nn_out, unsigned long long* band_min,
                              uint32_t* iso_idx, double* iso_best, cudaStream_t s) {
  MT_COUNT_LAUNCH(1);
  k_separation_init<<<1, 96, 0, s>>>(band_min);
  if (n > 0) {
    MT_COUNT_LAUNCH(1);
    k_separation<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(hi, lo, order, n, mask, nn_out, band_min,
                                                             band_min + 65, iso_idx, iso_best);
  }
  return cudaGetLastError();
}

int separation_strips_log2(int64_t n) {
  int k = 10;  // about 16 roots per strip, 2^10 .. 2^20 strips
  while (k < 20 && ((int64_t)1 << (k + 4)) < n) ++k;
  return k;
}

cudaError_t launch_strip_index(const double2* hi, int64_t n, int log2s, uint64_t* keys, uint32_t* vals,
                               uint64_t* keys_alt, uint32_t* vals_alt, void* rtmp, uint32_t* offs,
                               cudaStream_t s) {
  const int S = 1 << log2s;
  if (n > 0) {
    MT_COUNT_LAUNCH(1);
    k_strip_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(hi, n, S, S / SEP_WIDTH, keys, vals);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, rtmp, s);
    if (e != cudaSuccess) return e;
  }
  MT_COUNT_LAUNCH(1);
  k_strip_offsets<<<(unsigned)((S + 1 + 255) / 256), 256, 0, s>>>(keys, n, S, offs);
  return cudaGetLastError();
}

cudaError_t launch_separation_strips(const double2* hi, const double2* lo, const uint8_t* mask,
                                     const uint64_t* skeys, const uint32_t* sidx, const uint32_t* offs,
                                     int log2s, const uint32_t* iso_idx, const double* iso_best, int64_t niso,
                                     uint32_t* iso2_idx, double* iso2_best, double* nn_out,
                                     unsigned long long* band_min, cudaStream_t s) {
  if (niso <= 0) return cudaSuccess;
  const int S = 1 << log2s;
  const double scale = S / SEP_WIDTH;
  MT_COUNT_LAUNCH(1);
  k_separation_strip_thread<<<(unsigned)((niso + 127) / 128), 128, 0, s>>>(
      hi, lo, mask, skeys, sidx, offs, S, scale, iso_idx, iso_best, band_min + 65, nn_out, band_min, iso2_idx,
      iso2_best, band_min + 66);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // tier 3 reads its count from the device: a grid-stride loop over it
  const int64_t blocks = std::min<int64_t>(niso, 152 * 8);
  MT_COUNT_LAUNCH(1);
  k_separation_strip_block<<<(unsigned)blocks, SEP_BS, 0, s>>>(hi, lo, mask, skeys, sidx, offs, S, scale,
                                                               iso2_idx, iso2_best, band_min + 66, nn_out,
                                                               band_min);
  return cudaGetLastError();
}

}  // namespace mt
