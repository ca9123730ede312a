// mt_batch.cu -- many polynomials in one pass: every s_{l,n} with
// l >= 2, n >= 1, l + n <= max_order (eq. polySimple), as the paper's
// misSimpleQuick does one type at a time (Sec. 6.3.1).
//
// GB300 design.  The degrees of the polynomials differ by orders of
// magnitude (2 .. 2^14 for l + n <= 16), so one launch per polynomial would
// leave the GPU mostly idle.  Instead the work of all polynomials is laid
// end to end: seeds of all level lines in one launch, all level-line chunks
// drained by one persistent launch through an atomic chunk queue, all
// Newton descents drained by one persistent launch with per-lane refill
// (k_descend's scheme, each lane looking up the polynomial of the start it
// pops), then one sort by (polynomial, Re) and the segmented root-set,
// type and certificate kernels (SegView).
#include "mt_levelline.cuh"

namespace mt {

// largest p with off[p] <= x (off ascending, off[0] = 0)
__device__ __forceinline__ int find_seg(const int64_t* __restrict__ off, int np, int64_t x) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_seed_lift_batch(const BatchEntry* __restrict__ E, const int64_t* __restrict__ seed_off,
                                  int np, int64_t total, double lambda0, int shrink, double2* seeds,
                                  DevCounters* ctr) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0;
  if (g < total) {
    const int p = find_seg(seed_off, np, g);
    const BatchEntry e = E[p];
    seeds[g] = lift_seed(e.P, lambda0, e.N0, e.log2N0, shrink, g - seed_off[p], steps);
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->seed_newton, steps);
}

// persistent: lanes pop level-line chunks of any polynomial from one queue
__global__ void k_walk_batch(const BatchEntry* __restrict__ E, const int64_t* __restrict__ chunk_off,
                             int np, int64_t total, double lambda0, int M, int every,
                             const double2* __restrict__ seeds, double2* __restrict__ starts,
                             DevCounters* ctr) {
  __shared__ double2 ph[64];
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double c, s;
    unit_phase((uint64_t)q, (uint64_t)M, c, s);
    ph[q] = make_double2(lambda0 * c, lambda0 * s);
  }
  __syncthreads();
  unsigned long long steps = 0, fails = 0;
  for (;;) {
    const int64_t c = (int64_t)atomicAdd(&ctr->queue_head2, 1ull);
    if (c >= total) break;
    const int p = find_seg(chunk_off, np, c);
    const BatchEntry e = E[p];
    fails += walk_chunk(e.P, ph, M, every, e.L, e.nchunks, c - chunk_off[p], seeds + e.seed_off,
                        starts + e.start_off, steps) ? 1 : 0;
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

// persistent Newton descents over the starts of all polynomials (k_descend
// with the polynomial looked up per start)
__global__ void __launch_bounds__(128) k_descend_batch(const BatchEntry* __restrict__ E,
                                                       const int64_t* __restrict__ start_off,
                                                       int np, int64_t count, double tol2,
                                                       const double2* __restrict__ starts,
                                                       double2* __restrict__ cand,
                                                       uint8_t* __restrict__ status,
                                                       uint16_t* __restrict__ seg,
                                                       DevCounters* ctr) {
  const unsigned lane = threadIdx.x & 31;
  int64_t idx = -1;
  double zr = 0.0, zi = 0.0, rdiv2 = 16.0, prev2 = 1e300;
  int it = 0, m = 1, lcap = -1, cap = 20;
  unsigned long long steps = 0, orbit = 0, nconv = 0, ndiv = 0, nto = 0;
  for (;;) {
    const unsigned need = __ballot_sync(0xffffffffu, idx < 0);
    if (need) {
      unsigned long long base = 0;
      if (lane == (unsigned)(__ffs(need) - 1))
        base = atomicAdd(&ctr->queue_head, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, __ffs(need) - 1);
      if (idx < 0) {
        idx = (int64_t)(base + __popc(need & lanemask_lt()));
        if (idx < count) {
          const int p = find_seg(start_off, np, idx);
          const BatchEntry e = E[p];
          m = e.P.m;
          lcap = e.P.lcap;
          cap = e.cap;
          seg[idx] = (uint16_t)p;
          const double2 z0 = starts[idx];
          zr = z0.x;
          zi = z0.y;
          it = 0;
          prev2 = 1e300;
          rdiv2 = fmax(16.0, 4.0 * fma(zr, zr, zi * zi));
        }
      }
    }
    const bool active = idx >= 0 && idx < count;
    if (!__any_sync(0xffffffffu, active)) break;
    if (active) {
      double vr, vi, dr, di;
      orbit_f64(m, lcap, 1.0, zr, zi, vr, vi, dr, di);
      double qr, qi;
      cdiv_f64(vr, vi, dr, di, qr, qi);
      zr -= qr;
      zi -= qi;
      ++it;
      ++steps;
      orbit += (unsigned)m;
      const double s2 = fma(qr, qr, qi * qi);
      int outcome = -1;
      if (!finite2(zr, zi) || fma(zr, zr, zi * zi) > rdiv2) outcome = 1;
      else if (s2 < tol2) outcome = 0;
      else if (s2 >= 0.25 * prev2 && s2 < floor2_f64(zr, zi)) outcome = 0;
      else if (it >= cap) outcome = 2;
      prev2 = s2;
      if (outcome >= 0) {
        cand[idx] = make_double2(zr, zi);
        status[idx] = (uint8_t)outcome;
        nconv += outcome == 0;
        ndiv += outcome == 1;
        nto += outcome == 2;
        idx = -1;
      }
    }
  }
  warp_add_u64(&ctr->desc_newton, steps);
  warp_add_u64(&ctr->desc_orbit, orbit);
  warp_add_u64(&ctr->n_conv, nconv);
  warp_add_u64(&ctr->n_diverge, ndiv);
  warp_add_u64(&ctr->n_timeout, nto);
}

// (pair id, value) keys for the stable pass that groups candidates by polynomial
__global__ void k_seg_keys(const uint32_t* __restrict__ vals, const uint16_t* __restrict__ seg,
                           const uint8_t* __restrict__ status, int64_t count,
                           uint64_t* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint32_t v = vals[i];
  // not-converged candidates sort after every polynomial's roots
  keys[i] = status[v] == 0 ? (uint64_t)seg[v] : 0xffffull;
}

cudaError_t launch_seed_lift_batch(const BatchEntry* E, const int64_t* seed_off, int np,
                                   int64_t total, double lambda0, int shrink, double2* seeds,
                                   DevCounters* ctr, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int bs = 128;
  MT_COUNT_LAUNCH(1);
  k_seed_lift_batch<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(E, seed_off, np, total, lambda0,
                                                                     shrink, seeds, ctr);
  return cudaGetLastError();
}

cudaError_t launch_walk_batch(const BatchEntry* E, const int64_t* chunk_off, int np, int64_t total,
                              double lambda0, int M, int every, const double2* seeds,
                              double2* starts, DevCounters* ctr, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int bs = 64;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_batch, bs, 0);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (total + bs - 1) / bs;
  if (grid > need) grid = need;
  MT_COUNT_LAUNCH(1);
  k_walk_batch<<<(unsigned)grid, bs, 0, s>>>(E, chunk_off, np, total, lambda0, M, every, seeds, starts,
                                             ctr);
  return cudaGetLastError();
}

cudaError_t launch_descend_batch(const BatchEntry* E, const int64_t* start_off, int np,
                                 int64_t count, double tol, const double2* starts, double2* cand,
                                 uint8_t* status, uint16_t* seg, DevCounters* ctr, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int bs = 128;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend_batch, bs, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > 2) per_sm = 2;  // 8 warps/SM saturate the binary64 pipe (as launch_descend)
  int64_t grid = (int64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (count + bs - 1) / bs;
  if (grid > need) grid = need;
  MT_COUNT_LAUNCH(1);
  k_descend_batch<<<(unsigned)grid, bs, 0, s>>>(E, start_off, np, count, tol * tol, starts, cand,
                                                status, seg, ctr);
  return cudaGetLastError();
}

cudaError_t launch_seg_keys(const uint32_t* vals, const uint16_t* seg, const uint8_t* status,
                            int64_t count, uint64_t* keys, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_seg_keys<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(vals, seg, status, count, keys);
  return cudaGetLastError();
}

}  // namespace mt
