// mt_newton.cu -- step a4 (Newton descents) and a0 (plain evaluation).
//
// Newton map N_P(z) = z - P(z)/P'(z) (Sec. 3.3, eq. Newton).  Each start of
// the discrete level line is iterated until the step drops below tol, the
// iterate jumps far away (a long-distance jump, Sec. 6.4.1), or the cap
// max{20, I_N log2 d} of Algorithm S_par is reached.
//
// GB300 design.  Descent lengths vary (about 10-12 steps when convergent,
// the cap when not; Sec. 6.4.1), which is the paper's own objection to a
// GPU port (Sec. 6.4.5: lock-step lanes would make the worst case the
// norm).  The kernel is persistent: a grid of (SMs x resident blocks) warps
// drains one atomic work queue; a lane that finishes its descent is refilled
// at the next step through a warp vote (__ballot_sync) and one atomicAdd per
// warp, so lanes never idle while the queue holds work.
#include "mt_common.cuh"

namespace mt {

// LIST: the starts list[0 .. *nlist) only (start list[t] for queue entry
// t); the queue is ctr->queue_head2 then.
template <bool LIST>
__global__ void __launch_bounds__(128) k_descend(PolyDev P, const double2* __restrict__ starts,
                                                 int64_t count, double tol2, int cap,
                                                 double2* __restrict__ cand,
                                                 uint8_t* __restrict__ status, DevCounters* ctr,
                                                 const uint32_t* __restrict__ list = nullptr,
                                                 const unsigned long long* __restrict__ nlist = nullptr) {
  if (LIST) count = (int64_t)*nlist < count ? (int64_t)*nlist : count;
  unsigned long long* queue = LIST ? &ctr->queue_head2 : &ctr->queue_head;
  const unsigned lane = threadIdx.x & 31;
  int64_t idx = -1;  // current queue entry (-1: idle, >= count: queue drained)
  int64_t at = 0;    // its start
  double zr = 0.0, zi = 0.0, rdiv2 = 16.0, prev2 = 1e300;
  int it = 0;
  unsigned long long steps = 0, nconv = 0, ndiv = 0, nto = 0;
  for (;;) {
    // refill idle lanes from the queue (one atomic per warp)
    const unsigned need = __ballot_sync(0xffffffffu, idx < 0);
    if (need) {
      unsigned long long base = 0;
      if (lane == (unsigned)(__ffs(need) - 1)) base = atomicAdd(queue, (unsigned long long)__popc(need));
      base = __shfl_sync(0xffffffffu, base, __ffs(need) - 1);
      if (idx < 0) {
        idx = (int64_t)(base + __popc(need & lanemask_lt()));
        if (idx < count) {
          at = LIST ? (int64_t)list[idx] : idx;
          const double2 z0 = starts[at];
          zr = z0.x;
          zi = z0.y;
          it = 0;
          prev2 = 1e300;
          // long jump: beyond twice the start radius and outside D(0, 4)
          rdiv2 = fmax(16.0, 4.0 * fma(zr, zr, zi * zi));
        }
      }
    }
    const bool active = idx >= 0 && idx < count;
    if (!__any_sync(0xffffffffu, active)) break;
    if (active) {
      double vr, vi, dr, di;
      eval_P(P, zr, zi, vr, vi, dr, di);
      double qr, qi;
      cdiv_f64(vr, vi, dr, di, qr, qi);
      zr -= qr;
      zi -= qi;
      ++it;
      ++steps;
      const double s2 = fma(qr, qr, qi * qi);
      int outcome = -1;
      // Past the finiteness test z, hence q, is finite, so |z|^2, s2, rdiv2,
      // tol2 and prev2 are all in [+0, +inf], and prev2 >= tol2 >= 1e-300 (a
      // step below tol2 ends the descent): they compare as integers
      // (s2 >= prev2 / 4 as ord(s2) >= ord(prev2) - ORD_QUARTER).
      if (!finite2(zr, zi) || ord_f64(fma(zr, zr, zi * zi)) > ord_f64(rdiv2)) outcome = 1;
      else if (ord_f64(s2) < ord_f64(tol2)) outcome = 0;  // the step that met tol also squared the error
      // binary64 rounding floor: steps stopped shrinking within a few ulp of z
      // (between two close roots Newton also stalls, at |step| ~ their
      // separation^2 / distance, far above this floor)
      else if (ord_f64(s2) >= ord_f64(prev2) - ORD_QUARTER && s2 < floor2_f64(zr, zi)) outcome = 0;
      else if (it >= cap) outcome = 2;
      prev2 = s2;
      if (outcome >= 0) {
        cand[at] = make_double2(zr, zi);
        status[at] = (uint8_t)outcome;
        nconv += outcome == 0;
        ndiv += outcome == 1;
        nto += outcome == 2;
        idx = -1;
      }
    }
  }
  warp_add_u64(&ctr->desc_newton, steps);
  if (!LIST) {  // a list's outcomes are counted where it joins the others
    warp_add_u64(&ctr->n_conv, nconv);
    warp_add_u64(&ctr->n_diverge, ndiv);
    warp_add_u64(&ctr->n_timeout, nto);
  }
}

// Descents on q_{l,n} (multiple roots, Thm fact_mis), evaluated as the
// product p_n prod s_{j,n} (orbit_q_f64), so that values keep their relative
// accuracy up to a multiple root.  Near a root of multiplicity mu Newton
// contracts linearly, |step_{k+1}| / |step_k| -> 1 - 1/mu (eq. newtonLin).
// When three successive ratios agree and give mu within 0.15 of an integer
// m >= 2, a trial step z - m P/P' is taken (eq. newtonAcc).  Next to a
// multiple root it lands much closer, the next plain step is short, and the
// Newton step of p_n (of which the multiple root is a simple root) is m times
// that of q: the lane then keeps the factor m, which converges quadratically.
// A cluster looks the same from afar, but there the trial lands near its
// centre, where one of the two tests fails: the trial is undone and the lane
// stays on plain Newton, which separates the cluster.
// If an accelerated lane stops contracting (it circles a cluster), it falls
// back to plain Newton the same way.  Persistent, with the refill of
// k_descend; the per-lane state adds the trial point and the factor.
__global__ void __launch_bounds__(128) k_descend_q(PolyDev P, const double2* __restrict__ starts,
                                                   int64_t count, double tol2, int cap,
                                                   double2* __restrict__ cand,
                                                   uint8_t* __restrict__ status, DevCounters* ctr) {
  const unsigned lane = threadIdx.x & 31;
  int64_t idx = -1;
  double zr = 0.0, zi = 0.0, rdiv2 = 16.0, prev2 = 1e300, r_prev = 0.0, acc2 = 0.0, wpr = 0.0, wpi = 0.0;
  int it = 0, lin = 0, mult = 1, pending = 0, trial = 0, no_acc = 0;
  unsigned long long steps = 0, nconv = 0, ndiv = 0, nto = 0;
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
          const double2 z0 = starts[idx];
          zr = z0.x;
          zi = z0.y;
          it = 0;
          prev2 = 1e300;
          r_prev = 0.0;
          lin = 0;
          mult = 1;
          pending = 0;
          trial = 0;
          no_acc = 0;
          rdiv2 = fmax(16.0, 4.0 * fma(zr, zr, zi * zi));
        }
      }
    }
    const bool active = idx >= 0 && idx < count;
    if (!__any_sync(0xffffffffu, active)) break;
    if (active) {
      double vr, vi, dr, di;
      orbit_q_f64(P.l, P.n, zr, zi, vr, vi, dr, di);
      double qr, qi;
      cdiv_f64(vr, vi, dr, di, qr, qi);
      ++it;
      ++steps;
      int outcome = -1;
      bool undo = false;
      if (trial) {  // the first plain step after a trial step
        // next to a root of multiplicity m, a simple root of p_n (Thm fact_mis),
        // the p_n step is m times the q step; the weighted centre of a cluster
        // (a multiple root with a simple one nearby) gives another ratio
        const double sq2 = fma(qr, qr, qi * qi);
        bool ok = sq2 <= 0.25 * acc2;
        if (ok) {
          double pr, pi, pdr, pdi, tr, ti;
          orbit_pn_f64(P.n, zr, zi, pr, pi, pdr, pdi);
          cdiv_f64(pr, pi, pdr, pdi, tr, ti);
          const double ratio2 = fma(tr, tr, ti * ti) / sq2, m = (double)trial;
          ok = ratio2 >= 0.5625 * m * m && ratio2 <= 1.5625 * m * m;  // within 25 % of m
        }
        if (ok) {
          mult = trial;
        } else {  // landed in a cluster: back to the point before the trial
          zr = wpr;
          zi = wpi;
          no_acc = 1;
          lin = 0;
          undo = true;
        }
        trial = 0;
      }
      if (!undo) {
        double f = (double)mult;
        const bool was_pending = pending != 0;
        if (was_pending) {
          wpr = zr;
          wpi = zi;
          f = (double)pending;
        }
        qr *= f;
        qi *= f;
        zr -= qr;
        zi -= qi;
        const double s2 = fma(qr, qr, qi * qi);
        if (was_pending) {
          acc2 = s2;
          trial = pending;
          pending = 0;
        }
        if (!finite2(zr, zi) || fma(zr, zr, zi * zi) > rdiv2) outcome = 1;
        else if (s2 < tol2) outcome = 0;
        else if (s2 >= 0.25 * prev2 && s2 < floor2_f64(zr, zi)) outcome = 0;
        if (outcome == 0 && (mult > 1 || s2 > 0.09 * prev2)) {
          // a multiple root (accelerated, or still contracting linearly at
          // the stop, which leaves it tens of ulps short): finish on p_n,
          // where it is a simple root, if p_n sees its root right there
          double pr, pi, pdr, pdi, tr, ti;
          orbit_pn_f64(P.n, zr, zi, pr, pi, pdr, pdi);
          cdiv_f64(pr, pi, pdr, pdi, tr, ti);
          const double lim = 1e-9 * (1.0 + fabs(zr) + fabs(zi));
          if (fma(tr, tr, ti * ti) <= lim * lim) {
            zr -= tr;
            zi -= ti;
            for (int k = 0; k < 3; ++k) {
              orbit_pn_f64(P.n, zr, zi, pr, pi, pdr, pdi);
              cdiv_f64(pr, pi, pdr, pdi, tr, ti);
              if (!finite2(tr, ti)) break;
              zr -= tr;
              zi -= ti;
            }
            steps += 4;
          }
        }
        if (outcome < 0 && !was_pending && it > 1) {
          const double r = sqrt(s2 / prev2);
          if (mult > 1) {
            if (r >= 0.9) {  // circling a cluster: plain Newton from here
              mult = 1;
              no_acc = 1;
              lin = 0;
            }
          } else {
            lin = (r > 0.35 && r < 0.98 && fabs(r - r_prev) < 0.03 * r) ? lin + 1 : 0;
            if (lin >= 3 && !no_acc) {
              const double mu = 1.0 / (1.0 - r);
              const int m = (int)(mu + 0.5);
              if (m >= 2 && fabs(mu - m) < 0.15) pending = m;
              lin = 0;
            }
          }
          r_prev = r;
        }
        prev2 = s2;
      }
      if (outcome < 0 && it >= cap) outcome = 2;
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
  warp_add_u64(&ctr->n_conv, nconv);
  warp_add_u64(&ctr->n_diverge, ndiv);
  warp_add_u64(&ctr->n_timeout, nto);
}

__global__ void k_eval(PolyDev P, const double2* __restrict__ c, int64_t count,
                       double2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double2 z = c[i];
  double vr, vi, dr, di;
  eval_P(P, z.x, z.y, vr, vi, dr, di);
  out[2 * i] = make_double2(vr, vi);
  out[2 * i + 1] = make_double2(dr, di);
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

cudaError_t launch_descend(const PolyDev& P, const double2* starts, int64_t count, double tol,
                           int cap, double2* cand, uint8_t* status, DevCounters* ctr, int block,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int bs = 128;
  (void)block;
  int per_sm = 0;
  cudaError_t e = P.kind == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend_q, bs, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend<false>, bs, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // The binary64 pipe (2 DFMA lanes per SM on GB300) is saturated by 8 warps
  // per SM; more resident lanes only lengthen the tail in which a warp waits
  // for its last descents.  Measured at p_20: 10 blocks/SM 4.18 ms, 4 blocks
  // 3.76 ms, 2 blocks 3.56 ms, 1 block 3.88 ms.
  if (per_sm > 2) per_sm = 2;
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  const int64_t need = (count + bs - 1) / bs;
  if (grid > need) grid = need;
  MT_COUNT_LAUNCH(1);
  if ((e = ktimer_begin(KS_DESC64, s)) != cudaSuccess) return e;
  if (P.kind == 2)
    k_descend_q<<<(unsigned)grid, bs, 0, s>>>(P, starts, count, tol * tol, cap, cand, status, ctr);
  else
    k_descend<false><<<(unsigned)grid, bs, 0, s>>>(P, starts, count, fmax(tol * tol, 1e-300), cap, cand, status,
                                                   ctr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return ktimer_end(s);
}

cudaError_t launch_descend_list(const PolyDev& P, const double2* starts, const uint32_t* list,
                                const unsigned long long* nlist, int64_t count, double tol, int cap,
                                double2* cand, uint8_t* status, DevCounters* ctr, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (P.kind == 2) return cudaErrorInvalidValue;  // q_{l,n} has no mixed tier
  const int bs = 128;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_descend<true>, bs, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > 2) per_sm = 2;  // as launch_descend
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  const int64_t need = (count + bs - 1) / bs;
  if (grid > need) grid = need;
  if ((e = cudaMemsetAsync(&ctr->queue_head2, 0, sizeof(ctr->queue_head2), s)) != cudaSuccess) return e;
  MT_COUNT_LAUNCH(1);
  if ((e = ktimer_begin(KS_DESC64, s)) != cudaSuccess) return e;
  k_descend<true><<<(unsigned)grid, bs, 0, s>>>(P, starts, count, fmax(tol * tol, 1e-300), cap, cand, status, ctr,
                                                list, nlist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return ktimer_end(s);
}

cudaError_t launch_eval(const PolyDev& P, const double2* c, int64_t count, double2* out,
                        cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int bs = 128;
  MT_COUNT_LAUNCH(1);
  k_eval<<<(unsigned)((count + bs - 1) / bs), bs, 0, s>>>(P, c, count, out);
  return cudaGetLastError();
}

}  // namespace mt
