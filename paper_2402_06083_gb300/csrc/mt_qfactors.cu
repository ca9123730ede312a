// mt_qfactors.cu -- q_{l,n} in the double-double tier, through its factors.
//
// eq. polySimple gives s_{j,n} = q_{j,n} / q_{j-1,n}; telescoped from
// q_{0,n} = p_n (with s_{1,n} = p_n, eq. hypCase) it reads
//   q_{l,n} = p_n^2 prod_{j=2..l} s_{j,n}.
// Every factor has simple roots only, so the roots of q with their
// multiplicities are the union of the factors' roots, a root counted once
// per factor that holds it: Hyp(k), k | n, lies in p_n (twice) and in the
// s_{j,n} with k | j - 1, which gives Thm fact_mis' eta_l(k) =
// floor((l-1)/k) + 2; Mis(j,k) lies in s_{j,n} alone (eq. polyMisSimple).
// The host splits each factor with its own certified double-double split
// (mt_api.cu) and these kernels merge the lists: the Hyp roots come from
// p_n, the Mis roots from the s_{j,n}, and a final sort orders the union by
// (Re, Im) (eq. defLexi).
#include "mt_common.cuh"

namespace mt {

__global__ void k_qf_append(const double2* __restrict__ roots, const uint8_t* __restrict__ type, int64_t count,
                            int j, int l, int n, double2* __restrict__ u_roots, uint8_t* __restrict__ u_pre,
                            uint8_t* __restrict__ u_per, uint8_t* __restrict__ u_mult, int64_t cap,
                            unsigned long long* cnt) {
  const unsigned lane = threadIdx.x & 31;
  unsigned long long nmult = 0, nbad = 0, nreal = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
  for (int64_t base = i0; base < count; base += stride) {  // warp-uniform trip count
    const int64_t i = base + threadIdx.x;
    bool take = false;
    int k = 0, mu = 0;
    if (i < count) {
      const int t = type[i];
      if (j == 0) {  // p_n: Hyp(k), k | n
        k = t;
        if (k >= 1 && k <= n && n % k == 0) {
          take = true;
          mu = (l - 1) / k + 2;
        } else {
          ++nbad;
        }
      } else if (t < 32) {  // s_{j,n}: Mis(j,k), k | n
        k = t;
        if (k >= 1 && k <= n && n % k == 0) {
          take = true;
          mu = 1;
        } else {
          ++nbad;
        }
      } else if (!(t - 32 >= 1 && t - 32 <= n && n % (t - 32) == 0 && (j - 1) % (t - 32) == 0)) {
        ++nbad;  // neither Mis(j,k) nor one of the Hyp(k) of s_{j,n}
      }
    }
    // one atomic per warp for the positions
    const unsigned m = __ballot_sync(0xffffffffu, take);
    unsigned long long b = 0;
    if (lane == 0 && m) b = atomicAdd(&cnt[0], (unsigned long long)__popc(m));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (take) {
      const int64_t pos = (int64_t)b + __popc(m & lanemask_lt());
      if (pos < cap) {
        u_roots[pos] = roots[i];
        u_pre[pos] = (uint8_t)j;
        u_per[pos] = (uint8_t)k;
        u_mult[pos] = (uint8_t)mu;
      }
      nmult += mu;
      nreal += roots[i].y == 0.0;
    }
  }
  warp_add_u64(&cnt[1], nmult);
  warp_add_u64(&cnt[2], nbad);
  warp_add_u64(&cnt[3], nreal);
}

__global__ void k_qf_keys(const double2* __restrict__ z, const uint32_t* __restrict__ perm, int64_t cap,
                          const unsigned long long* __restrict__ n_dev, int use_im, uint64_t* __restrict__ keys,
                          uint32_t* __restrict__ vals) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)*n_dev < cap ? (int64_t)*n_dev : cap;
  if (p >= nn) return;
  const uint32_t i = perm ? perm[p] : (uint32_t)p;
  keys[p] = f64_key(use_im ? z[i].y : z[i].x);
  vals[p] = i;
}

__global__ void k_qf_gather(const uint32_t* __restrict__ perm, int64_t cap,
                            const unsigned long long* __restrict__ n_dev, const double2* __restrict__ u_roots,
                            const uint8_t* __restrict__ u_pre, const uint8_t* __restrict__ u_per,
                            const uint8_t* __restrict__ u_mult, double2* __restrict__ roots,
                            uint8_t* __restrict__ pre, uint8_t* __restrict__ per, uint8_t* __restrict__ mult) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)*n_dev < cap ? (int64_t)*n_dev : cap;
  if (p >= nn) return;
  const uint32_t i = perm[p];
  roots[p] = u_roots[i];
  if (pre) pre[p] = u_pre[i];
  if (per) per[p] = u_per[i];
  if (mult) mult[p] = u_mult[i];
}

cudaError_t launch_qf_append(const double2* roots, const uint8_t* type, int64_t count, int j, int l, int n,
                             double2* u_roots, uint8_t* u_pre, uint8_t* u_per, uint8_t* u_mult, int64_t cap,
                             unsigned long long* cnt, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t nb = std::min<int64_t>((count + 255) / 256, (int64_t)device_sm_count() * 8);
  MT_COUNT_LAUNCH(1);
  k_qf_append<<<(unsigned)nb, 256, 0, s>>>(roots, type, count, j, l, n, u_roots, u_pre, u_per, u_mult, cap, cnt);
  return cudaGetLastError();
}

cudaError_t launch_qf_keys(const double2* z, const uint32_t* perm, int64_t cap, const unsigned long long* n_dev,
                           int use_im, uint64_t* keys, uint32_t* vals, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_qf_keys<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(z, perm, cap, n_dev, use_im, keys, vals);
  return cudaGetLastError();
}

cudaError_t launch_qf_gather(const uint32_t* perm, int64_t cap, const unsigned long long* n_dev,
                             const double2* u_roots, const uint8_t* u_pre, const uint8_t* u_per,
                             const uint8_t* u_mult, double2* roots, uint8_t* pre, uint8_t* per, uint8_t* mult,
                             cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_qf_gather<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(perm, cap, n_dev, u_roots, u_pre, u_per, u_mult, roots,
                                                             pre, per, mult);
  return cudaGetLastError();
}

}  // namespace mt
