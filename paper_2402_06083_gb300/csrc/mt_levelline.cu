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
#include "mt_levelline.cuh"

namespace mt {

__global__ void k_seed_lift(PolyDev P, double lambda0, int64_t N0, int log2N0, int shrink,
                            double2* seeds, DevCounters* ctr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0;
  if (j <= N0 / 2) seeds[j] = lift_seed(P, lambda0, N0, log2N0, shrink, j, steps);
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->seed_newton, steps);
}

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
  if (j < nchunks) fails = walk_chunk(P, ph, M, every, L, nchunks, j, seeds, starts, steps) ? 1 : 0;
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

// Chunks [j0, j0 + nch) only, starts written from index j0 L / every on
// (streamed splits, which walk the level line a range of chunks at a time).
__global__ void k_walk_range(PolyDev P, double lambda0, int M, int every, int64_t L, int64_t nchunks,
                             int64_t j0, int64_t nch, const double2* __restrict__ seeds,
                             double2* __restrict__ starts, DevCounters* ctr) {
  __shared__ double2 ph[64];
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double c, s;
    unit_phase((uint64_t)q, (uint64_t)M, c, s);
    ph[q] = make_double2(lambda0 * c, lambda0 * s);
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, fails = 0;
  if (i < nch) {
    const int64_t j = j0 + i;
    fails = walk_chunk_from(P, ph, M, every, L, nchunks, j, seeds[j], seeds[j + 1], starts, steps,
                            j0 * L / every)
                ? 1
                : 0;
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->walk_fail, fails);
}

cudaError_t launch_walk_range(const PolyDev& P, double lambda0, int M, int every, int64_t L, int64_t nchunks,
                              int64_t j0, int64_t nch, const double2* seeds, double2* starts, DevCounters* ctr,
                              cudaStream_t s, int block) {
  if (nch <= 0) return cudaSuccess;
  const int bs = (block >= 32 && block <= 1024 && block % 32 == 0) ? block : 64;
  MT_COUNT_LAUNCH(1);
  k_walk_range<<<(unsigned)((nch + bs - 1) / bs), bs, 0, s>>>(P, lambda0, M, every, L, nchunks, j0, nch, seeds,
                                                              starts, ctr);
  return cudaGetLastError();
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
                        cudaStream_t s, int block) {
  const int bs = (block >= 32 && block <= 1024 && block % 32 == 0) ? block : 64;
  const int64_t grid = (nchunks + bs - 1) / bs;
  MT_COUNT_LAUNCH(1);
  cudaError_t e = ktimer_begin(KS_WALK, s);
  if (e != cudaSuccess) return e;
  k_walk<<<(unsigned)grid, bs, 0, s>>>(P, lambda0, M, every, L, nchunks, seeds, starts, ctr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return ktimer_end(s);
}

// Repairs of the mixed tier in binary64, inside the same launch sequence
// (no host round trip).  Seeds whose binary32 lift failed are lifted again;
// chunks whose binary32 walk missed the next seed (a skipped turn, or a
// binary32 end seed farther off than the end check allows near a cluster)
// are walked again from both end seeds lifted again in binary64 (kept
// local: the other chunks met the array's seeds already).  A repaired item
// takes its failure off walk_fail; one that fails again stays counted and
// the host then repeats the split in binary64.  Lanes without a flag exit
// at once.
__global__ void k_seed_repair(PolyDev P, double lambda0, int64_t N0, int log2N0, int shrink,
                              double2* __restrict__ seeds, uint8_t* __restrict__ seed_bad,
                              DevCounters* ctr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long steps = 0, fixed = 0;
  if (j <= N0 / 2 && seed_bad[j]) {
    seeds[j] = lift_seed(P, lambda0, N0, log2N0, shrink, j, steps);
    seed_bad[j] = 0;
    fixed = 1;
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->seed_newton, steps);
  warp_add_u64(&ctr->walk_fail, 0ull - fixed);
}

__global__ void k_walk_repair(PolyDev P, double lambda0, int M, int every, int64_t L, int64_t nchunks,
                              int64_t N0, int log2N0, int shrink, const double2* __restrict__ seeds,
                              double2* __restrict__ starts, uint8_t* __restrict__ chunk_fail,
                              DevCounters* ctr, int64_t j0, int64_t nch) {
  __shared__ double2 ph[64];
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double c, s;
    unit_phase((uint64_t)q, (uint64_t)M, c, s);
    ph[q] = make_double2(lambda0 * c, lambda0 * s);
  }
  __syncthreads();
  const int64_t jl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = j0 + jl;
  unsigned long long steps = 0, fixed = 0;
  if (jl < nch && j < nchunks && chunk_fail[j]) {
    const double2 a = lift_seed(P, lambda0, N0, log2N0, shrink, j, steps);
    const double2 b = lift_seed(P, lambda0, N0, log2N0, shrink, j + 1, steps);
    if (!walk_chunk_from(P, ph, M, every, L, nchunks, j, a, b, starts, steps, j0 * L / every)) {
      chunk_fail[j] = 0;
      fixed = 1;
    }
  }
  warp_add_u64(&ctr->walk_newton, steps);
  warp_add_u64(&ctr->walk_fail, 0ull - fixed);
}

cudaError_t launch_mixed_repair_seeds(const PolyDev& P, double lambda0, int64_t N0, int shrink,
                                      double2* seeds, uint8_t* seed_bad, DevCounters* ctr,
                                      cudaStream_t s) {
  int log2N0 = 0;
  while ((int64_t(1) << log2N0) < N0) ++log2N0;
  const int64_t n = N0 / 2 + 1;
  MT_COUNT_LAUNCH(1);
  k_seed_repair<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(P, lambda0, N0, log2N0, shrink, seeds,
                                                            seed_bad, ctr);
  return cudaGetLastError();
}

cudaError_t launch_mixed_repair_walk(const PolyDev& P, double lambda0, int M, int every, int64_t L,
                                     int64_t nchunks, int shrink, const double2* seeds,
                                     double2* starts, uint8_t* chunk_fail, DevCounters* ctr,
                                     cudaStream_t s, int64_t j0, int64_t nch) {
  if (nch < 0) nch = nchunks - j0;
  if (nch <= 0) return cudaSuccess;
  const int64_t N0 = 2 * nchunks;
  int log2N0 = 0;
  while ((int64_t(1) << log2N0) < N0) ++log2N0;
  MT_COUNT_LAUNCH(1);
  k_walk_repair<<<(unsigned)((nch + 127) / 128), 128, 0, s>>>(P, lambda0, M, every, L, nchunks, N0, log2N0,
                                                              shrink, seeds, starts, chunk_fail, ctr, j0, nch);
  return cudaGetLastError();
}

}  // namespace mt
