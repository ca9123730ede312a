// mt_dedup.cu -- step a5: the separated, conjugate-symmetric, sorted root set.
//
// Semantics follow the paper's nset (Sec. 6.1): two points are the same root
// when max(|dRe|, |dIm|) < eps (eq. nsetAsumption); only the upper half
// plane is stored and a point with |Im| < eps/2 is real (Im := 0); the set
// is ordered by (Re, Im) (eq. defLexi).
//
// GB300 design.  The paper inserts one root at a time into bars of a
// sorted container.  Here the whole candidate array is handled at once:
// fold + key -> LSD radix sort of Re keys -> each sorted candidate checks
// the earlier candidates of its Re window -> exclusive scan -> gather.
// Every kernel is a coalesced pass over HBM; the radix sort ranks keys
// stably inside a block (digit peers of a warp by ballots).
#include "mt_common.cuh"

namespace mt {

// ---------------------------------------------------------------------------
// counters
__global__ void k_init_counters(DevCounters* c) {
  unsigned long long* w = (unsigned long long*)c;
  const int nw = (int)(sizeof(DevCounters) / sizeof(unsigned long long));
  for (int i = threadIdx.x; i < nw; i += blockDim.x) w[i] = 0ull;
  __syncthreads();
  if (threadIdx.x == 0) c->min_radius_bits = 0x7ff0000000000000ull;  // +inf
}

cudaError_t launch_init_counters(DevCounters* ctr, cudaStream_t s) {
  MT_COUNT_LAUNCH(1);
  k_init_counters<<<1, 128, 0, s>>>(ctr);
  return cudaGetLastError();
}

__global__ void k_keys_plain(const double2* __restrict__ pts, int64_t count,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  keys[i] = f64_key(pts[i].x);
  vals[i] = (uint32_t)i;
}

cudaError_t launch_keys_plain(const double2* pts, int64_t count, uint64_t* keys, uint32_t* vals,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_keys_plain<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(pts, count, keys, vals);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fold + keys
__global__ void k_fold_keys(const uint8_t* __restrict__ status, double2* __restrict__ cand,
                            int64_t count, double eps, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint64_t key = ~0ull;
  if (status[i] == 0) {
    double2 z = cand[i];
    z.y = fabs(z.y);               // conjugate fold: P has real coefficients
    if (z.y < 0.5 * eps) z.y = 0.0;  // indistinguishable from its conjugate: real
    cand[i] = z;
    key = f64_key(z.x);
  }
  keys[i] = key;
  vals[i] = (uint32_t)i;
}

// The same over a list of candidates (the mixed tier's finished group
// heads, list[0 .. *n_list)): entry t holds candidate list[t]; the
// converged ones are counted in *n_ok (they sort first).
__global__ void k_fold_keys_list(const uint32_t* __restrict__ list, const unsigned long long* __restrict__ n_list,
                                 int64_t cap, const uint8_t* __restrict__ status, double2* __restrict__ cand,
                                 double eps, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                 unsigned long long* n_ok) {
  const int64_t nl = (int64_t)*n_list < cap ? (int64_t)*n_list : cap;
  unsigned long long ok = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl;
       t += (int64_t)gridDim.x * blockDim.x) {  // grid-stride: few counter atomics
    const uint32_t i = list[t];
    uint64_t key = ~0ull;
    if (status[i] == 0) {
      double2 z = cand[i];
      z.y = fabs(z.y);
      if (z.y < 0.5 * eps) z.y = 0.0;
      cand[i] = z;
      key = f64_key(z.x);
      ++ok;
    }
    keys[t] = key;
    vals[t] = i;
  }
  warp_add_u64(n_ok, ok);
}

cudaError_t launch_fold_keys_list(const uint32_t* list, const unsigned long long* n_list, int64_t cap,
                                  const uint8_t* status, double2* cand, double eps, uint64_t* keys, uint32_t* vals,
                                  unsigned long long* n_ok, cudaStream_t s) {
  if (cap <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(n_ok, 0, sizeof(*n_ok), s);
  if (e != cudaSuccess) return e;
  MT_COUNT_LAUNCH(1);
  const int64_t nb = std::min<int64_t>((cap + 255) / 256, (int64_t)device_sm_count() * 8);
  k_fold_keys_list<<<(unsigned)nb, 256, 0, s>>>(list, n_list, cap, status, cand, eps, keys, vals, n_ok);
  return cudaGetLastError();
}

cudaError_t launch_fold_keys(const uint8_t* status, double2* cand, int64_t count, double eps,
                             uint64_t* keys, uint32_t* vals, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_fold_keys<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(status, cand, count, eps, keys, vals);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of u32 (three passes: tile sums, scan of sums, tile scan).
constexpr int SCAN_BS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int64_t SCAN_TILE = (int64_t)SCAN_BS * SCAN_ITEMS;

__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v,
                                                                  unsigned long long* sh,
                                                                  unsigned long long* total) {
  // warp scan
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) sh[lane] = t;
  }
  __syncthreads();
  const unsigned long long warp_off = w ? sh[w - 1] : 0;
  if (total) *total = sh[nw - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_tile_sums(const uint32_t* __restrict__ in, int64_t n,
                                 unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  unsigned long long acc = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int64_t i = base + (int64_t)k * SCAN_BS + threadIdx.x;
    if (i < n) acc += in[i];
  }
  unsigned long long tot;
  block_excl_scan_u64(acc, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(unsigned long long* sums, int64_t nb, unsigned long long* total) {
  __shared__ unsigned long long sh[32];
  // one block: each thread owns a contiguous run of sums
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  unsigned long long acc = 0;
  for (int64_t b = b0; b < b0 + per && b < nb; ++b) acc += sums[b];
  unsigned long long tot;
  unsigned long long off = block_excl_scan_u64(acc, sh, &tot);
  for (int64_t b = b0; b < b0 + per && b < nb; ++b) {
    const unsigned long long v = sums[b];
    sums[b] = off;
    off += v;
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void k_scan_tiles(const uint32_t* in, uint32_t* out, int64_t n,
                             const unsigned long long* __restrict__ sums) {
  __shared__ unsigned long long sh[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  // each thread owns SCAN_ITEMS consecutive elements (blocked arrangement)
  const int64_t t0 = base + (int64_t)threadIdx.x * SCAN_ITEMS;
  // a full run of 8 moves as two 16-byte words where both buffers are
  // 16-byte aligned (t0 is a multiple of 8)
  const bool full = t0 + SCAN_ITEMS <= n && ((((uintptr_t)in) | ((uintptr_t)out)) & 15u) == 0;
  uint32_t v[SCAN_ITEMS];
  unsigned long long acc = 0;
  if (full) {
    const uint4 a = *(const uint4*)(in + t0), b = *(const uint4*)(in + t0 + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = (t0 + k < n) ? in[t0 + k] : 0u;
  }
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) acc += v[k];
  unsigned long long off = block_excl_scan_u64(acc, sh, nullptr) + sums[blockIdx.x];
  uint32_t o[SCAN_ITEMS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    o[k] = (uint32_t)off;
    off += v[k];
  }
  if (full) {
    *(uint4*)(out + t0) = make_uint4(o[0], o[1], o[2], o[3]);
    *(uint4*)(out + t0 + 4) = make_uint4(o[4], o[5], o[6], o[7]);
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
      if (t0 + k < n) out[t0 + k] = o[k];
  }
}

size_t scan_temp_bytes(int64_t n) {
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(nb + 1) * sizeof(unsigned long long);
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, void* temp,
                                  unsigned long long* total, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned long long* sums = (unsigned long long*)temp;
  MT_COUNT_LAUNCH(1);
  k_scan_tile_sums<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, n, sums);
  MT_COUNT_LAUNCH(1);
  k_scan_sums<<<1, 1024, 0, s>>>(sums, nb, total);
  MT_COUNT_LAUNCH(1);
  k_scan_tiles<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, out, n, sums);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, stable, bound by HBM traffic (a pass reads
// each key once for the counts, then reads and writes key and value: 32
// bytes per element for 64-bit keys and 32-bit values).
//
// A pass is three launches over one persistent grid of G blocks.  Block b
// owns the contiguous tiles [nt b / G, nt (b+1) / G) of the nt tiles of
// RS_TILE elements.  k_rs_hist counts the digits of each block's range;
// k_rs_offsets scans those counts digit-major (digit d of block b starts
// after every smaller digit and after digit d of blocks before b); the
// scatter then walks its range tile by tile, carrying per-digit output
// positions, so the order within a digit is the input order (stability).
// Inside a tile, warp w holds elements [256 w, 256 w + 256) of it, item k of
// lane j being element 256 w + 32 k + j: loads coalesce per item, and the
// rank of an element among its digit is counted within its warp (a running
// count per digit and warp in shared memory) plus the counts of the warps
// before it.  The tile is then staged in shared memory in digit order and
// written out with consecutive threads on consecutive addresses of a digit's
// run.  The next tile's keys and values are loaded into registers while the
// current one is ranked and written.
constexpr int RS_BS = 256;
constexpr int RS_WARPS = RS_BS / 32;
constexpr int RS_ITEMS = 8;
constexpr int64_t RS_TILE = (int64_t)RS_BS * RS_ITEMS;
constexpr int RS_GRID_MAX = 2048;

// n_dev: NULL, or the number of entries on the device (at most n)
__device__ __forceinline__ int64_t rs_count(int64_t n, const unsigned long long* n_dev) {
  if (!n_dev) return n;
  const int64_t d = (int64_t)*n_dev;
  return d < n ? d : n;
}

// The lanes of the warp whose value d (a digit 0..255, or 256 for no
// element) equals this lane's.  BAL: nine ballots, one per bit (measured
// faster on the 64-bit keys of the root sets, whose high bytes repeat
// along a warp); else one match (faster on the finish keys' uniform
// digits).
template <bool BAL>
__device__ __forceinline__ unsigned rs_peers(unsigned d) {
  if (!BAL) return __match_any_sync(0xffffffffu, d);
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned v = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? v : ~v;
  }
  return peers;
}

// block b's tiles [t0, t1) of the ceil(n / RS_TILE) tiles
__device__ __forceinline__ void rs_range(int64_t n, int64_t& t0, int64_t& t1) {
  const int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  t0 = nt * blockIdx.x / gridDim.x;
  t1 = nt * (blockIdx.x + 1) / gridDim.x;
}

template <bool BAL>
__global__ void __launch_bounds__(RS_BS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                   int shift, uint32_t* __restrict__ hist,
                                                   const unsigned long long* __restrict__ n_dev) {
  __shared__ uint32_t cnt[256];
  n = rs_count(n, n_dev);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  cnt[t] = 0;
  __syncthreads();
  int64_t t0, t1;
  rs_range(n, t0, t1);
  for (int64_t tl = t0; tl < t1; ++tl) {
    const int64_t base = tl * RS_TILE + w * (RS_ITEMS * 32) + lane;
    unsigned dg[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
      const int64_t i = base + k * 32;
      dg[k] = i < n ? (unsigned)(keys[i] >> shift) & 255u : 256u;
    }
    // BAL (64-bit keys, whose high digits repeat along a warp): lanes that
    // share a digit add once; else (the finish keys' uniform digits, where
    // lanes rarely share one) one shared-memory atomic per element
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
      if (BAL) {
        const unsigned peers = rs_peers<true>(dg[k]);
        if (dg[k] < 256u && (peers & lanemask_lt()) == 0) atomicAdd(&cnt[dg[k]], (uint32_t)__popc(peers));
      } else if (dg[k] < 256u) {
        atomicAdd(&cnt[dg[k]], 1u);
      }
    }
  }
  __syncthreads();
  hist[(int64_t)t * gridDim.x + blockIdx.x] = cnt[t];  // digit-major
}

// per digit d (block d): exclusive scan of the G block counts of d into
// offs[d][.], and their total into tot[d]; the scatter adds the digit's base
// (the totals of the smaller digits).  G <= RS_GRID_MAX = 2 * blockDim.x.
__global__ void k_rs_offsets(const uint32_t* __restrict__ hist, uint32_t* __restrict__ offs,
                             uint32_t* __restrict__ tot, int G) {
  __shared__ unsigned long long sh[32];
  const int64_t row = (int64_t)blockIdx.x * G;
  const int b0 = 2 * threadIdx.x;
  const uint32_t c0 = b0 < G ? hist[row + b0] : 0u;
  const uint32_t c1 = b0 + 1 < G ? hist[row + b0 + 1] : 0u;
  unsigned long long total;
  const unsigned long long off = block_excl_scan_u64((unsigned long long)c0 + c1, sh, &total);
  if (b0 < G) offs[row + b0] = (uint32_t)off;
  if (b0 + 1 < G) offs[row + b0 + 1] = (uint32_t)(off + c0);
  if (threadIdx.x == 0) tot[blockIdx.x] = (uint32_t)total;
}

__device__ __forceinline__ void rs_load(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                        int64_t base, int64_t n, uint64_t* key, uint32_t* val) {
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int64_t i = base + k * 32;
    key[k] = i < n ? kin[i] : 0ull;
    val[k] = i < n ? vin[i] : 0u;
  }
}

template <bool BAL>
__global__ void __launch_bounds__(RS_BS, 3) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint64_t* __restrict__ kout,
                                                         uint32_t* __restrict__ vout, int64_t n, int shift,
                                                         const uint32_t* __restrict__ offs,
                                                         const uint32_t* __restrict__ dtot,
                                                         const unsigned long long* __restrict__ n_dev) {
  __shared__ uint64_t sk[RS_TILE];
  __shared__ uint32_t sv[RS_TILE];
  __shared__ uint32_t wc[RS_WARPS][256];  // per warp: running count, then the warps-before prefix
  __shared__ uint32_t lbase[256];         // staged position of the tile's first element of digit d
  __shared__ uint32_t gpos[256];          // output position of the next element of digit d
  __shared__ uint32_t wsum[RS_WARPS];
  n = rs_count(n, n_dev);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  int64_t t0, t1;
  rs_range(n, t0, t1);
  {  // digit t starts after the smaller digits' totals and digit t of the blocks before
    const uint32_t c = dtot[t];
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    gpos[t] = before + x - c + offs[(int64_t)t * gridDim.x + blockIdx.x];
  }
  uint64_t key[RS_ITEMS];
  uint32_t val[RS_ITEMS];
  const int64_t wl = w * (RS_ITEMS * 32) + lane;  // the thread's first element within a tile
  if (t0 < t1) rs_load(kin, vin, t0 * RS_TILE + wl, n, key, val);
  for (int64_t tl = t0; tl < t1; ++tl) {
    uint64_t nkey[RS_ITEMS];
    uint32_t nval[RS_ITEMS];
    if (tl + 1 < t1) rs_load(kin, vin, (tl + 1) * RS_TILE + wl, n, nkey, nval);
#pragma unroll
    for (int q = 0; q < 256 / 32; ++q) wc[w][lane + 32 * q] = 0;
    __syncwarp();
    const int64_t base = tl * RS_TILE + wl;
    unsigned dg[RS_ITEMS], rk[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
      const bool valid = base + k * 32 < n;
      dg[k] = valid ? (unsigned)(key[k] >> shift) & 255u : 256u;
      const unsigned peers = rs_peers<BAL>(dg[k]);
      const unsigned lt = __popc(peers & lanemask_lt());
      const uint32_t before = valid ? wc[w][dg[k]] : 0u;
      __syncwarp();
      if (valid && lt == 0) wc[w][dg[k]] = before + __popc(peers);
      __syncwarp();
      rk[k] = before + lt;
    }
    __syncthreads();
    // thread t owns digit t: prefix over the warps, and the tile's count r
    uint32_t r = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) {
      const uint32_t c = wc[q][t];
      wc[q][t] = r;
      r += c;
    }
    {  // exclusive scan of the counts over the digits
      uint32_t x = r;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[w] = x;
      __syncthreads();
      uint32_t before = 0;
      for (int q = 0; q < w; ++q) before += wsum[q];
      lbase[t] = before + x - r;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
      if (dg[k] < 256u) {
        const uint32_t p = lbase[dg[k]] + wc[w][dg[k]] + rk[k];
        sk[p] = key[k];
        sv[p] = val[k];
      }
    }
    __syncthreads();
    const int64_t cnt = (n - tl * RS_TILE) < RS_TILE ? (n - tl * RS_TILE) : RS_TILE;
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
      const int j = k * RS_BS + t;
      if (j < cnt) {
        const uint64_t kk = sk[j];
        const unsigned d = (unsigned)(kk >> shift) & 255u;
        const uint32_t pos = gpos[d] + (uint32_t)j - lbase[d];
        kout[pos] = kk;
        vout[pos] = sv[j];
      }
    }
    __syncthreads();
    gpos[t] += r;
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
      key[k] = nkey[k];
      val[k] = nval[k];
    }
  }
}

// blocks of the persistent grid: as many as are resident at once, at most
// one per tile and RS_GRID_MAX
static int64_t rs_grid(int64_t n) {
  static int per_sm = 0;
  if (!per_sm) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_rs_scatter<true>, RS_BS, 0) != cudaSuccess || b < 1)
      b = 1;
    per_sm = b;
  }
  const int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  return std::max<int64_t>(1, std::min<int64_t>({nt, (int64_t)device_sm_count() * per_sm, (int64_t)RS_GRID_MAX}));
}

size_t radix_temp_bytes(int64_t n) {
  const int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  const int64_t nh = 256 * std::max<int64_t>(1, std::min<int64_t>(nt, RS_GRID_MAX));
  return (size_t)nh * 2 * sizeof(uint32_t) + 256 * sizeof(uint32_t);
}

// one pass: digit [shift, shift + 8) from (k0, v0) to (k1, v1)
static cudaError_t rs_pass(const uint64_t* k0, const uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                           int shift, void* temp, const unsigned long long* n_dev, bool bal, cudaStream_t s) {
  const int64_t G = rs_grid(n);
  const int64_t nh = 256 * G;
  uint32_t* hist = (uint32_t*)temp;
  uint32_t* offs = hist + nh;
  uint32_t* dtot = offs + nh;
  MT_COUNT_LAUNCH(1);
  if (bal) k_rs_hist<true><<<(unsigned)G, RS_BS, 0, s>>>(k0, n, shift, hist, n_dev);
  else k_rs_hist<false><<<(unsigned)G, RS_BS, 0, s>>>(k0, n, shift, hist, n_dev);
  MT_COUNT_LAUNCH(1);
  k_rs_offsets<<<256, RS_GRID_MAX / 2, 0, s>>>(hist, offs, dtot, (int)G);
  MT_COUNT_LAUNCH(1);
  if (bal) k_rs_scatter<true><<<(unsigned)G, RS_BS, 0, s>>>(k0, v0, k1, v1, n, shift, offs, dtot, n_dev);
  else k_rs_scatter<false><<<(unsigned)G, RS_BS, 0, s>>>(k0, v0, k1, v1, n, shift, offs, dtot, n_dev);
  return cudaGetLastError();
}

cudaError_t radix_sort_bits(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                            int64_t n, void* temp, int begin_bit, int end_bit, bool* in_alt,
                            cudaStream_t s) {
  *in_alt = false;
  if (n <= 1) return cudaSuccess;
  uint64_t* k0 = keys;
  uint32_t* v0 = vals;
  uint64_t* k1 = keys_alt;
  uint32_t* v1 = vals_alt;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    cudaError_t e = rs_pass(k0, v0, k1, v1, n, shift, temp, nullptr, false, s);
    if (e != cudaSuccess) return e;
    uint64_t* tk = k0; k0 = k1; k1 = tk;
    uint32_t* tv = v0; v0 = v1; v1 = tv;
    *in_alt = !*in_alt;
  }
  return cudaSuccess;
}

cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, void* temp, cudaStream_t s,
                             const unsigned long long* n_dev) {
  if (n <= 1) return cudaSuccess;
  uint64_t* k0 = keys;
  uint32_t* v0 = vals;
  uint64_t* k1 = keys_alt;
  uint32_t* v1 = vals_alt;
  for (int shift = 0; shift < 64; shift += 8) {
    cudaError_t e = rs_pass(k0, v0, k1, v1, n, shift, temp, n_dev, true, s);
    if (e != cudaSuccess) return e;
    uint64_t* tk = k0; k0 = k1; k1 = tk;
    uint32_t* tv = v0; v0 = v1; v1 = tv;
  }
  // 8 passes: the result is back in (keys, vals)
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Cluster: sorted candidate p is a new root unless an earlier candidate q
// with Re_p - Re_q < eps has |Im_p - Im_q| < eps (Chebyshev pixel rule).
__global__ void k_cluster(const double2* __restrict__ cand, const uint32_t* __restrict__ vals,
                          int64_t count, const unsigned long long* __restrict__ n_valid,
                          double eps, uint32_t* __restrict__ flag, DevCounters* ctr, SegView sv) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const int64_t nv = (int64_t)*n_valid;
  if (p >= nv) { flag[p] = 0; return; }
  const double2 z = cand[vals[p]];
  const uint16_t sp = sv.seg ? sv.seg[vals[p]] : 0;
  uint32_t rep = 1;
  int scanned = 0;
  for (int64_t q = p - 1; q >= 0; --q) {
    const uint32_t vq = vals[q];
    if (sv.seg && sv.seg[vq] != sp) break;  // another polynomial of the batch
    const double2 y = cand[vq];
    if (z.x - y.x >= eps) break;
    if (fabs(z.y - y.y) < eps) { rep = 0; break; }
    if (++scanned >= 4096) { atomicAdd(&ctr->cluster_overflow, 1ull); break; }
  }
  flag[p] = rep;
}

cudaError_t launch_cluster(const double2* cand, const uint32_t* vals, int64_t count,
                           const unsigned long long* n_valid, double eps, uint32_t* flag,
                           DevCounters* ctr, cudaStream_t s, SegView sv) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_cluster<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(cand, vals, count, n_valid, eps, flag,
                                                            ctr, sv);
  return cudaGetLastError();
}

__global__ void k_compact(const double2* __restrict__ cand, const uint32_t* __restrict__ vals,
                          const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                          int64_t count, double2* __restrict__ reps, DevCounters* ctr,
                          SegView sv) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  if (flag[p]) {
    reps[pos[p]] = cand[vals[p]];
    if (sv.rep_seg) sv.rep_seg[pos[p]] = sv.seg[vals[p]];
  }
  if (p == count - 1) ctr->n_reps = (unsigned long long)pos[p] + flag[p];
}

// Streamed splits.  Each piece's representatives are appended to one list
// G at *g_count (read here, advanced by k_advance after the launch).
__global__ void k_compact_append(const double2* __restrict__ cand, const uint32_t* __restrict__ vals,
                                 const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                                 int64_t count, double2* __restrict__ G,
                                 const unsigned long long* __restrict__ g_count, int64_t g_cap) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count || !flag[p]) return;
  const int64_t k = (int64_t)*g_count + pos[p];
  if (k < g_cap) G[k] = cand[vals[p]];
}
__global__ void k_advance(unsigned long long* g_count, const uint32_t* __restrict__ flag,
                          const uint32_t* __restrict__ pos, int64_t count) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && count > 0)
    *g_count += (unsigned long long)pos[count - 1] + flag[count - 1];
}
// valid entries of this piece: converged descents since the last call
__global__ void k_piece_valid(const DevCounters* __restrict__ ctr, unsigned long long* snap,
                              unsigned long long* n_valid) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *n_valid = ctr->n_conv - *snap;
    *snap = ctr->n_conv;
  }
}
// the end point of every descent in 32-bit fixed point, 2^-29 per unit
// (|coordinate| <= 4, clamped beyond; INT_MIN marks a divergent descent):
// the double-double pass marks its level-line pieces from these
__device__ __forceinline__ int fix29(double x) {
  const double t = rint(x * 536870912.0);
  return t > 2147483647.0 ? 2147483647 : (t < -2147483647.0 ? -2147483647 : (int)t);
}
__global__ void k_cand_fix(const double2* __restrict__ cand, const uint8_t* __restrict__ status,
                           int64_t count, int2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double2 z = cand[i];
  const bool ok = status[i] != 1 && isfinite(z.x) && isfinite(z.y);
  out[i] = ok ? make_int2(fix29(z.x), fix29(z.y)) : make_int2((int)0x80000000, 0);
}

cudaError_t launch_stream_append(const double2* cand, const uint8_t* status, const uint32_t* vals,
                                 const uint32_t* flag, const uint32_t* pos, int64_t count, double2* G,
                                 unsigned long long* g_count, int64_t g_cap, int2* candq, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((count + 255) / 256);
  MT_COUNT_LAUNCH(2);
  k_compact_append<<<grid, 256, 0, s>>>(cand, vals, flag, pos, count, G, g_count, g_cap);
  k_advance<<<1, 32, 0, s>>>(g_count, flag, pos, count);
  if (candq) {
    MT_COUNT_LAUNCH(1);
    k_cand_fix<<<grid, 256, 0, s>>>(cand, status, count, candq);
  }
  return cudaGetLastError();
}

cudaError_t launch_piece_valid(const DevCounters* ctr, unsigned long long* snap, unsigned long long* n_valid,
                               cudaStream_t s) {
  MT_COUNT_LAUNCH(1);
  k_piece_valid<<<1, 32, 0, s>>>(ctr, snap, n_valid);
  return cudaGetLastError();
}

cudaError_t launch_compact(const double2* cand, const uint32_t* vals, const uint32_t* flag,
                           const uint32_t* pos, int64_t count, double2* reps, DevCounters* ctr,
                           cudaStream_t s, SegView sv) {
  if (count <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_compact<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(cand, vals, flag, pos, count, reps, ctr,
                                                            sv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Emission of the full list: rep u (upper half, sorted by Re) yields
// (Re, -Im), (Re, +Im) if complex, (Re, 0) if real, at position pos[u].
__global__ void k_emit(const double2* __restrict__ reps, const unsigned long long* __restrict__ n_reps,
                       int64_t cap_reps, const uint32_t* __restrict__ mult,
                       const uint32_t* __restrict__ pos, const uint8_t* __restrict__ type,
                       int mis_code, double2* __restrict__ out, uint8_t* __restrict__ is_mis,
                       int64_t cap_out, SegView sv) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= cap_reps || u >= (int64_t)*n_reps) return;
  const double2 z = reps[u];
  const int64_t p = pos[u];
  const uint16_t sg = sv.rep_seg ? sv.rep_seg[u] : 0;
  if (sv.tab) mis_code = (sv.tab[sg].kind == 1 && sv.tab[sg].n < 32) ? sv.tab[sg].n : -1;
  const uint8_t im = !type || mis_code < 0 ? 0
                     : mis_code == MIS_CODE_RAW ? type[u] : (uint8_t)(type[u] == mis_code);
  if (sv.out_seg) {
    if (p < cap_out) sv.out_seg[p] = sg;
    if (mult[u] == 2 && p + 1 < cap_out) sv.out_seg[p + 1] = sg;
  }
  if (mult[u] == 1) {
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

cudaError_t launch_emit(const double2* reps, const unsigned long long* n_reps, int64_t cap_reps,
                        const uint32_t* mult, const uint32_t* pos, const uint8_t* type,
                        int mis_code, double2* out, uint8_t* is_mis, int64_t cap_out,
                        cudaStream_t s, SegView sv) {
  if (cap_reps <= 0) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_emit<<<(unsigned)((cap_reps + 255) / 256), 256, 0, s>>>(reps, n_reps, cap_reps, mult, pos, type,
                                                            mis_code, out, is_mis, cap_out, sv);
  return cudaGetLastError();
}

// Exact ties of Re between distinct roots (rare): sort each run of equal Re
// by Im so the list follows eq. defLexi.  One thread per run start.
__global__ void k_fix_ties(double2* out, const unsigned long long* __restrict__ n_full,
                           int64_t cap_out, uint8_t* is_mis, SegView sv, double2* out_lo) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)*n_full;
  if (n > cap_out) n = cap_out;
  if (p + 1 >= n) return;
  // a run: equal Re within one polynomial
  // Re equal as binary64 values, on the integer pipe: equal bits, or both
  // zeros of either sign
  auto same = [&](int64_t a, int64_t b) {
    const long long ba = __double_as_longlong(out[a].x), bb = __double_as_longlong(out[b].x);
    return (ba == bb || ((ba | bb) << 1) == 0) && (!sv.out_seg || sv.out_seg[a] == sv.out_seg[b]);
  };
  if (p > 0 && same(p - 1, p)) return;  // not the start of a run
  if (!same(p + 1, p)) return;
  int64_t e = p + 1;
  while (e < n && same(e, p) && e - p < 4096) ++e;
  // insertion sort of [p, e) (runs are tiny): by Im, or for double-double
  // roots by the value itself (eq. defLexi): equal Re hi parts are ordered
  // by Re lo, then by Im hi and Im lo (normalised pairs: a larger hi part
  // never has a smaller value)
  auto after = [&](const double2& a, const double2& al, const double2& b, const double2& bl) {
    if (!out_lo) return a.y > b.y;
    if (al.x != bl.x) return al.x > bl.x;
    if (a.y != b.y) return a.y > b.y;
    return al.y > bl.y;
  };
  for (int64_t i = p + 1; i < e; ++i) {
    const double2 v = out[i];
    const double2 vl = out_lo ? out_lo[i] : make_double2(0.0, 0.0);
    const uint8_t m = is_mis ? is_mis[i] : 0;
    int64_t j = i - 1;
    while (j >= p && after(out[j], out_lo ? out_lo[j] : make_double2(0.0, 0.0), v, vl)) {
      out[j + 1] = out[j];
      if (out_lo) out_lo[j + 1] = out_lo[j];
      if (is_mis) is_mis[j + 1] = is_mis[j];
      --j;
    }
    out[j + 1] = v;
    if (out_lo) out_lo[j + 1] = vl;
    if (is_mis) is_mis[j + 1] = m;
  }
}

cudaError_t launch_fix_ties(double2* out, const unsigned long long* n_full, int64_t cap_out,
                            uint8_t* is_mis, cudaStream_t s, SegView sv, double2* out_lo) {
  if (cap_out <= 1) return cudaSuccess;
  MT_COUNT_LAUNCH(1);
  k_fix_ties<<<(unsigned)((cap_out + 255) / 256), 256, 0, s>>>(out, n_full, cap_out, is_mis, sv,
                                                               out_lo);
  return cudaGetLastError();
}

}  // namespace mt
