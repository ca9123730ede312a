// mt_api.cu -- host orchestration and the C ABI (include/mtsplit.h).
//
// One split = one ordered sequence of kernel launches on the caller's
// stream (Algorithm S_par of Sec. 4.2, single GPU):
//   seeds (lift)  ->  level-line walk  ->  persistent Newton descents  ->
//   fold + radix sort + cluster + compact  ->  classify  ->  certify  ->
//   emit the sorted conjugate-closed list
// followed by one device-to-host copy of the counters.  If roots are
// missing, (M, c_L) are doubled and the sequence is replayed (Sec. 4.1:
// "if some roots are missing, N can be increased").
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/mtsplit.h"
#include "mt_internal.h"

using namespace mt;

thread_local unsigned long long mt::g_launches = 0;

namespace {

thread_local std::string g_err;

mt_status fail(mt_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mt_status fail(mt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(MT_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                             \
  } while (0)

// the device's f64_key0 on the host: -0 as +0, then an order-preserving
// map of the binary64 bits to unsigned integers
uint64_t host_key0(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  if ((b << 1) == 0) b = 0;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// Bump allocator over the caller's workspace.
struct Carve {
  char* base;
  size_t off = 0, cap;
  Carve(void* b, size_t c) : base((char*)b), cap(c) {}
  template <class T>
  T* take(int64_t n) {
    const size_t bytes = align_up((size_t)(n > 0 ? n : 1) * sizeof(T));
    T* p = base ? (T*)(base + off) : nullptr;
    off += bytes;
    return p;
  }
  void* take_bytes(size_t bytes) {
    void* p = base ? (void*)(base + off) : nullptr;
    off += align_up(bytes);
    return p;
  }
};

}  // namespace

// The polynomial domain and the kernel descriptor, shared with mt_static.cu.
// The mixed walk re-takes its binary64 anchor every WALK_ANCHOR_TURNS
// turns of the phase (M sub-steps a turn).  Its binary32 perturbation then
// spans at most that many turns of the line, still resolved far below the
// sub-step's 1e-2 stop; each anchor is a binary64 orbit, which at one per
// turn made half of the walk's time.
constexpr int WALK_ANCHOR_TURNS = 1;

bool mt::valid_poly(int kind, int l, int n) {
  if (kind == 0) return n >= 1 && n <= 40;
  if (kind == 1) return l >= 2 && n >= 1 && l + n <= 41;
  if (kind == 2) return l >= 1 && n >= 1 && l + n <= 40;
  return false;
}

PolyDev mt::make_poly(int kind, int l, int n) {
  PolyDev P;
  P.kind = kind;
  P.l = l;
  P.n = n;
  if (kind == 0) {
    P.m = n;
    P.lcap = -1;
    P.log2d = n - 1;
  } else if (kind == 1) {
    P.m = l + n - 1;
    P.lcap = l - 1;
    P.log2d = l + n - 2;
  } else {  // q_{l,n} = p_{l+n} - p_l
    P.m = l + n;
    P.lcap = l;
    P.log2d = l + n - 1;
  }
  return P;
}

namespace {

struct Plan {
  PolyDev P;
  int kind;
  int prec;        // tier of this attempt (MT_FP64 or MT_MIXED)
  int walk_block;  // CUDA block size of the walk
  int64_t degree;
  double lambda0;
  int M, cL, every;
  int64_t N0, nchunks, L, S;
  double tol;
  int cap;
  double eps;
  double cert_tol;
  int shrink;
  // MT_DD: the double-double pass
  int dd;             // 1: run it when the base pass is not certified complete
  int dd_all;         // 1: every root is redone
  int raw_types = 0;  // 1: d_is_mis receives each root's type code (q_{l,n} through its factors)
  double dd_R;        // zone radius
  double dd_margin;   // chunks / main reps within dd_R + dd_margin are revisited
  double eps_dd, tol_dd, cert_tol_dd;
  int64_t dd_Ls;      // sub-steps per redone piece of the level line
  int64_t dd_npieces; // pieces of the upper half
  int64_t dd_nb;      // pieces per dd batch
  int64_t dd_zcap;    // zone candidate capacity
  int64_t dd_near_cap;
  int64_t dd_pcap;     // redone pieces the id list holds
  int64_t dd_bad_cap;  // zone centres the dd pass accepts
  // streamed split (stream_P > 1): the level line in stream_P pieces of at
  // most S_p starts; their root sets appended to a list of G_cap entries
  int64_t stream_P;
  int64_t S_p;
  int64_t G_cap;
};

constexpr int DD_MAX_BAD = 1 << 24;  // zone centres the dd pass accepts

// ---------------------------------------------------------------------------
// Autotune table: (kind, l, n, tier) -> chunk length and walk block size
// measured fastest by mt_autotune; used when the options leave them at 0.
struct TuneKey {
  int kind, l, n, prec;
  bool operator==(const TuneKey& o) const {
    return kind == o.kind && l == o.l && n == o.n && prec == o.prec;
  }
};
struct TuneKeyHash {
  size_t operator()(const TuneKey& k) const {
    return ((size_t)k.kind * 131 + (size_t)k.l) * 131 * 131 + (size_t)k.n * 131 + (size_t)k.prec;
  }
};
struct TuneVal {
  int chunk_log2, walk_block;
};
std::mutex g_tune_mu;
std::unordered_map<TuneKey, TuneVal, TuneKeyHash> g_tune;

bool tuned(int kind, int l, int n, int prec, TuneVal* v) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey{kind, l, n, prec});
  if (it == g_tune.end()) return false;
  *v = it->second;
  return true;
}

// hyperbolic: a twentieth of the minimal separation 118.4 / 4^n (Sec. 6.3.2);
// s_{l,n}: a fiftieth of the tip separation ~6.4e3 / 8^(l+n) of this family.
double raw_eps(int kind, int l, int n) {
  return (kind == 0) ? fmin(1e-9, 0.05 * 118.4 / std::ldexp(1.0, 2 * n))
                     : fmin(1e-9, 128.0 / std::ldexp(1.0, 3 * (l + n)));
}

// the binary64 pixel: never below 64 ulp(2)
double default_eps(int kind, int l, int n) {
  return fmax(raw_eps(kind, l, n), 64.0 * std::ldexp(1.0, -51));
}

bool make_plan(int kind, int l, int n, const mt_options* o, int retry, Plan* pl) {
  if (!valid_poly(kind, l, n)) return false;
  Plan p{};  // value-initialised: padding is zero, so plans compare with memcmp
  p.kind = kind;
  p.prec = MT_FP64;
  if (o && (o->prec == MT_MIXED || o->prec == MT_DD)) {
    // attempt 0 in the mixed tier; a failed attempt repeats in binary64
    if (retry == 0) p.prec = MT_MIXED;
    else retry -= 1;
  }
  p.P = make_poly(kind, l, n);
  p.degree = int64_t(1) << p.P.log2d;
  p.lambda0 = (o && o->lambda0 > 0) ? o->lambda0 : (kind == 0 ? 5.0 : 100.0);
  p.M = (o && o->M > 0) ? o->M : 8;
  p.cL = (o && o->c_L > 0) ? o->c_L : 4;
  p.M <<= retry;
  p.cL <<= retry;
  if (p.M > 64 || (p.M & (p.M - 1)) || (p.cL & (p.cL - 1)) || p.M % p.cL) return false;
  p.every = p.M / p.cL;
  const int64_t Md = (int64_t)p.M * p.degree;  // sub-steps around the whole line
  int64_t N0;
  TuneVal tv{0, 0};
  const bool have_tune = tuned(kind, kind == 0 ? 0 : l, n, p.prec, &tv);
  // one lane per chunk: 32-thread blocks spread the 2^14 - 2^17 lanes over the
  // 152 SMs more evenly than 64 (mt_autotune, p_20 / p_22 / p_24: best at 32)
  p.walk_block = (o && o->block > 0) ? o->block : (have_tune && tv.walk_block > 0 ? tv.walk_block : 32);
  if (o && o->chunk_log2 > 0) {
    N0 = Md >> o->chunk_log2;
  } else if (have_tune && tv.chunk_log2 > 0) {
    N0 = Md >> tv.chunk_log2;
  } else if (p.prec == MT_MIXED) {
    // the binary32 walk is latency-bound with one lane per chunk: 2^16 lanes
    // instead of 2^14 pay for the extra seed lifts from p_22 up (measured:
    // p_24 36.2 -> 33.8 ms, p_26 with dd zones 185 -> 172 ms), and 2^17
    // lanes (chunks of 4096 sub-steps) from p_28 up (p_28 MT_DD: walk 29.3 ->
    // 25.0 ms, the seed lift 0.6 -> 1.2 ms)
    N0 = std::min<int64_t>(int64_t(1) << 17,
                           std::max<int64_t>(Md / 128, std::min<int64_t>(int64_t(1) << 15, Md / 16)));
    N0 = std::max<int64_t>(N0, std::min<int64_t>(int64_t(1) << 18, Md >> 12));
  } else {
    // binary64: the walk already keeps the binary64 pipe busy; more chunks
    // would only add seed lifts
    N0 = std::min<int64_t>(int64_t(1) << 15, Md / 16);
  }
  // streamed split: when the upper half holds more than 2^31 starts (the
  // root-set indices are 32-bit), or when asked for
  int64_t P = (o && o->stream_pieces > 0) ? o->stream_pieces : 1;
  const int64_t S_all = (Md / 2) / p.every;
  if (!(o && o->stream_pieces > 0) && S_all > (int64_t(1) << 31))
    while ((S_all / P) > (int64_t(1) << 28)) P <<= 1;
  if (P & (P - 1)) return false;
  if (P > 1) {
    // one lane per chunk: a piece needs tens of thousands of chunks to fill
    // the GPU, so streamed splits cut the line finer
    if (!(o && o->chunk_log2 > 0)) N0 = std::min<int64_t>(int64_t(1) << 20, Md / 16);
    // automatic streaming (p_32 and up) starts in binary64: there the mixed
    // tier leaves roots its dd zones do not recover (as at p_30), and the
    // binary64 repeat would cost a second full pass
    if (!(o && o->stream_pieces > 0)) p.prec = MT_FP64;
  }
  // L must be a multiple of 'every' and N0 >= 2
  while (N0 > 2 && (Md / N0) % p.every) N0 >>= 1;
  if (N0 < 2) N0 = 2;
  if (N0 > (int64_t(1) << 20)) return false;
  if ((Md / N0) % p.every) return false;
  p.N0 = N0;
  p.nchunks = N0 / 2;
  p.L = Md / N0;
  p.S = (Md / 2) / p.every + 1;
  p.stream_P = P;
  if (P > 1) {
    if (p.nchunks % P) return false;
    p.S_p = (p.nchunks / P) * p.L / p.every + 1;
    // distinct roots of the upper half (~ deg / 2), with room for the roots
    // that several pieces reach; checked after the last piece
    p.G_cap = std::min<int64_t>(p.S, p.degree / 8 * 5 + 4096);
    if (p.S_p > (int64_t(1) << 31) || p.G_cap > (int64_t(1) << 32) - 1) return false;
  }
  const bool dd = o && o->prec == MT_DD;
  // the base pass of MT_DD runs with the binary64 settings; the user's tol
  // and cert_tol then apply to the double-double pass
  p.tol = (o && o->tol > 0 && !dd) ? o->tol : 1e-13;
  const double IN = (kind == 0) ? 1.0 : 2.6;  // Sec. 4.2
  p.cap = std::max(20, (int)std::ceil(IN * p.P.log2d));
  // q_{l,n}: descents to multiple roots contract linearly until their
  // multiplicity is recognised: twice the cap of Algorithm S_par
  if (kind == 2) p.cap *= 2;
  p.eps = (o && o->eps_dup > 0) ? o->eps_dup : default_eps(kind, l, n);
  // the step that meets tol leaves an error ~ tol^2 / (root separation); keep
  // it well inside the separation pixel so duplicates of a root always merge
  p.tol = std::min(p.tol, 0.05 * p.eps);
  p.cert_tol = (o && o->cert_tol > 0 && !dd) ? o->cert_tol : 1e-12;
  p.shrink = 2 << retry;  // iso-angle shrink steps per lifted level
  if (dd) {
    p.dd = 1;
    p.dd_all = o->dd_all ? 1 : 0;
    // a zone must hold the whole cluster binary64 cannot resolve around its
    // centre.  By -2 the roots of p_n lie ~k^2 / 4^n from -2, so the part of
    // that cluster closer than a fixed binary64 resolution grows like 4^n:
    // 1e-11 holds it at p_28 and p_29 (a third of the pieces of 1e-9) but
    // loses roots at p_32, where 1e-9 is needed; the Misiurewicz
    // polynomials keep 1e-9
    const double R0 = (kind == 0 && n <= 29) ? 1e-11 : 1e-9;
    p.dd_R = o->dd_radius > 0 ? o->dd_radius : R0;
    p.dd_margin = std::max(1e-11, 100.0 * p.eps);
    p.eps_dd = std::max(1e-28, raw_eps(kind, l, n));
    p.tol_dd = std::min(o->tol > 0 ? o->tol : 1e-26, 0.05 * p.eps_dd);
    p.cert_tol_dd = o->cert_tol > 0 ? o->cert_tol : 1e-20;
    p.dd_Ls = std::min<int64_t>(p.L, 32);
    p.dd_npieces = (Md / 2) / p.dd_Ls;
    if (p.dd_npieces > (int64_t(1) << 31)) return false;
    p.dd_nb = std::min<int64_t>(p.dd_npieces, (int64_t(1) << 20) / (p.dd_Ls / p.every));
    // zone capacities: every point in dd_all mode; otherwise 2^21 points, or
    // S / 16 from p_29 up, where the zones grow to 10^5 - 10^6 centres
    p.dd_zcap = 2 * p.S + 64;
    if (!p.dd_all) p.dd_zcap = std::min<int64_t>(p.dd_zcap, std::max<int64_t>(int64_t(1) << 21, p.S / 16));
    p.dd_near_cap = p.dd_all ? p.S : std::min<int64_t>(p.S, std::max<int64_t>(int64_t(1) << 21, p.S / 64));
    // zone centres: at most one per 256 starts (p_31: 1.2 M of 8.4 M; p_32:
    // 5.7 M of 2^24)
    p.dd_bad_cap = std::min<int64_t>(DD_MAX_BAD, std::max<int64_t>(4096, p.S / 256));
    // the ids of redone pieces: all of them in memory; streamed, a sixteenth
    p.dd_pcap = (P > 1 && !p.dd_all)
                    ? std::min<int64_t>(p.dd_npieces, std::max<int64_t>(int64_t(1) << 24, p.dd_npieces / 16))
                    : p.dd_npieces;
    if (P > 1) {  // the rep arrays of the final stage hold G_cap entries
      if (p.dd_all) return false;  // the whole streamed line in dd: not offered
      p.dd_near_cap = std::min<int64_t>(p.dd_near_cap, p.G_cap);
    }
  }
  *pl = p;
  return true;
}

// Scratch of the double-double pass (dd arrays are pairs of doubles).
struct DdBuffers {
  unsigned long long* cnt;  // [0] centres [1] polish list [2] zone points [3] zone reps
                            // [4] kept main multiplicity [5] zone multiplicity [6] main reps
  double2* bad;
  uint64_t *bad_klo, *bad_khi;  // the centres' windows of radius dd_R + dd_margin as integer keys
  uint32_t *pflag, *ppos;  // per piece of the level line: redo flag, its scan
  int64_t* pids;           // redone pieces
  void* pscan;
  uint32_t *scnt, *soff;   // seeds per piece of a batch and their scan
  void* sscan;
  dd *sx, *sy, *stx, *sty, *zcx, *zcy, *zrx, *zry;
  uint8_t *st_ok, *ztype, *zpass;
  uint32_t* near;
  uint64_t *zkeys, *zkeys_alt;
  uint32_t *zvals, *zvals_alt, *zflag, *zpos, *zmult, *zmpos;
  void *zradix, *zscan;
};

struct Buffers {
  DevCounters* ctr;
  double2 *seeds, *starts, *cand, *reps;
  uint8_t *status, *type, *pass;
  uint64_t *keys, *keys_alt;
  uint32_t *vals, *vals_alt, *flag, *pos, *mult, *mpos;
  double* radius;
  void *scan_tmp, *radix_tmp, *anchors;
  uint8_t *seed_bad, *chunk_fail;  // mixed tier: items the binary64 repairs redo
  // streamed split: the appended list, its counters (count, converged
  // snapshot, valid in the piece), the fixed-point end points of all descents
  // (for the dd pass) and the drop flags of the final reps
  double2* G;
  unsigned long long* gstate;
  int2* candq;
  int64_t candq_n;
  uint8_t* drop;
  DdBuffers d;
  size_t bytes;
};

dd* take_dd(Carve& c, int64_t n) { return reinterpret_cast<dd*>(c.take<double2>(n)); }

Buffers carve(const Plan& p, void* ws, size_t cap) {
  Carve c(ws, cap);
  Buffers b{};
  b.ctr = c.take<DevCounters>(1);
  b.seeds = c.take<double2>(p.nchunks + 1);
  if (p.stream_P > 1) {
    // one piece of the line at a time; the sort buffers also serve the final
    // root set over the appended list
    const int64_t Sp = p.S_p, Gc = p.G_cap, Mx = std::max(Sp, Gc);
    b.starts = c.take<double2>(Sp);
    b.cand = c.take<double2>(Sp);
    b.status = c.take<uint8_t>(Sp);
    b.keys = c.take<uint64_t>(Mx);
    b.keys_alt = c.take<uint64_t>(Mx);
    b.vals = c.take<uint32_t>(Mx);
    b.vals_alt = c.take<uint32_t>(Mx);
    b.flag = c.take<uint32_t>(Mx);
    b.pos = c.take<uint32_t>(Mx);
    b.mult = b.flag;
    b.mpos = b.pos;
    b.scan_tmp = c.take_bytes(scan_temp_bytes(Mx));
    b.radix_tmp = c.take_bytes(radix_temp_bytes(Mx));
    b.G = c.take<double2>(Gc);
    b.gstate = c.take<unsigned long long>(4);
    b.candq = p.dd ? c.take<int2>(p.S) : nullptr;
    b.candq_n = p.S;
    b.reps = c.take<double2>(Gc);
    b.type = c.take<uint8_t>(Mx);  // also the finish links of a mixed piece
    b.pass = c.take<uint8_t>(Gc);
    b.radius = c.take<double>(Gc);
    b.drop = c.take<uint8_t>(Gc);
    b.anchors = (p.prec == MT_MIXED) ? c.take_bytes(mixed_anchor_bytes(p.P, Sp)) : nullptr;
    b.seed_bad = (p.prec == MT_MIXED) ? c.take<uint8_t>(p.nchunks + 1) : nullptr;
    b.chunk_fail = (p.prec == MT_MIXED) ? c.take<uint8_t>(p.nchunks) : nullptr;
  } else {
    b.starts = c.take<double2>(p.S);
    b.cand = c.take<double2>(p.S);
    b.reps = b.starts;  // starts are dead once the descents are done
    b.status = c.take<uint8_t>(p.S);
    b.keys = c.take<uint64_t>(p.S);
    b.keys_alt = c.take<uint64_t>(p.S);
    b.vals = c.take<uint32_t>(p.S);
    b.vals_alt = c.take<uint32_t>(p.S);
    b.flag = c.take<uint32_t>(p.S);
    b.pos = c.take<uint32_t>(p.S);
    b.type = c.take<uint8_t>(p.S);
    b.mult = b.flag;  // flag/pos are dead after compaction
    b.mpos = b.pos;
    b.pass = c.take<uint8_t>(p.S);
    b.radius = c.take<double>(p.S);
    b.scan_tmp = c.take_bytes(scan_temp_bytes(p.S));
    b.radix_tmp = c.take_bytes(radix_temp_bytes(p.S));
    b.anchors = (p.prec == MT_MIXED) ? c.take_bytes(mixed_anchor_bytes(p.P, p.S)) : nullptr;
    b.seed_bad = (p.prec == MT_MIXED) ? c.take<uint8_t>(p.nchunks + 1) : nullptr;
    b.chunk_fail = (p.prec == MT_MIXED) ? c.take<uint8_t>(p.nchunks) : nullptr;
  }
  b.d = DdBuffers{};
  if (p.dd) {
    DdBuffers& d = b.d;
    const int64_t nst = p.dd_nb * (p.dd_Ls / p.every) + 1;
    d.cnt = c.take<unsigned long long>(8);
    d.bad = c.take<double2>(p.dd_bad_cap);
    d.bad_klo = c.take<uint64_t>(p.dd_bad_cap);
    d.bad_khi = c.take<uint64_t>(p.dd_bad_cap);
    d.pflag = c.take<uint32_t>(p.dd_npieces);
    d.ppos = c.take<uint32_t>(p.dd_npieces);
    d.pids = c.take<int64_t>(p.dd_pcap);
    d.pscan = c.take_bytes(scan_temp_bytes(p.dd_npieces));
    d.sx = take_dd(c, 2 * p.dd_nb);
    d.sy = take_dd(c, 2 * p.dd_nb);
    d.scnt = c.take<uint32_t>(p.dd_nb);
    d.soff = c.take<uint32_t>(p.dd_nb);
    d.sscan = c.take_bytes(scan_temp_bytes(p.dd_nb));
    d.stx = take_dd(c, nst);
    d.sty = take_dd(c, nst);
    d.st_ok = c.take<uint8_t>(nst);
    d.near = c.take<uint32_t>(p.dd_near_cap);
    d.zcx = take_dd(c, p.dd_zcap);
    d.zcy = take_dd(c, p.dd_zcap);
    d.zrx = take_dd(c, p.dd_zcap);
    d.zry = take_dd(c, p.dd_zcap);
    d.zkeys = c.take<uint64_t>(p.dd_zcap);
    d.zkeys_alt = c.take<uint64_t>(p.dd_zcap);
    d.zvals = c.take<uint32_t>(p.dd_zcap);
    d.zvals_alt = c.take<uint32_t>(p.dd_zcap);
    d.zflag = c.take<uint32_t>(p.dd_zcap);
    d.zpos = c.take<uint32_t>(p.dd_zcap);
    d.zmult = c.take<uint32_t>(p.dd_zcap);
    d.zmpos = c.take<uint32_t>(p.dd_zcap);
    d.ztype = c.take<uint8_t>(p.dd_zcap);
    d.zpass = c.take<uint8_t>(p.dd_zcap);
    d.zradix = c.take_bytes(radix_temp_bytes(p.dd_zcap));
    d.zscan = c.take_bytes(scan_temp_bytes(p.dd_zcap));
  }
  b.bytes = c.off;
  return b;
}

size_t plan_bytes(const Plan& p) { return carve(p, nullptr, 0).bytes; }

int max_attempts(const mt_options* o) {
  if (o && o->max_retries < 0) return 0;  // the first attempt only
  const int r = o ? std::max(0, o->max_retries) : 1;
  return (o && (o->prec == MT_MIXED || o->prec == MT_DD)) ? r + 1 : r;
}

size_t workspace_for(int kind, int l, int n, const mt_options* o) {
  const int retries = max_attempts(o);
  size_t best = 0;
  for (int r = 0; r <= retries; ++r) {
    Plan p;
    if (!make_plan(kind, l, n, o, r, &p)) {
      if (r == 0) return 0;
      break;
    }
    best = std::max(best, plan_bytes(p));
  }
  return best;
}

struct EventSet {
  cudaEvent_t e[8] = {};
  bool ok = false;
  EventSet() {
    ok = true;
    for (auto& x : e)
      if (cudaEventCreate(&x) != cudaSuccess) {
        x = nullptr;
        ok = false;
      }
  }
  ~EventSet() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
};

// Per-kernel timers (ktimer_begin / ktimer_end of mt_internal.h): event
// pairs around single launches.  A plain pass uses the thread's set, whose
// events are created on first use; a captured graph owns a set created
// before the capture, its pairs recorded as external event nodes that every
// replay re-records.  Launches beyond CAP per pass go untimed (counted).
struct KTimers {
  static constexpr int CAP = 64;
  cudaEvent_t a[CAP] = {}, b[CAP] = {};
  int slot[CAP] = {};
  int used = 0, open = -1, untimed = 0;
  bool capturing = false;
  explicit KTimers(bool eager) {
    for (int k = 0; eager && k < CAP; ++k) make(k);
  }
  ~KTimers() {
    for (int k = 0; k < CAP; ++k) {
      if (a[k]) cudaEventDestroy(a[k]);
      if (b[k]) cudaEventDestroy(b[k]);
    }
  }
  bool make(int k) {
    if (!a[k] && cudaEventCreate(&a[k]) != cudaSuccess) a[k] = nullptr;
    if (!b[k] && cudaEventCreate(&b[k]) != cudaSuccess) b[k] = nullptr;
    return a[k] && b[k];
  }
  void reset(bool cap) {
    used = 0;
    open = -1;
    untimed = 0;
    capturing = cap;
  }
  // per-slot sums in ms of the recorded pairs (after the stream synchronised)
  int sums(float* ms) const {
    for (int q = 0; q < KS_N; ++q) ms[q] = 0.f;
    for (int k = 0; k < used; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, a[k], b[k]) == cudaSuccess) ms[slot[k]] += t;
    }
    return used;
  }
};
thread_local KTimers* t_kt = nullptr;        // armed for the pass being enqueued
thread_local KTimers* t_kt_plain = nullptr;  // the thread's set for plain passes

}  // namespace

namespace mt {
cudaError_t ktimer_begin(int slot, cudaStream_t s) {
  KTimers* t = t_kt;
  if (!t) return cudaSuccess;
  t->open = -1;
  if (t->used >= KTimers::CAP || (!t->capturing && !t->make(t->used)) || !t->a[t->used]) {
    ++t->untimed;
    return cudaSuccess;
  }
  const int k = t->used++;
  t->slot[k] = slot;
  t->open = k;
  return t->capturing ? cudaEventRecordWithFlags(t->a[k], s, cudaEventRecordExternal)
                      : cudaEventRecord(t->a[k], s);
}
cudaError_t ktimer_end(cudaStream_t s) {
  KTimers* t = t_kt;
  if (!t || t->open < 0) return cudaSuccess;
  const int k = t->open;
  t->open = -1;
  return t->capturing ? cudaEventRecordWithFlags(t->b[k], s, cudaEventRecordExternal)
                      : cudaEventRecord(t->b[k], s);
}
}  // namespace mt

namespace {

void fill_stats(const Plan& p, const DevCounters& h, mt_stats* st) {
  if (!st) return;
  st->degree = p.degree;
  st->n_roots = (int64_t)h.n_full;
  st->n_real = (int64_t)h.n_reps_real;
  st->n_starts = p.S;
  st->n_conv = (int64_t)h.n_conv;
  st->n_repeat = (int64_t)h.n_conv - (int64_t)h.n_reps;
  st->n_diverge = (int64_t)h.n_diverge;
  st->n_timeout = (int64_t)h.n_timeout;
  st->walk_newton = (int64_t)h.walk_newton;
  st->desc_newton = (int64_t)h.desc_newton;
  st->steps_fp32 = (int64_t)h.steps_fp32;
  st->steps_dd = (int64_t)h.steps_dd;
  st->seed_newton = (int64_t)h.seed_newton;
  st->desc_fp32 = (int64_t)h.desc_fp32;
  st->n_finish = (int64_t)h.n_finish;
  st->n_tip64 = (int32_t)h.n_tip64;
  st->finish_newton = (int64_t)h.finish_newton;
  st->walk_fail = (int64_t)h.walk_fail;
  st->n_cert_pass = (int64_t)h.n_cert_pass;
  for (int i = 0; i < MT_MAX_TYPES; ++i) st->count_by_type[i] = (int64_t)h.type_count[i];
  st->M = p.M;
  st->c_L = p.cL;
  st->n_chunks = (int32_t)p.nchunks;
  double mn, mx;
  memcpy(&mn, &h.min_radius_bits, 8);
  memcpy(&mx, &h.max_radius_bits, 8);
  st->min_cert_radius = h.n_cert_pass ? mn : 0.0;
  st->max_cert_radius = h.n_cert_pass ? mx : 0.0;
  st->eps_dup = p.eps;
  st->prec_used = p.prec;
  st->n_mult = (p.kind == 2) ? (int64_t)h.n_mult_full : (int64_t)h.n_full;
}

// Stage boundaries are marked with events; inside a stream capture they
// are recorded as external event nodes so they still time the graph.
cudaError_t mark(cudaEvent_t e, cudaStream_t s, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// The pass's output list: representatives with their multiplicities, sorted
// (ties ordered), low parts zero.  An MT_DD pass that is not streamed emits
// after the host has seen its counters: when the double-double pass runs,
// it writes the whole list itself, so the binary64 list is only written
// when that pass does not run.
bool defer_emit(const Plan& p) { return p.dd && p.stream_P <= 1; }
mt_status emit_base(const Plan& p, const Buffers& b, double2* out, double2* out_lo, int64_t cap_out,
                    uint8_t* is_mis, cudaStream_t s) {
  const int mis_code = p.raw_types ? MIS_CODE_RAW : (p.kind == 1 && p.P.n < 32) ? p.P.n : -1;
  CK(launch_emit(b.reps, &b.ctr->n_reps, p.S, b.mult, b.mpos, b.type, mis_code, out, is_mis, cap_out,
                 s));
  CK(launch_fix_ties(out, &b.ctr->n_full, cap_out, is_mis, s));
  if (out_lo) CK(cudaMemsetAsync(out_lo, 0, (size_t)cap_out * sizeof(double2), s));
  return MT_OK;
}

// One pass of the whole sequence, enqueued on s (no host synchronisation).
mt_status enqueue_pass(const Plan& p, const Buffers& b, double2* out, double2* out_lo,
                       int64_t cap_out, uint8_t* is_mis, cudaStream_t s, EventSet& ev,
                       bool capturing) {
  CK(launch_init_counters(b.ctr, s));
  CK(mark(ev.e[0], s, capturing));
  if (p.prec == MT_MIXED) {
    CK(launch_seed_lift_mixed(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.seed_bad, b.ctr, s));
    CK(launch_mixed_repair_seeds(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.seed_bad, b.ctr, s));
  } else {
    CK(launch_seed_lift(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.ctr, s));
  }
  CK(mark(ev.e[6], s, capturing));
  if (p.prec == MT_MIXED) {
    CK(launch_walk_mixed(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, WALK_ANCHOR_TURNS * p.M, b.seeds, b.starts,
                         b.chunk_fail, b.ctr, s, p.walk_block));
    CK(launch_mixed_repair_walk(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, p.shrink, b.seeds,
                                b.starts, b.chunk_fail, b.ctr, s));
  } else {
    CK(launch_walk(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, b.seeds, b.starts, b.ctr, s,
                   p.walk_block));
  }
  CK(mark(ev.e[1], s, capturing));
  if (p.prec == MT_MIXED) {
    // the root-set buffers are free until the fold: the sort of the binary32
    // end points in keys / vals, the finish lists in flag / pos / vals_alt / type
    FinishScratch fin{b.keys, b.keys_alt, b.vals, b.vals_alt, b.flag, b.pos, b.vals_alt, b.type,
                      b.scan_tmp, b.radix_tmp, &b.ctr->n_finish};
    CK(launch_descend_mixed(p.P, b.starts, p.S, p.tol, p.cap, b.cand, b.status, b.anchors, fin, b.ctr, s));
  } else {
    CK(launch_descend(p.P, b.starts, p.S, p.tol, p.cap, b.cand, b.status, b.ctr, 0, s));
  }
  CK(mark(ev.e[2], s, capturing));
  if (p.prec == MT_MIXED) {
    // the root set of the finished group heads only: every follower holds
    // its head's root (the list of heads is still in vals_alt)
    CK(launch_fold_keys_list(b.vals_alt, &b.ctr->n_finish, p.S, b.status, b.cand, p.eps, b.keys, b.vals,
                             &b.ctr->n_heads_conv, s));
    CK(radix_sort_pairs(b.keys, b.vals, b.keys_alt, b.vals_alt, p.S, b.radix_tmp, s, &b.ctr->n_finish));
    CK(launch_cluster(b.cand, b.vals, p.S, &b.ctr->n_heads_conv, p.eps, b.flag, b.ctr, s));
  } else {
    CK(launch_fold_keys(b.status, b.cand, p.S, p.eps, b.keys, b.vals, s));
    CK(radix_sort_pairs(b.keys, b.vals, b.keys_alt, b.vals_alt, p.S, b.radix_tmp, s));
    CK(launch_cluster(b.cand, b.vals, p.S, &b.ctr->n_conv, p.eps, b.flag, b.ctr, s));
  }
  CK(launch_exclusive_scan(b.flag, b.pos, p.S, b.scan_tmp, nullptr, s));
  CK(launch_compact(b.cand, b.vals, b.flag, b.pos, p.S, b.reps, b.ctr, s));
  CK(mark(ev.e[3], s, capturing));
  if (p.kind == 0) {  // types from the certificate's own orbit
    CK(launch_certify_typed(p.P, b.reps, &b.ctr->n_reps, p.S, p.cert_tol, p.eps, b.type, b.mult, b.pass,
                            b.radius, b.ctr, s));
    CK(launch_exclusive_scan(b.mult, b.mpos, p.S, b.scan_tmp, &b.ctr->n_full, s));
  } else {
    CK(launch_classify(p.P, b.reps, &b.ctr->n_reps, p.S, p.eps, 0, b.type, b.mult, b.ctr, s));
    CK(launch_exclusive_scan(b.mult, b.mpos, p.S, b.scan_tmp, &b.ctr->n_full, s));
    CK(launch_certify(p.P, b.reps, &b.ctr->n_reps, p.S, p.cert_tol, b.mult, b.pass, b.radius, b.ctr,
                      s, SegView(), p.kind == 2 ? b.type : nullptr));
  }
  CK(mark(ev.e[4], s, capturing));
  if (!defer_emit(p)) {
    const mt_status rc = emit_base(p, b, out, out_lo, cap_out, is_mis, s);
    if (rc != MT_OK) return rc;
  }
  CK(mark(ev.e[5], s, capturing));
  return MT_OK;
}

mt_status read_counters(const Buffers& b, DevCounters* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h, b.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return MT_OK;
}

// Streamed split (stream_P > 1).  The level line is walked and descended a
// range of chunks at a time; each piece's candidates get their own root set
// (fold, sort, cluster), whose representatives are appended to the list G.
// The root set of G -- the same clustering rule over fewer points, roots
// reached from several pieces merging there -- is the split's, and is typed,
// certified and emitted as in one pass.  Stage times are summed over the
// pieces (*tm: walk, descents, piece root sets).
struct StreamTimes {
  float walk = 0.f, descend = 0.f, dedup = 0.f;
};

mt_status run_streamed(const Plan& p, const Buffers& b, double2* out, double2* out_lo, int64_t cap_out,
                       uint8_t* is_mis, cudaStream_t s, EventSet& ev, DevCounters* h, StreamTimes* tm) {
  unsigned long long* gcount = b.gstate;      // entries of G
  unsigned long long* snap = b.gstate + 1;    // converged descents before this piece
  unsigned long long* nvalid = b.gstate + 2;  // converged descents of this piece
  CK(launch_init_counters(b.ctr, s));
  CK(cudaMemsetAsync(b.gstate, 0, 4 * sizeof(unsigned long long), s));
  CK(cudaEventRecord(ev.e[0], s));
  const bool mixed = p.prec == MT_MIXED;
  if (mixed) {
    CK(launch_seed_lift_mixed(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.seed_bad, b.ctr, s));
    CK(launch_mixed_repair_seeds(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.seed_bad, b.ctr, s));
  } else {
    CK(launch_seed_lift(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.ctr, s));
  }
  CK(cudaEventRecord(ev.e[6], s));
  const int64_t C = p.nchunks / p.stream_P;
  std::vector<cudaEvent_t> pe((size_t)(4 * p.stream_P), nullptr);
  struct Guard {
    std::vector<cudaEvent_t>& v;
    ~Guard() {
      for (auto e : v)
        if (e) cudaEventDestroy(e);
    }
  } guard{pe};
  for (auto& e : pe) CK(cudaEventCreate(&e));
  for (int64_t k = 0; k < p.stream_P; ++k) {
    const int64_t j0 = k * C;
    const int64_t Sk = C * p.L / p.every + (k == p.stream_P - 1 ? 1 : 0);
    CK(cudaEventRecord(pe[4 * k], s));
    if (mixed) {
      CK(launch_walk_mixed(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, WALK_ANCHOR_TURNS * p.M, b.seeds, b.starts, b.chunk_fail,
                           b.ctr, s, p.walk_block, j0, C));
      CK(launch_mixed_repair_walk(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, p.shrink, b.seeds, b.starts,
                                  b.chunk_fail, b.ctr, s, j0, C));
    } else {
      CK(launch_walk_range(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, j0, C, b.seeds, b.starts, b.ctr, s,
                           p.walk_block));
    }
    CK(cudaEventRecord(pe[4 * k + 1], s));
    CK(cudaMemsetAsync(&b.ctr->queue_head, 0, sizeof(unsigned long long), s));
    if (mixed) {
      // the sort buffers are free until the fold: the sort of the binary32
      // end points in keys / vals, the finish lists in flag / pos / vals_alt / type
      FinishScratch fin{b.keys, b.keys_alt, b.vals, b.vals_alt, b.flag, b.pos, b.vals_alt, b.type,
                        b.scan_tmp, b.radix_tmp, &b.ctr->n_finish};
      CK(launch_descend_mixed(p.P, b.starts, Sk, p.tol, p.cap, b.cand, b.status, b.anchors, fin, b.ctr, s));
    } else {
      CK(launch_descend(p.P, b.starts, Sk, p.tol, p.cap, b.cand, b.status, b.ctr, 0, s));
    }
    CK(cudaEventRecord(pe[4 * k + 2], s));
    CK(launch_piece_valid(b.ctr, snap, nvalid, s));
    CK(launch_fold_keys(b.status, b.cand, Sk, p.eps, b.keys, b.vals, s));
    CK(radix_sort_pairs(b.keys, b.vals, b.keys_alt, b.vals_alt, Sk, b.radix_tmp, s));
    CK(launch_cluster(b.cand, b.vals, Sk, nvalid, p.eps, b.flag, b.ctr, s));
    CK(launch_exclusive_scan(b.flag, b.pos, Sk, b.scan_tmp, nullptr, s));
    CK(launch_stream_append(b.cand, b.status, b.vals, b.flag, b.pos, Sk, b.G, gcount, p.G_cap,
                            b.candq ? b.candq + j0 * p.L / p.every : nullptr, s));
    CK(cudaEventRecord(pe[4 * k + 3], s));
  }
  CK(cudaEventRecord(ev.e[1], s));
  CK(cudaEventRecord(ev.e[2], s));
  unsigned long long ng = 0;
  CK(cudaMemcpyAsync(&ng, gcount, sizeof(ng), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int64_t k = 0; k < p.stream_P; ++k) {
    float a = 0.f, c = 0.f, d = 0.f;
    cudaEventElapsedTime(&a, pe[4 * k], pe[4 * k + 1]);
    cudaEventElapsedTime(&c, pe[4 * k + 1], pe[4 * k + 2]);
    cudaEventElapsedTime(&d, pe[4 * k + 2], pe[4 * k + 3]);
    tm->walk += a;
    tm->descend += c;
    tm->dedup += d;
  }
  if ((int64_t)ng > p.G_cap)
    return fail(MT_ECAPACITY, "the pieces of the streamed split found %llu representatives, the list holds %lld",
                ng, (long long)p.G_cap);
  const int64_t nG = (int64_t)ng;
  // the root set of G (its points are folded already)
  CK(launch_keys_plain(b.G, nG, b.keys, b.vals, s));
  CK(radix_sort_pairs(b.keys, b.vals, b.keys_alt, b.vals_alt, nG, b.radix_tmp, s));
  CK(launch_cluster(b.G, b.vals, nG, gcount, p.eps, b.flag, b.ctr, s));
  CK(launch_exclusive_scan(b.flag, b.pos, nG, b.scan_tmp, nullptr, s));
  CK(launch_compact(b.G, b.vals, b.flag, b.pos, nG, b.reps, b.ctr, s));
  CK(cudaEventRecord(ev.e[3], s));
  CK(launch_classify(p.P, b.reps, &b.ctr->n_reps, nG, p.eps, 0, b.type, b.mult, b.ctr, s));
  CK(launch_exclusive_scan(b.mult, b.mpos, nG, b.scan_tmp, &b.ctr->n_full, s));
  CK(launch_certify(p.P, b.reps, &b.ctr->n_reps, nG, p.cert_tol, b.mult, b.pass, b.radius, b.ctr, s,
                    SegView(), p.kind == 2 ? b.type : nullptr));
  CK(cudaEventRecord(ev.e[4], s));
  const int mis_code = p.raw_types ? MIS_CODE_RAW : (p.kind == 1 && p.P.n < 32) ? p.P.n : -1;
  CK(launch_emit(b.reps, &b.ctr->n_reps, nG, b.mult, b.mpos, b.type, mis_code, out, is_mis, cap_out, s));
  CK(launch_fix_ties(out, &b.ctr->n_full, cap_out, is_mis, s));
  if (out_lo) CK(cudaMemsetAsync(out_lo, 0, (size_t)cap_out * sizeof(double2), s));
  CK(cudaEventRecord(ev.e[5], s));
  return read_counters(b, h, s);
}

mt_status run_pass(const Plan& p, const Buffers& b, double2* out, double2* out_lo, int64_t cap_out,
                   uint8_t* is_mis, cudaStream_t s, EventSet& ev, DevCounters* h, KTimers** kt_out) {
  if (!t_kt_plain) t_kt_plain = new KTimers(false);
  t_kt_plain->reset(false);
  t_kt = t_kt_plain;
  mt_status rc = enqueue_pass(p, b, out, out_lo, cap_out, is_mis, s, ev, false);
  t_kt = nullptr;
  if (rc != MT_OK) return rc;
  *kt_out = t_kt_plain;
  return read_counters(b, h, s);
}

// ---------------------------------------------------------------------------
// CUDA-graph cache (mt_options.use_graph): the launch sequence of a pass is
// captured once per (plan, buffers) and replayed.  Capture runs on a stream
// of the library (the legacy default stream cannot capture), joined to the
// caller's stream with events.
struct GraphEntry {
  Plan p;
  void *work, *out, *out_lo, *is_mis;
  int64_t cap;
  int device;
  cudaGraphExec_t exec = nullptr;
  EventSet* ev = nullptr;
  KTimers* kt = nullptr;
  unsigned long long launches = 0;  // kernels in the graph
};
thread_local std::vector<GraphEntry> t_graphs;
thread_local cudaStream_t t_gstream = nullptr;
thread_local EventSet* t_join = nullptr;

bool same_plan(const Plan& a, const Plan& b) { return memcmp(&a, &b, sizeof(Plan)) == 0; }

mt_status run_pass_graph(const Plan& p, const Buffers& b, void* work, double2* out, double2* out_lo,
                         int64_t cap_out, uint8_t* is_mis, cudaStream_t s, DevCounters* h,
                         EventSet** ev_out, KTimers** kt_out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (!t_gstream) CK(cudaStreamCreateWithFlags(&t_gstream, cudaStreamNonBlocking));
  if (!t_join) t_join = new EventSet();
  GraphEntry* g = nullptr;
  for (auto& e : t_graphs)
    if (e.device == dev && e.work == work && e.out == out && e.out_lo == out_lo &&
        e.is_mis == is_mis && e.cap == cap_out && same_plan(e.p, p))
      g = &e;
  if (!g) {
    if (t_graphs.size() >= 8) {  // bounded cache: drop the oldest
      cudaGraphExecDestroy(t_graphs.front().exec);
      delete t_graphs.front().ev;
      delete t_graphs.front().kt;
      t_graphs.erase(t_graphs.begin());
    }
    GraphEntry e;
    e.p = p;
    e.work = work;
    e.out = out;
    e.out_lo = out_lo;
    e.is_mis = is_mis;
    e.cap = cap_out;
    e.device = dev;
    e.ev = new EventSet();
    e.kt = new KTimers(true);
    e.kt->reset(true);
    CK(cudaStreamBeginCapture(t_gstream, cudaStreamCaptureModeThreadLocal));
    const unsigned long long l0 = g_launches;
    t_kt = e.kt;
    mt_status rc = enqueue_pass(p, b, out, out_lo, cap_out, is_mis, t_gstream, *e.ev, true);
    t_kt = nullptr;
    e.launches = g_launches - l0;
    g_launches = l0;  // counted when the graph runs
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(t_gstream, &graph);
    if (rc != MT_OK) {
      if (graph) cudaGraphDestroy(graph);
      delete e.ev;
      delete e.kt;
      return rc;
    }
    if (ce != cudaSuccess) {
      delete e.ev;
      delete e.kt;
      return fail(MT_ECUDA, "stream capture failed: %s", cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      delete e.ev;
      delete e.kt;
      return fail(MT_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    t_graphs.push_back(e);
    g = &t_graphs.back();
  }
  CK(cudaEventRecord(t_join->e[0], s));  // the graph runs after the caller's prior work
  CK(cudaStreamWaitEvent(t_gstream, t_join->e[0], 0));
  CK(cudaGraphLaunch(g->exec, t_gstream));
  g_launches += g->launches;
  CK(cudaEventRecord(t_join->e[1], t_gstream));
  CK(cudaStreamWaitEvent(s, t_join->e[1], 0));  // and the caller's later work after the graph
  *ev_out = g->ev;
  *kt_out = g->kt;
  return read_counters(b, h, s);
}

// ---------------------------------------------------------------------------
// The double-double pass (MT_DD) after a base pass whose result is not
// certified complete; see mt_ddtier.cu for the method.  Host decisions
// (zone centres sorted by Re, the list of chunks to redo) need a few small
// synchronous copies; the bulk stays on the device.
struct DdReport {
  int64_t zones = 0, zone_roots = 0, pieces = 0;
  float ms = 0.f;
};

mt_status run_dd(const Plan& p, const Buffers& b, double2* out, double2* out_lo, int64_t cap_out,
                 uint8_t* is_mis, cudaStream_t s, DevCounters* h, DdReport* rep) {
  const DdBuffers& d = b.d;
  EventSet ev;
  if (!ev.ok) return fail(MT_ECUDA, "cudaEventCreate failed");
  CK(cudaEventRecord(ev.e[0], s));
  CK(cudaMemsetAsync(d.cnt, 0, 8 * sizeof(unsigned long long), s));
  CK(cudaMemcpyAsync(&d.cnt[6], &b.ctr->n_reps, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  const unsigned long long* n_main = &d.cnt[6];
  int nbad = -1;  // "all" mode
  if (!p.dd_all) {
    CK(dd_collect_bad(b.reps, n_main, p.S, b.pass, b.radius, 2.0 * p.eps, d.bad, &d.cnt[0], (int)p.dd_bad_cap,
                      s));
    unsigned long long nb_h = 0;
    CK(cudaMemcpyAsync(&nb_h, &d.cnt[0], sizeof(nb_h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nb_h > (unsigned long long)p.dd_bad_cap)
      return fail(MT_ECERT, "%llu roots need the double-double pass, more than its %lld zones",
                  nb_h, (long long)p.dd_bad_cap);
    nbad = (int)nb_h;
    rep->zones = nbad;
    if (nbad == 0) return MT_OK;  // nothing the dd pass can improve
    std::vector<double2> hb((size_t)nbad);
    CK(cudaMemcpyAsync(hb.data(), d.bad, sizeof(double2) * nbad, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::sort(hb.begin(), hb.end(), [](const double2& a, const double2& c) { return a.x < c.x; });
    // the windows [x_f - R', x_f + R'] of the bulk zone tests (R' = Rm (1 + 2^-30), rounded outward)
    const double Rw = (p.dd_R + p.dd_margin) * (1.0 + std::ldexp(1.0, -30));
    std::vector<uint64_t> klo((size_t)nbad), khi((size_t)nbad);
    for (int f = 0; f < nbad; ++f) {
      klo[(size_t)f] = host_key0(std::nextafter(hb[(size_t)f].x - Rw, -INFINITY));
      khi[(size_t)f] = host_key0(std::nextafter(hb[(size_t)f].x + Rw, INFINITY));
    }
    CK(cudaMemcpyAsync(d.bad, hb.data(), sizeof(double2) * nbad, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d.bad_klo, klo.data(), sizeof(uint64_t) * nbad, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d.bad_khi, khi.data(), sizeof(uint64_t) * nbad, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  const double Rm = p.dd_R + p.dd_margin;
  // pieces of the level line to redo
  int64_t npieces = p.dd_npieces;
  if (p.dd_all) {
    CK(dd_piece_ids(nullptr, nullptr, p.dd_npieces, d.pids, p.dd_pcap, s));
  } else {
    CK(cudaMemsetAsync(d.pflag, 0, sizeof(uint32_t) * (size_t)p.dd_npieces, s));
    if (b.candq)  // streamed split: from the fixed-point end points of all descents
      CK(dd_mark_pieces_fix(b.candq, b.candq_n, p.every, p.dd_Ls, p.dd_npieces, d.bad, nbad, Rm, d.pflag, s));
    else
      CK(dd_mark_pieces(b.cand, b.status, p.S, p.every, p.dd_Ls, p.dd_npieces, d.bad, d.bad_klo, d.bad_khi,
                        nbad, Rm, d.pflag, s));
    CK(launch_exclusive_scan(d.pflag, d.ppos, p.dd_npieces, d.pscan, &d.cnt[7], s));
    CK(dd_piece_ids(d.pflag, d.ppos, p.dd_npieces, d.pids, p.dd_pcap, s));
    unsigned long long np_h = 0;
    CK(cudaMemcpyAsync(&np_h, &d.cnt[7], sizeof(np_h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((int64_t)np_h > p.dd_pcap)
      return fail(MT_EINCOMPLETE, "%llu level-line pieces to redo in double-double, more than the %lld held",
                  np_h, (long long)p.dd_pcap);
    npieces = (int64_t)np_h;
  }
  rep->pieces = npieces;
  // b.status is dead from here on: it becomes the drop flag of the main reps
  // (a streamed split has its own, sized for the final reps)
  uint8_t* drop = b.drop ? b.drop : b.status;
  CK(cudaMemsetAsync(drop, 0, (size_t)p.S, s));
  CK(dd_near_reps(b.reps, n_main, p.S, d.bad, d.bad_klo, d.bad_khi, nbad, Rm, d.near, &d.cnt[1], p.dd_near_cap,
                  s));
  // dd level line and descents, dd_nb pieces at a time
  const int64_t per_piece = p.dd_Ls / p.every;
  for (int64_t k0 = 0; k0 < npieces; k0 += p.dd_nb) {
    const int64_t nb = std::min<int64_t>(p.dd_nb, npieces - k0);
    const int64_t nst = nb * per_piece + 1;
    CK(cudaMemsetAsync(d.st_ok, 0, (size_t)nst, s));
    CK(dd_seeds(p.P, p.lambda0, 2 * p.dd_npieces, p.shrink, d.pids + k0, nb, d.scnt, d.soff, d.sscan,
                d.sx, d.sy, b.ctr, s));
    CK(dd_walk(p.P, p.lambda0, p.M, p.every, p.dd_Ls, p.dd_npieces, d.pids + k0, d.soff, nb, d.sx, d.sy,
               d.stx, d.sty, d.st_ok, b.ctr, s));
    CK(dd_descend(p.P, nst, d.stx, d.sty, d.st_ok, p.tol_dd, p.cap + 4, d.bad, nbad, p.dd_R, d.zcx,
                  d.zcy, &d.cnt[2], p.dd_zcap, b.ctr, s));
  }
  CK(dd_polish(p.P, b.reps, d.near, &d.cnt[1], p.dd_near_cap, p.dd_near_cap, p.tol_dd, d.bad, nbad,
               p.dd_R, p.dd_margin, drop, d.zcx, d.zcy, &d.cnt[2], p.dd_zcap, b.ctr, s));
  unsigned long long c_h[8];
  CK(cudaMemcpyAsync(c_h, d.cnt, sizeof(c_h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (c_h[1] > (unsigned long long)p.dd_near_cap || c_h[2] > (unsigned long long)p.dd_zcap)
    return fail(MT_EINCOMPLETE, "double-double zones too large (%llu polished, %llu zone points)",
                c_h[1], c_h[2]);
  // the zone's root set
  CK(dd_keys(d.zcx, d.zcy, &d.cnt[2], p.dd_zcap, p.eps_dd, d.zkeys, d.zvals, s));
  CK(radix_sort_pairs(d.zkeys, d.zvals, d.zkeys_alt, d.zvals_alt, p.dd_zcap, d.zradix, s, &d.cnt[2]));
  CK(dd_cluster(d.zcx, d.zcy, d.zvals, &d.cnt[2], p.dd_zcap, p.eps_dd, d.zflag, s));
  CK(launch_exclusive_scan(d.zflag, d.zpos, p.dd_zcap, d.zscan, &d.cnt[3], s));
  CK(dd_compact(d.zcx, d.zcy, d.zvals, d.zflag, d.zpos, p.dd_zcap, d.zrx, d.zry, s));
  CK(dd_type_cert(p.P, d.zrx, d.zry, &d.cnt[3], p.eps_dd, p.cert_tol_dd, b.reps, n_main, drop,
                  b.radius, p.cert_tol, d.ztype, d.zpass, d.zmult, p.dd_zcap, b.ctr, s));
  // merge with the kept main representatives and emit
  uint32_t* kmult = b.vals;  // dead after the base pass
  uint32_t* mpos = b.pos;
  CK(dd_keep(n_main, p.S, b.mult, drop, b.type, b.pass, kmult, b.ctr, s));
  CK(launch_exclusive_scan(kmult, mpos, p.S, b.scan_tmp, &d.cnt[4], s));
  CK(launch_exclusive_scan(d.zmult, d.zmpos, p.dd_zcap, d.zscan, &d.cnt[5], s));
  if (out_lo) CK(cudaMemsetAsync(out_lo, 0, (size_t)cap_out * sizeof(double2), s));
  const int mis_code = p.raw_types ? MIS_CODE_RAW : (p.kind == 1 && p.P.n < 32) ? p.P.n : -1;
  CK(dd_emit(b.reps, n_main, p.S, kmult, mpos, &d.cnt[4], b.type, mis_code, d.zrx, d.zry, &d.cnt[3],
             p.dd_zcap, d.zmult, d.zmpos, &d.cnt[5], d.ztype, out, out_lo, is_mis, cap_out, b.ctr, s));
  CK(launch_fix_ties(out, &b.ctr->n_full, cap_out, is_mis, s, SegView(), out_lo));
  CK(cudaEventRecord(ev.e[1], s));
  CK(cudaMemcpyAsync(c_h, d.cnt, sizeof(c_h), cudaMemcpyDeviceToHost, s));
  mt_status rc = read_counters(b, h, s);
  if (rc != MT_OK) return rc;
  rep->zone_roots = (int64_t)c_h[3];
  cudaEventElapsedTime(&rep->ms, ev.e[0], ev.e[1]);
  return MT_OK;
}

mt_status split_impl(int kind, int l, int n, const mt_options* o, double* d_roots,
                     double* d_roots_lo, int64_t cap, uint8_t* d_is_mis, void* d_work,
                     size_t work_bytes, int64_t* n_out, mt_stats* st, int raw_types = 0) {
  g_err.clear();
  if (!valid_poly(kind, l, n)) return fail(MT_EINVAL, "polynomial out of range (kind %d, l %d, n %d)", kind, l, n);
  if (cap < 0 || (cap > 0 && !d_roots)) return fail(MT_EINVAL, "bad output buffer");
  if (o && o->prec != MT_FP64 && o->prec != MT_MIXED && o->prec != MT_DD)
    return fail(MT_EINVAL, "unknown precision %d", o->prec);
  mt_options dflt;
  mt_default_options(&dflt);
  if (!o) o = &dflt;
  const size_t need = workspace_for(kind, l, n, o);
  if (need == 0) return fail(MT_EINVAL, "invalid options for this polynomial");
  if (!d_work || work_bytes < need)
    return fail(MT_ENOMEM, "workspace of %zu bytes needed, %zu given", need, work_bytes);
  if (((uintptr_t)d_work) % ALIGN) return fail(MT_EINVAL, "workspace must be 256-byte aligned");
  cudaStream_t s = (cudaStream_t)o->stream;
  EventSet ev;
  if (!ev.ok) return fail(MT_ECUDA, "cudaEventCreate failed");
  DevCounters h;
  Plan p;
  mt_status rc = MT_OK;
  int retry = 0;
  const unsigned long long launches0 = g_launches;
  const int max_retries = max_attempts(o);
  // a first attempt that could not run in the mixed tier (q_{l,n}, which is
  // binary64 only) was binary64 already: its binary64 repeat is skipped
  bool skip_repeat = false;
  if (o->prec == MT_MIXED || o->prec == MT_DD) {
    Plan p0;
    skip_repeat = make_plan(kind, l, n, o, 0, &p0) && p0.prec != MT_MIXED;
  }
  EventSet* evp = &ev;
  KTimers* ktp = nullptr;
  struct {
    int64_t n_roots = 0, n_cert = 0;
    int32_t walk_fail = 0, prec = 0;
  } first;
  DdReport ddr;
  StreamTimes stimes;
  bool dd_ran = false;
  for (;; ++retry) {
    if (skip_repeat && retry == 1) {
      if (retry >= max_retries) break;
      continue;
    }
    if (!make_plan(kind, l, n, o, retry, &p)) {
      if (retry == 0) return fail(MT_EINVAL, "no plan for this polynomial and these options");
      --retry;  // (M, c_L) cannot double further: the last attempt's result stands
      break;
    }
    p.raw_types = raw_types;
    Buffers b = carve(p, d_work, work_bytes);
    evp = &ev;
    ktp = nullptr;
    stimes = StreamTimes();
    if (p.stream_P > 1)
      rc = run_streamed(p, b, (double2*)d_roots, (double2*)d_roots_lo, cap, d_is_mis, s, ev, &h, &stimes);
    else if (o->use_graph && retry == 0)
      rc = run_pass_graph(p, b, d_work, (double2*)d_roots, (double2*)d_roots_lo, cap, d_is_mis, s, &h,
                          &evp, &ktp);
    else
      rc = run_pass(p, b, (double2*)d_roots, (double2*)d_roots_lo, cap, d_is_mis, s, ev, &h, &ktp);
    if (rc != MT_OK) return rc;
    // retry on missing roots or on a level-line chunk that skipped a turn
    // (q_{l,n}: the roots counted with their multiplicities, Thm fact_mis)
    const int64_t counted = (kind == 2) ? (int64_t)h.n_mult_full : (int64_t)h.n_full;
    bool done = counted == p.degree && h.walk_fail == 0;
    const bool certified = counted == p.degree && h.n_cert_pass == h.n_full;
    dd_ran = false;
    if (p.dd && (p.dd_all || !certified)) {
      // MT_DD: a certified complete list is the goal (it proves itself)
      ddr = DdReport();
      Plan pd = p;
      if (p.stream_P > 1) pd.S = p.G_cap;  // the final reps of a streamed split
      rc = run_dd(pd, b, (double2*)d_roots, (double2*)d_roots_lo, cap, d_is_mis, s, &h, &ddr);
      if (rc != MT_OK) return rc;
      dd_ran = true;
      done = (int64_t)h.n_full == p.degree && h.n_cert_pass == h.n_full;
    } else if (p.dd) {
      done = certified;
    }
    if (defer_emit(p) && !dd_ran) {
      rc = emit_base(p, b, (double2*)d_roots, (double2*)d_roots_lo, cap, d_is_mis, s);
      if (rc != MT_OK) return rc;
      const cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return fail(MT_ECUDA, "emit: %s", cudaGetErrorString(e));
    }
    if (retry == 0) {  // kept for the statistics: why a repeat followed
      first.n_roots = (int64_t)h.n_full;
      first.n_cert = (int64_t)h.n_cert_pass;
      first.walk_fail = (int32_t)h.walk_fail;
      first.prec = dd_ran ? MT_DD : p.prec;
    }
    if (done || retry >= max_retries) break;
  }
  if (st) {
    memset(st, 0, sizeof(*st));
    fill_stats(p, h, st);
    st->retries = retry;
    st->n_launches = (int64_t)(g_launches - launches0);
    float ms[5] = {0, 0, 0, 0, 0};
    cudaEventElapsedTime(&ms[0], evp->e[0], evp->e[5]);
    cudaEventElapsedTime(&ms[1], evp->e[0], evp->e[1]);
    cudaEventElapsedTime(&ms[2], evp->e[1], evp->e[2]);
    cudaEventElapsedTime(&ms[3], evp->e[2], evp->e[3]);
    cudaEventElapsedTime(&ms[4], evp->e[3], evp->e[4]);
    st->ms_total = ms[0];
    st->ms_walk = ms[1];
    st->ms_descend = ms[2];
    st->ms_dedup = ms[3];
    st->ms_certify = ms[4];
    cudaEventElapsedTime(&st->ms_seeds, evp->e[0], evp->e[6]);
    st->first_n_roots = first.n_roots;
    st->first_n_cert_pass = first.n_cert;
    st->first_walk_fail = first.walk_fail;
    st->first_prec = first.prec;
    if (ktp) {
      float kms[KS_N];
      st->n_k_timed = ktp->sums(kms);
      st->ms_k_walk = kms[KS_WALK];
      st->ms_k_desc64 = kms[KS_DESC64];
      st->ms_k_desc32 = kms[KS_DESC32];
      st->ms_k_finish = kms[KS_FINISH];
    }
    if (p.stream_P > 1) {  // summed over the pieces; the piece root sets count as dedup
      st->ms_walk = st->ms_seeds + stimes.walk;
      st->ms_descend = stimes.descend;
      st->ms_dedup += stimes.dedup;
    }
    if (dd_ran) {
      st->prec_used = MT_DD;
      st->ms_dd = ddr.ms;
      st->ms_total += ddr.ms;
      st->n_zones = ddr.zones;
      st->n_zone_roots = ddr.zone_roots;
      st->n_dd_pieces = ddr.pieces;
    }
  }
  if (n_out) *n_out = (int64_t)h.n_full;
  const int64_t counted = (kind == 2) ? (int64_t)h.n_mult_full : (int64_t)h.n_full;
  // a bounded scan of the root set or of the certificate's neighbour search
  // that stopped at its cap may have kept a duplicate or missed a neighbour;
  // a count that still matches with every root certified is proven anyway
  // (Thm certif), so the cap is reported only where the result falls short
  if (h.cluster_overflow && (counted != p.degree || h.n_cert_pass != h.n_full))
    return fail(MT_ETIMEOUT, "%llu bounded scans of the root set hit their cap; %lld roots found, degree %lld",
                h.cluster_overflow, (long long)counted, (long long)p.degree);
  if (counted != p.degree)
    return fail(MT_EINCOMPLETE, "found %lld roots%s, degree %lld (after %d retries)", (long long)counted,
                kind == 2 ? " with multiplicity" : "", (long long)p.degree, retry);
  if ((int64_t)h.n_full > cap)
    return fail(MT_ECAPACITY, "%lld roots do not fit in cap %lld", (long long)h.n_full,
                (long long)cap);
  if (h.n_cert_pass != h.n_full)
    return fail(MT_ECERT, "%lld of %lld roots certified", (long long)h.n_cert_pass,
                (long long)h.n_full);
  return MT_OK;
}

// ---------------------------------------------------------------------------
// Batched split of every s_{l,n} with l >= 2, n >= 1, l + n <= max_order.
struct BatchPlan {
  int np = 0;
  std::vector<BatchEntry> E;
  std::vector<PolyDev> polys;
  std::vector<int64_t> seed_off, chunk_off, start_off, deg;
  int64_t seeds_total = 0, chunks_total = 0, S = 0, deg_total = 0;
  double lambda0 = 100.0, eps = 0.0, tol = 0.0, cert_tol = 0.0;
  int M = 8, cL = 4, every = 2, shrink = 2;
};

bool make_batch_plan(int max_order, const mt_options* o, int retry, BatchPlan* bp) {
  if (max_order < 3 || max_order > 41) return false;
  BatchPlan b;
  b.M = ((o && o->M > 0) ? o->M : 8) << retry;
  b.cL = ((o && o->c_L > 0) ? o->c_L : 4) << retry;
  if (b.M > 64 || (b.M & (b.M - 1)) || (b.cL & (b.cL - 1)) || b.M % b.cL) return false;
  b.every = b.M / b.cL;
  b.shrink = 2 << retry;
  b.lambda0 = (o && o->lambda0 > 0) ? o->lambda0 : 100.0;
  b.eps = 1.0;
  for (int l = 2; l < max_order; ++l)
    for (int n = 1; l + n <= max_order; ++n) b.eps = std::min(b.eps, default_eps(1, l, n));
  if (o && o->eps_dup > 0) b.eps = o->eps_dup;
  b.tol = std::min((o && o->tol > 0) ? o->tol : 1e-13, 0.05 * b.eps);
  b.cert_tol = (o && o->cert_tol > 0) ? o->cert_tol : 1e-12;
  for (int l = 2; l < max_order; ++l)
    for (int n = 1; l + n <= max_order; ++n) {
      BatchEntry e;
      e.P = make_poly(1, l, n);
      const int64_t d = int64_t(1) << e.P.log2d;
      const int64_t Md = (int64_t)b.M * d;
      // chunks of 32 sub-steps, 64 from degree 4096 up (fewer seed lifts where
      // lanes are plentiful; measured on l + n <= 16: 8.8 -> 7.4 ms)
      int64_t N0 = std::max<int64_t>(2, Md / (d >= 4096 ? 64 : 32));
      while (N0 > 2 && (Md / N0) % b.every) N0 >>= 1;
      if ((Md / N0) % b.every) return false;
      e.N0 = N0;
      e.log2N0 = 0;
      while ((int64_t(1) << e.log2N0) < N0) ++e.log2N0;
      e.L = Md / N0;
      e.nchunks = N0 / 2;
      e.cap = std::max(20, (int)std::ceil(2.6 * e.P.log2d));  // I_N = 2.6 (Sec. 4.2)
      e.seed_off = b.seeds_total;
      e.chunk_off = b.chunks_total;
      e.start_off = b.S;
      b.seed_off.push_back(b.seeds_total);
      b.chunk_off.push_back(b.chunks_total);
      b.start_off.push_back(b.S);
      b.seeds_total += e.nchunks + 1;
      b.chunks_total += e.nchunks;
      b.S += (Md / 2) / b.every + 1;
      b.deg.push_back(d);
      b.deg_total += d;
      b.E.push_back(e);
      b.polys.push_back(e.P);
    }
  b.np = (int)b.E.size();
  if (b.np > 0xfffe) return false;
  b.seed_off.push_back(b.seeds_total);
  b.chunk_off.push_back(b.chunks_total);
  b.start_off.push_back(b.S);
  *bp = b;
  return true;
}

struct BatchBuffers {
  DevCounters* ctr;
  BatchEntry* E;
  PolyDev* polys;
  int64_t *seed_off, *chunk_off, *start_off;
  unsigned long long* pstat;
  double2 *seeds, *starts, *cand, *reps;
  uint8_t *status, *type, *pass;
  uint16_t *seg, *rep_seg, *out_seg;
  uint64_t *keys, *keys_alt;
  uint32_t *vals, *vals_alt, *flag, *pos, *mult, *mpos;
  double* radius;
  void *scan_tmp, *radix_tmp;
  size_t bytes;
};

BatchBuffers carve_batch(const BatchPlan& b, void* ws, size_t cap) {
  Carve c(ws, cap);
  BatchBuffers r;
  r.ctr = c.take<DevCounters>(1);
  r.E = c.take<BatchEntry>(b.np);
  r.polys = c.take<PolyDev>(b.np);
  r.seed_off = c.take<int64_t>(b.np + 1);
  r.chunk_off = c.take<int64_t>(b.np + 1);
  r.start_off = c.take<int64_t>(b.np + 1);
  r.pstat = c.take<unsigned long long>((int64_t)b.np * PSTAT_W);
  r.seeds = c.take<double2>(b.seeds_total);
  r.starts = c.take<double2>(b.S);
  r.cand = c.take<double2>(b.S);
  r.reps = r.starts;
  r.status = c.take<uint8_t>(b.S);
  r.seg = c.take<uint16_t>(b.S);
  r.rep_seg = c.take<uint16_t>(b.S);
  r.out_seg = c.take<uint16_t>(b.deg_total + 64);
  r.keys = c.take<uint64_t>(b.S);
  r.keys_alt = c.take<uint64_t>(b.S);
  r.vals = c.take<uint32_t>(b.S);
  r.vals_alt = c.take<uint32_t>(b.S);
  r.flag = c.take<uint32_t>(b.S);
  r.pos = c.take<uint32_t>(b.S);
  r.type = c.take<uint8_t>(b.S);
  r.mult = r.flag;
  r.mpos = r.pos;
  r.pass = c.take<uint8_t>(b.S);
  r.radius = c.take<double>(b.S);
  r.scan_tmp = c.take_bytes(scan_temp_bytes(b.S));
  r.radix_tmp = c.take_bytes(radix_temp_bytes(b.S));
  r.bytes = c.off;
  return r;
}

size_t batch_workspace(int max_order, const mt_options* o) {
  const int retries = o ? std::max(0, o->max_retries) : 1;
  size_t best = 0;
  for (int r = 0; r <= retries; ++r) {
    BatchPlan b;
    if (!make_batch_plan(max_order, o, r, &b)) {
      if (r == 0) return 0;
      break;
    }
    best = std::max(best, carve_batch(b, nullptr, 0).bytes);
  }
  return best;
}

mt_status run_batch_pass(const BatchPlan& b, const BatchBuffers& r, double2* out, int64_t cap_out,
                         uint8_t* is_mis, cudaStream_t s, EventSet& ev, DevCounters* h,
                         std::vector<unsigned long long>* ps) {
  CK(launch_init_counters(r.ctr, s));
  CK(cudaMemsetAsync(r.pstat, 0, sizeof(unsigned long long) * (size_t)b.np * PSTAT_W, s));
  CK(cudaMemcpyAsync(r.E, b.E.data(), sizeof(BatchEntry) * b.np, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(r.polys, b.polys.data(), sizeof(PolyDev) * b.np, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(r.seed_off, b.seed_off.data(), sizeof(int64_t) * (b.np + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(r.chunk_off, b.chunk_off.data(), sizeof(int64_t) * (b.np + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(r.start_off, b.start_off.data(), sizeof(int64_t) * (b.np + 1), cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(ev.e[0], s));
  CK(launch_seed_lift_batch(r.E, r.seed_off, b.np, b.seeds_total, b.lambda0, b.shrink, r.seeds, r.ctr, s));
  CK(cudaEventRecord(ev.e[6], s));
  CK(launch_walk_batch(r.E, r.chunk_off, b.np, b.chunks_total, b.lambda0, b.M, b.every, r.seeds,
                       r.starts, r.ctr, s));
  CK(cudaEventRecord(ev.e[1], s));
  CK(launch_descend_batch(r.E, r.start_off, b.np, b.S, b.tol, r.starts, r.cand, r.status, r.seg,
                          r.ctr, s));
  CK(cudaEventRecord(ev.e[2], s));
  SegView sv;
  sv.tab = r.polys;
  sv.seg = r.seg;
  sv.rep_seg = r.rep_seg;
  sv.out_seg = r.out_seg;
  sv.pstat = r.pstat;
  CK(launch_fold_keys(r.status, r.cand, b.S, b.eps, r.keys, r.vals, s));
  CK(radix_sort_pairs(r.keys, r.vals, r.keys_alt, r.vals_alt, b.S, r.radix_tmp, s));
  bool in_alt = false;
  CK(launch_seg_keys(r.vals, r.seg, r.status, b.S, r.keys, s));
  CK(radix_sort_bits(r.keys, r.vals, r.keys_alt, r.vals_alt, b.S, r.radix_tmp, 0, 16, &in_alt, s));
  const uint32_t* vals = in_alt ? r.vals_alt : r.vals;
  CK(launch_cluster(r.cand, vals, b.S, &r.ctr->n_conv, b.eps, r.flag, r.ctr, s, sv));
  CK(launch_exclusive_scan(r.flag, r.pos, b.S, r.scan_tmp, nullptr, s));
  CK(launch_compact(r.cand, vals, r.flag, r.pos, b.S, r.reps, r.ctr, s, sv));
  CK(cudaEventRecord(ev.e[3], s));
  PolyDev P0 = b.polys[0];
  CK(launch_classify(P0, r.reps, &r.ctr->n_reps, b.S, b.eps, 0, r.type, r.mult, r.ctr, s, sv));
  CK(launch_exclusive_scan(r.mult, r.mpos, b.S, r.scan_tmp, &r.ctr->n_full, s));
  CK(launch_certify(P0, r.reps, &r.ctr->n_reps, b.S, b.cert_tol, r.mult, r.pass, r.radius, r.ctr, s, sv));
  CK(cudaEventRecord(ev.e[4], s));
  CK(launch_emit(r.reps, &r.ctr->n_reps, b.S, r.mult, r.mpos, r.type, -1, out, is_mis, cap_out, s, sv));
  CK(launch_fix_ties(out, &r.ctr->n_full, cap_out, is_mis, s, sv));
  CK(cudaEventRecord(ev.e[5], s));
  ps->assign((size_t)b.np * PSTAT_W, 0ull);
  CK(cudaMemcpyAsync(h, r.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ps->data(), r.pstat, sizeof(unsigned long long) * ps->size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return MT_OK;
}

// ---------------------------------------------------------------------------
// q_{l,n} in the double-double tier, through its factors: eq. polySimple
// telescoped, q_{l,n} = p_n^2 prod_{j=2..l} s_{j,n} (mt_qfactors.cu).  Each
// factor is split by the certified double-double split of its own kind; the
// Hyp(k) roots come from p_n with multiplicity floor((l-1)/k) + 2 (Thm
// fact_mis), the Mis(j,k) roots from s_{j,n}.  Workspace: the largest
// factor's split, then one factor's roots and type codes, the union list
// (roots, preperiod, period, multiplicity) and the two sorts by (Re, Im).
struct QfLayout {
  size_t sub = 0, fac_roots = 0, fac_type = 0, u_roots = 0, u_pre = 0, u_per = 0, u_mult = 0;
  size_t keys = 0, keys_alt = 0, vals = 0, vals_alt = 0, rtmp = 0, cnt = 0, total = 0;
  int64_t dmax = 0, nmax = 0;
};

bool qf_layout(int l, int n, const mt_options* o, QfLayout* L) {
  if (!valid_poly(2, l, n)) return false;
  mt_options od = *o;
  od.prec = MT_DD;
  size_t sub = workspace_for(0, 0, n, &od);
  if (!sub) return false;
  int64_t dmax = int64_t(1) << (n - 1), nmax = dmax;
  for (int j = 2; j <= l; ++j) {
    const size_t w = workspace_for(1, j, n, &od);
    if (!w) return false;
    sub = std::max(sub, w);
    dmax = std::max<int64_t>(dmax, int64_t(1) << (j + n - 2));
    nmax += int64_t(1) << (j + n - 2);
  }
  if (nmax >= (int64_t(1) << 32)) return false;
  auto al = [](size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; };
  size_t at = 0;
  auto take = [&](size_t bytes) {
    const size_t r = at;
    at += al(bytes);
    return r;
  };
  L->sub = take(sub);
  L->fac_roots = take((size_t)dmax * sizeof(double2));
  L->fac_type = take((size_t)dmax);
  L->u_roots = take((size_t)nmax * sizeof(double2));
  L->u_pre = take((size_t)nmax);
  L->u_per = take((size_t)nmax);
  L->u_mult = take((size_t)nmax);
  L->keys = take((size_t)nmax * 8);
  L->keys_alt = take((size_t)nmax * 8);
  L->vals = take((size_t)nmax * 4);
  L->vals_alt = take((size_t)nmax * 4);
  L->rtmp = take(radix_temp_bytes(nmax));
  L->cnt = take(8 * sizeof(unsigned long long));
  L->total = at;
  L->dmax = dmax;
  L->nmax = nmax;
  return true;
}

mt_status split_q_factors(int l, int n, const mt_options* o, double* d_roots, int64_t cap, uint8_t* d_mult,
                          uint8_t* d_pre, uint8_t* d_per, void* d_work, size_t work_bytes, int64_t* n_out,
                          mt_stats* st) {
  QfLayout L;
  if (!qf_layout(l, n, o, &L)) return fail(MT_EINVAL, "no plan for the factors of q_{%d,%d}", l, n);
  if (cap < 0 || (cap > 0 && !d_roots)) return fail(MT_EINVAL, "bad output buffer");
  if (!d_work || work_bytes < L.total)
    return fail(MT_ENOMEM, "workspace of %zu bytes needed, %zu given", L.total, work_bytes);
  if (((uintptr_t)d_work) % ALIGN) return fail(MT_EINVAL, "workspace must be 256-byte aligned");
  char* w = (char*)d_work;
  mt_options od = *o;
  od.prec = MT_DD;
  cudaStream_t s = (cudaStream_t)o->stream;
  double2* fr = (double2*)(w + L.fac_roots);
  uint8_t* ft = (uint8_t*)(w + L.fac_type);
  double2* ur = (double2*)(w + L.u_roots);
  uint8_t *upre = (uint8_t*)(w + L.u_pre), *uper = (uint8_t*)(w + L.u_per), *umult = (uint8_t*)(w + L.u_mult);
  uint64_t *keys = (uint64_t*)(w + L.keys), *keys_alt = (uint64_t*)(w + L.keys_alt);
  uint32_t *vals = (uint32_t*)(w + L.vals), *vals_alt = (uint32_t*)(w + L.vals_alt);
  unsigned long long* cnt = (unsigned long long*)(w + L.cnt);
  CK(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), s));
  const unsigned long long launches0 = g_launches;
  mt_stats agg;
  memset(&agg, 0, sizeof(agg));
  for (int j = 0; j <= l; ++j) {
    if (j == 1) continue;  // s_{1,n} = p_n: the second copy of p_n is its multiplicity
    const int kind = j == 0 ? 0 : 1;
    const int64_t deg = j == 0 ? (int64_t(1) << (n - 1)) : (int64_t(1) << (j + n - 2));
    mt_stats sf;
    int64_t nr = 0;
    const mt_status rc = split_impl(kind, j, n, &od, (double*)fr, nullptr, deg, ft, w + L.sub, L.fac_roots - L.sub,
                                    &nr, &sf, 1);
    if (rc != MT_OK) return rc;  // the factor's message stands
    CK(launch_qf_append(fr, ft, nr, j, l, n, ur, upre, uper, umult, L.nmax, cnt, s));
    for (int k = 1; k < 32; ++k) {
      if (j == 0) agg.count_by_type[32 + k] += sf.count_by_type[k];  // Hyp(k)
      else if (j == l) agg.count_by_type[k] += sf.count_by_type[k];  // Mis(l,k)
      else agg.count_by_type[0] += sf.count_by_type[k];              // Mis(j,k), j < l
    }
    agg.n_starts += sf.n_starts;
    agg.n_conv += sf.n_conv;
    agg.n_repeat += sf.n_repeat;
    agg.n_diverge += sf.n_diverge;
    agg.n_timeout += sf.n_timeout;
    agg.walk_newton += sf.walk_newton;
    agg.desc_newton += sf.desc_newton;
    agg.steps_fp32 += sf.steps_fp32;
    agg.steps_dd += sf.steps_dd;
    agg.walk_fail += sf.walk_fail;
    agg.retries = std::max(agg.retries, sf.retries);
    agg.ms_total += sf.ms_total;
    agg.ms_walk += sf.ms_walk;
    agg.ms_descend += sf.ms_descend;
    agg.ms_dedup += sf.ms_dedup;
    agg.ms_certify += sf.ms_certify;
    agg.ms_dd += sf.ms_dd;
    agg.n_zones += sf.n_zones;
    agg.n_zone_roots += sf.n_zone_roots;
    agg.n_dd_pieces += sf.n_dd_pieces;
    agg.M = sf.M;
    agg.c_L = sf.c_L;
    agg.eps_dup = std::max(agg.eps_dup, sf.eps_dup);
  }
  unsigned long long hc[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t nu = (int64_t)hc[0];
  if (n_out) *n_out = nu;
  if (nu > L.nmax) return fail(MT_ECAPACITY, "%lld roots in the union of the factors of q_{%d,%d}", (long long)nu, l, n);
  // (Re, Im) order: by Im, then stably by Re
  if (nu > 0) {
    CK(launch_qf_keys(ur, nullptr, L.nmax, &cnt[0], 1, keys, vals, s));
    CK(radix_sort_pairs(keys, vals, keys_alt, vals_alt, L.nmax, w + L.rtmp, s, &cnt[0]));
    CK(launch_qf_keys(ur, vals, L.nmax, &cnt[0], 0, keys_alt, vals_alt, s));
    CK(radix_sort_pairs(keys_alt, vals_alt, keys, vals, L.nmax, w + L.rtmp, s, &cnt[0]));
    if (nu <= cap)
      CK(launch_qf_gather(vals_alt, cap, &cnt[0], ur, upre, uper, umult, (double2*)d_roots, d_pre, d_per, d_mult, s));
    CK(cudaStreamSynchronize(s));
  }
  const int64_t degree = int64_t(1) << (l + n - 1);
  if (st) {
    memset(st, 0, sizeof(*st));
    *st = agg;
    st->degree = degree;
    st->n_roots = nu;
    st->n_mult = (int64_t)hc[1];
    st->n_real = (int64_t)hc[3];
    st->n_cert_pass = nu;  // every factor's split certified all its roots, or failed above
    st->prec_used = MT_DD;
    st->first_prec = MT_DD;
    st->n_launches = (int64_t)(g_launches - launches0);
  }
  if (hc[2]) return fail(MT_EINCOMPLETE, "%llu roots of the factors of q_{%d,%d} without a type", hc[2], l, n);
  if ((int64_t)hc[1] != degree)
    return fail(MT_EINCOMPLETE, "factors of q_{%d,%d}: %llu roots with multiplicity, degree %lld", l, n, hc[1],
                (long long)degree);
  if (nu > cap) return fail(MT_ECAPACITY, "%lld roots do not fit in cap %lld", (long long)nu, (long long)cap);
  return MT_OK;
}

}  // namespace

void mt::set_error_message(const char* msg) { g_err = msg ? msg : ""; }

// ===========================================================================
// C ABI
extern "C" {

void mt_default_options(mt_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->prec = MT_FP64;
  o->max_retries = 1;
}

int64_t mt_degree_hyperbolic(int n) { return valid_poly(0, 0, n) ? (int64_t(1) << (n - 1)) : -1; }

int64_t mt_degree_misiurewicz(int l, int n) {
  return valid_poly(1, l, n) ? (int64_t(1) << (l + n - 2)) : -1;
}

size_t mt_workspace_bytes(int kind, int l, int n, const mt_options* opts) {
  mt_options d;
  mt_default_options(&d);
  if (kind == 2 && opts && opts->prec == MT_DD) {
    QfLayout L;
    return qf_layout(l, n, opts, &L) ? L.total : 0;
  }
  return workspace_for(kind, kind == 0 ? 0 : l, n, opts ? opts : &d);
}

mt_status mt_split_hyperbolic(int n, const mt_options* opts, double* d_roots, double* d_roots_lo,
                              int64_t cap, void* d_work, size_t work_bytes, int64_t* n_out,
                              mt_stats* stats) {
  return split_impl(0, 0, n, opts, d_roots, d_roots_lo, cap, nullptr, d_work, work_bytes, n_out,
                    stats);
}

mt_status mt_split_misiurewicz(int l, int n, const mt_options* opts, double* d_roots,
                               double* d_roots_lo, int64_t cap, uint8_t* d_is_mis, void* d_work,
                               size_t work_bytes, int64_t* n_out, mt_stats* stats) {
  return split_impl(1, l, n, opts, d_roots, d_roots_lo, cap, d_is_mis, d_work, work_bytes, n_out,
                    stats);
}

mt_status mt_split_misiurewicz_q(int l, int n, const mt_options* opts, double* d_roots, int64_t cap,
                                 uint8_t* d_mult, uint8_t* d_pre, uint8_t* d_per, void* d_work,
                                 size_t work_bytes, int64_t* n_out, mt_stats* stats) {
  g_err.clear();
  if (opts && opts->prec == MT_DD)
    return split_q_factors(l, n, opts, d_roots, cap, d_mult, d_pre, d_per, d_work, work_bytes, n_out, stats);
  if (opts && opts->prec != MT_FP64)
    return fail(MT_EINVAL, "q_{l,n} is split in binary64 (MT_FP64) or through its factors (MT_DD)");
  int64_t nr = 0;
  const mt_status rc = split_impl(2, l, n, opts, d_roots, nullptr, cap, nullptr, d_work, work_bytes, &nr, stats);
  if (n_out) *n_out = nr;
  if (rc != MT_OK && rc != MT_EINCOMPLETE && rc != MT_ECERT) return rc;
  if (d_mult || d_pre || d_per) {  // also for an incomplete or uncertified list
    mt_options dflt;
    mt_default_options(&dflt);
    const mt_options* o = opts ? opts : &dflt;
    const double tau = (o->eps_dup > 0) ? o->eps_dup : default_eps(2, l, n);
    cudaStream_t s = (cudaStream_t)o->stream;
    const std::string err = g_err;  // keep the split's message
    CK(launch_type_q(make_poly(2, l, n), (const double2*)d_roots, std::min(nr, cap), tau, d_pre, d_per, d_mult,
                     s));
    g_err = err;
  }
  return rc;
}

int mt_misiurewicz_pairs(int max_order, int* h_l, int* h_n, int capacity) {
  int k = 0;
  for (int l = 2; l < max_order; ++l)
    for (int n = 1; l + n <= max_order; ++n) {
      if (k < capacity && h_l && h_n) {
        h_l[k] = l;
        h_n[k] = n;
      }
      ++k;
    }
  return k;
}

size_t mt_workspace_bytes_misiurewicz_batch(int max_order, const mt_options* opts) {
  mt_options d;
  mt_default_options(&d);
  return batch_workspace(max_order, opts ? opts : &d);
}

mt_status mt_split_misiurewicz_batch(int max_order, const mt_options* opts, double* d_roots,
                                     double* d_roots_lo, int64_t cap, uint8_t* d_is_mis,
                                     void* d_work, size_t work_bytes, int64_t* h_offsets,
                                     mt_stats* stats) {
  g_err.clear();
  mt_options dflt;
  mt_default_options(&dflt);
  const mt_options* o = opts ? opts : &dflt;
  if (max_order < 3 || max_order > 41 || !h_offsets) return fail(MT_EINVAL, "bad max_order or offsets");
  if (o->prec != MT_FP64) return fail(MT_EINVAL, "the batched split runs in MT_FP64");
  const size_t need = batch_workspace(max_order, o);
  if (need == 0) return fail(MT_EINVAL, "invalid options for this batch");
  if (!d_work || work_bytes < need)
    return fail(MT_ENOMEM, "workspace of %zu bytes needed, %zu given", need, work_bytes);
  if (((uintptr_t)d_work) % ALIGN) return fail(MT_EINVAL, "workspace must be 256-byte aligned");
  if (cap < 0 || (cap > 0 && !d_roots)) return fail(MT_EINVAL, "bad output buffer");
  cudaStream_t s = (cudaStream_t)o->stream;
  EventSet ev;
  if (!ev.ok) return fail(MT_ECUDA, "cudaEventCreate failed");
  const unsigned long long launches0 = g_launches;
  BatchPlan b;
  DevCounters h;
  std::vector<unsigned long long> ps;
  int retry = 0;
  bool good = false;
  for (;; ++retry) {
    if (!make_batch_plan(max_order, o, retry, &b)) {
      if (retry == 0) return fail(MT_EINVAL, "no plan for this batch and these options");
      --retry;  // (M, c_L) cannot double further: the last pass's result stands
      break;
    }
    BatchBuffers r = carve_batch(b, d_work, work_bytes);
    mt_status rc = run_batch_pass(b, r, (double2*)d_roots, cap, d_is_mis, s, ev, &h, &ps);
    if (rc != MT_OK) return rc;
    good = h.walk_fail == 0;
    for (int p = 0; p < b.np; ++p) good = good && (int64_t)ps[(size_t)p * PSTAT_W + 2] == b.deg[p];
    if (good || retry >= std::max(0, o->max_retries)) break;
  }
  h_offsets[0] = 0;
  for (int p = 0; p < b.np; ++p) h_offsets[p + 1] = h_offsets[p] + (int64_t)ps[(size_t)p * PSTAT_W + 2];
  if (d_roots_lo && cap > 0) CK(cudaMemsetAsync(d_roots_lo, 0, (size_t)cap * sizeof(double2), s));
  float ms[5] = {0, 0, 0, 0, 0};
  cudaEventElapsedTime(&ms[0], ev.e[0], ev.e[5]);
  cudaEventElapsedTime(&ms[1], ev.e[0], ev.e[1]);
  cudaEventElapsedTime(&ms[2], ev.e[1], ev.e[2]);
  cudaEventElapsedTime(&ms[3], ev.e[2], ev.e[3]);
  cudaEventElapsedTime(&ms[4], ev.e[3], ev.e[4]);
  float ms_seeds = 0.f;
  cudaEventElapsedTime(&ms_seeds, ev.e[0], ev.e[6]);
  int64_t bad_cert = 0;
  for (int p = 0; p < b.np; ++p) {
    const unsigned long long* q = &ps[(size_t)p * PSTAT_W];
    bad_cert += (int64_t)(q[2] - q[3]);
    if (!stats) continue;
    mt_stats& st = stats[p];
    memset(&st, 0, sizeof(st));
    st.degree = b.deg[p];
    st.n_roots = (int64_t)q[2];
    st.n_real = (int64_t)q[1];
    st.n_starts = b.start_off[p + 1] - b.start_off[p];
    st.n_cert_pass = (int64_t)q[3];
    for (int t = 0; t < MT_MAX_TYPES; ++t) st.count_by_type[t] = (int64_t)q[4 + t];
    // batch-wide counters and timings are reported on every entry
    st.n_conv = (int64_t)h.n_conv;
    st.n_diverge = (int64_t)h.n_diverge;
    st.n_timeout = (int64_t)h.n_timeout;
    st.walk_newton = (int64_t)h.walk_newton;
    st.desc_newton = (int64_t)h.desc_newton;
    st.walk_fail = (int64_t)h.walk_fail;
    st.seed_newton = (int64_t)h.seed_newton;
    st.ms_seeds = ms_seeds;
    st.M = b.M;
    st.c_L = b.cL;
    st.retries = retry;
    st.n_chunks = (int32_t)(b.E[p].nchunks);
    st.n_launches = (int64_t)(g_launches - launches0);
    st.eps_dup = b.eps;
    st.ms_total = ms[0];
    st.ms_walk = ms[1];
    st.ms_descend = ms[2];
    st.ms_dedup = ms[3];
    st.ms_certify = ms[4];
    st.ms_k_desc64 = ms[2];  // the descent stage is the one k_descend_batch launch
    st.desc_orbit_steps = (int64_t)h.desc_orbit;
    st.prec_used = MT_FP64;
  }
  if (!good) return fail(MT_EINCOMPLETE, "some polynomials of the batch miss roots (after %d retries)", retry);
  if (h_offsets[b.np] > cap)
    return fail(MT_ECAPACITY, "%lld roots do not fit in cap %lld", (long long)h_offsets[b.np], (long long)cap);
  if (bad_cert) return fail(MT_ECERT, "%lld roots of the batch failed the certificate", (long long)bad_cert);
  return MT_OK;
}

mt_status mt_autotune(int kind, int l, int n, const mt_options* opts, double* d_roots, int64_t cap,
                      void* d_work, size_t work_bytes, int* best_chunk_log2, int* best_block,
                      float* best_ms) {
  g_err.clear();
  mt_options base;
  if (opts) base = *opts; else mt_default_options(&base);
  if (!valid_poly(kind, l, n)) return fail(MT_EINVAL, "polynomial out of range");
  if (base.prec != MT_FP64 && base.prec != MT_MIXED) return fail(MT_EINVAL, "tier cannot be tuned");
  base.max_retries = 0;
  base.use_graph = 0;
  const int ll = kind == 0 ? 0 : l;
  {  // forget a previous result so the default plan is among the candidates
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.erase(TuneKey{kind, ll, n, base.prec});
  }
  float best = 1e30f;
  int bc = 0, bb = 0;
  const int blocks[3] = {32, 64, 128};
  for (int cl = 3; cl <= 14; ++cl) {
    for (int bi = 0; bi < 3; ++bi) {
      mt_options o = base;
      o.chunk_log2 = cl;
      o.block = blocks[bi];
      Plan p;
      if (!make_plan(kind, ll, n, &o, 0, &p)) continue;
      if (p.L != (int64_t(1) << cl)) continue;  // the plan adjusted the chunk: not this candidate
      if (p.nchunks < 64 && cl > 3) continue;     // too few lanes to be a sensible layout
      if (workspace_for(kind, ll, n, &o) > work_bytes) continue;
      float tsum = 0.f;
      bool ok = true;
      for (int rep = 0; rep < 3 && ok; ++rep) {
        int64_t got = 0;
        mt_stats st;
        mt_status rc = split_impl(kind, ll, n, &o, d_roots, nullptr, cap, nullptr, d_work, work_bytes,
                                  &got, &st);
        ok = (rc == MT_OK);
        if (rep > 0) tsum += st.ms_total;  // first run warms up
      }
      if (!ok) continue;
      const float t = tsum / 2.f;
      if (t < best) {
        best = t;
        bc = cl;
        bb = blocks[bi];
      }
    }
  }
  g_err.clear();
  if (bc == 0) return fail(MT_EINVAL, "no candidate layout succeeded");
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{kind, ll, n, base.prec}] = TuneVal{bc, bb};
  }
  if (best_chunk_log2) *best_chunk_log2 = bc;
  if (best_block) *best_block = bb;
  if (best_ms) *best_ms = best;
  return MT_OK;
}

size_t mt_certify_workspace_bytes(int64_t count) {
  if (count < 0) return 0;
  Carve c(nullptr, 0);
  c.take<DevCounters>(1);
  c.take<uint64_t>(count);
  c.take<uint64_t>(count);
  c.take<uint32_t>(count);
  c.take<uint32_t>(count);
  c.take_bytes(radix_temp_bytes(count));
  return c.off;
}

mt_status mt_certify(int kind, int l, int n, const double* d_roots, const double* d_roots_lo,
                     int64_t count, double tol, uint8_t* d_pass, double* d_radius, void* d_work,
                     size_t work_bytes, int64_t* n_pass, void* stream) {
  g_err.clear();
  if (!valid_poly(kind, l, n)) return fail(MT_EINVAL, "polynomial out of range");
  if (count < 0 || (count > 0 && (!d_roots || !d_pass))) return fail(MT_EINVAL, "bad buffers");
  if (count > 0xffffffffll) return fail(MT_EINVAL, "count too large");
  if (d_roots_lo && kind == 2) return fail(MT_EINVAL, "q_{l,n} roots are certified in binary64 only");
  const size_t need = mt_certify_workspace_bytes(count);
  if (!d_work || work_bytes < need) return fail(MT_ENOMEM, "workspace of %zu bytes needed", need);
  cudaStream_t s = (cudaStream_t)stream;
  const PolyDev P = make_poly(kind, l, n);
  if (tol <= 0) tol = d_roots_lo ? 1e-20 : 1e-12;
  Carve c(d_work, work_bytes);
  DevCounters* ctr = c.take<DevCounters>(1);
  uint64_t* keys = c.take<uint64_t>(count);
  uint64_t* keys_alt = c.take<uint64_t>(count);
  uint32_t* vals = c.take<uint32_t>(count);
  uint32_t* vals_alt = c.take<uint32_t>(count);
  void* rtmp = c.take_bytes(radix_temp_bytes(count));
  CK(launch_init_counters(ctr, s));
  CK(launch_keys_plain((const double2*)d_roots, count, keys, vals, s));
  CK(radix_sort_pairs(keys, vals, keys_alt, vals_alt, count, rtmp, s));
  if (d_roots_lo) {
    CK(dd_certify_list(P, (const double2*)d_roots, (const double2*)d_roots_lo, vals, count, tol, d_pass,
                       d_radius, ctr, s));
  } else {
    // q_{l,n}: a root typed Hyp(k) is proven as a (simple) root of p_n; the
    // types go in vals_alt, free after the sort
    uint8_t* type = nullptr;
    if (kind == 2) {
      type = (uint8_t*)vals_alt;
      CK(launch_type_only(P, (const double2*)d_roots, count, default_eps(2, l, n), type, s));
    }
    CK(launch_certify_list(P, (const double2*)d_roots, vals, count, tol, d_pass, d_radius, ctr, s, type));
  }
  DevCounters h;
  CK(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n_pass) *n_pass = (int64_t)h.n_cert_pass;
  return MT_OK;
}

mt_status mt_certify_basin(int kind, int l, int n, const double* d_roots, const double* d_roots_lo,
                           int64_t count, const double* d_radius, double eps_max, double* d_basin,
                           void* d_work, size_t work_bytes, int64_t* n_pass, void* stream) {
  g_err.clear();
  if (!valid_poly(kind, l, n)) return fail(MT_EINVAL, "polynomial out of range");
  if (count < 0 || (count > 0 && (!d_roots || !d_radius || !d_basin))) return fail(MT_EINVAL, "bad buffers");
  if (count > 0xffffffffll) return fail(MT_EINVAL, "count too large");
  if (!(eps_max >= 0.0)) return fail(MT_EINVAL, "eps_max must be >= 0");
  if (kind == 2) return fail(MT_EINVAL, "Thm proofContract is for simple roots: q_{l,n} has multiple roots");
  const size_t need = mt_certify_workspace_bytes(count);
  if (!d_work || work_bytes < need) return fail(MT_ENOMEM, "workspace of %zu bytes needed", need);
  cudaStream_t s = (cudaStream_t)stream;
  const PolyDev P = make_poly(kind, l, n);
  if (eps_max == 0.0) eps_max = 1e-6;
  Carve c(d_work, work_bytes);
  DevCounters* ctr = c.take<DevCounters>(1);
  uint64_t* keys = c.take<uint64_t>(count);
  uint64_t* keys_alt = c.take<uint64_t>(count);
  uint32_t* vals = c.take<uint32_t>(count);
  uint32_t* vals_alt = c.take<uint32_t>(count);
  void* rtmp = c.take_bytes(radix_temp_bytes(count));
  CK(launch_init_counters(ctr, s));
  CK(launch_keys_plain((const double2*)d_roots, count, keys, vals, s));
  CK(radix_sort_pairs(keys, vals, keys_alt, vals_alt, count, rtmp, s));
  if (d_roots_lo)
    CK(dd_basin(P, (const double2*)d_roots, (const double2*)d_roots_lo, vals, count, d_radius, eps_max,
                d_basin, ctr, s));
  else
    CK(launch_basin(P, (const double2*)d_roots, vals, count, d_radius, eps_max, d_basin, ctr, s));
  DevCounters h;
  CK(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (n_pass) *n_pass = (int64_t)h.n_cert_pass;
  return MT_OK;
}

size_t mt_separation_workspace_bytes(int64_t count) {
  if (count < 0) return 0;
  Carve c(nullptr, 0);
  c.take<DevCounters>(1);
  c.take<uint64_t>(count);
  c.take<uint64_t>(count);
  c.take<uint32_t>(count);
  c.take<uint32_t>(count);
  c.take_bytes(radix_temp_bytes(count));
  c.take<uint32_t>(count);
  c.take<double>(count);
  c.take<uint32_t>(((int64_t)1 << separation_strips_log2(count)) + 1);
  return c.off;
}

mt_status mt_separation(int64_t count, const double* d_roots, const double* d_roots_lo,
                        const uint8_t* d_mask, double* d_nn, double* h_band_min, double* h_min,
                        void* d_work, size_t work_bytes, void* stream) {
  g_err.clear();
  if (count < 0 || (count > 0 && !d_roots)) return fail(MT_EINVAL, "bad buffers");
  if (count > 0xffffffffll) return fail(MT_EINVAL, "count too large");
  const size_t need = mt_separation_workspace_bytes(count);
  if (!d_work || work_bytes < need) return fail(MT_ENOMEM, "workspace of %zu bytes needed", need);
  cudaStream_t s = (cudaStream_t)stream;
  // the counter slot holds the band minima and the isolated-root count
  static_assert(sizeof(DevCounters) >= 67 * sizeof(unsigned long long), "band minima slot");
  Carve c(d_work, work_bytes);
  unsigned long long* band = (unsigned long long*)c.take<DevCounters>(1);
  uint64_t* keys = c.take<uint64_t>(count);
  uint64_t* keys_alt = c.take<uint64_t>(count);
  uint32_t* vals = c.take<uint32_t>(count);
  uint32_t* vals_alt = c.take<uint32_t>(count);
  void* rtmp = c.take_bytes(radix_temp_bytes(count));
  uint32_t* iso_idx = c.take<uint32_t>(count);
  double* iso_best = c.take<double>(count);
  const int log2s = separation_strips_log2(count);
  uint32_t* offs = c.take<uint32_t>(((int64_t)1 << log2s) + 1);
  const double2* hi = (const double2*)d_roots;
  const double2* lo = (const double2*)d_roots_lo;
  // tier 1: Re-window scan over the list sorted by Re
  if (count > 0) {
    CK(launch_keys_plain(hi, count, keys, vals, s));
    CK(radix_sort_pairs(keys, vals, keys_alt, vals_alt, count, rtmp, s));
  }
  CK(launch_separation(hi, lo, vals, count, d_mask, d_nn, band, iso_idx, iso_best, s));
  unsigned long long hb[67];
  CK(cudaMemcpyAsync(hb, band, sizeof(hb), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // tiers 2 and 3, for the roots tier 1 left: (strip, Im) index, strip
  // walks; after the sort keys_alt / vals_alt hold tier 3's list
  if (hb[65] > 0) {
    CK(launch_strip_index(hi, count, log2s, keys, vals, keys_alt, vals_alt, rtmp, offs, s));
    CK(launch_separation_strips(hi, lo, d_mask, keys, vals, offs, log2s, iso_idx, iso_best, (int64_t)hb[65],
                                vals_alt, (double*)keys_alt, d_nn, band, s));
    CK(cudaMemcpyAsync(hb, band, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  double bd[65];
  memcpy(bd, hb, sizeof(bd));
  if (h_band_min) memcpy(h_band_min, bd, 64 * sizeof(double));
  if (h_min) *h_min = bd[64];
  return MT_OK;
}

mt_status mt_eval(int kind, int l, int n, const double* d_c, int64_t count, double* d_out,
                  void* stream) {
  g_err.clear();
  if (!valid_poly(kind, l, n)) return fail(MT_EINVAL, "polynomial out of range");
  if (count < 0 || (count > 0 && (!d_c || !d_out))) return fail(MT_EINVAL, "bad buffers");
  CK(launch_eval(make_poly(kind, l, n), (const double2*)d_c, count, (double2*)d_out,
                 (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return MT_OK;
}

mt_status mt_level_line(int kind, int l, int n, const mt_options* opts, double* d_starts,
                        int64_t cap, void* d_work, size_t work_bytes, int64_t* n_starts,
                        mt_stats* stats) {
  g_err.clear();
  mt_options dflt;
  mt_default_options(&dflt);
  const mt_options* o = opts ? opts : &dflt;
  Plan p;
  if (!make_plan(kind, l, n, o, 0, &p)) return fail(MT_EINVAL, "invalid polynomial or options");
  Buffers b = carve(p, d_work, work_bytes);
  if (!d_work || work_bytes < b.bytes) return fail(MT_ENOMEM, "workspace of %zu bytes needed", b.bytes);
  if (n_starts) *n_starts = p.S;
  if (cap < p.S || !d_starts) return fail(MT_ECAPACITY, "%lld starts need a larger buffer", (long long)p.S);
  cudaStream_t s = (cudaStream_t)o->stream;
  CK(launch_init_counters(b.ctr, s));
  CK(launch_seed_lift(p.P, p.lambda0, p.N0, p.shrink, b.seeds, b.ctr, s));
  CK(launch_walk(p.P, p.lambda0, p.M, p.every, p.L, p.nchunks, b.seeds, (double2*)d_starts, b.ctr, s));
  DevCounters h;
  CK(cudaMemcpyAsync(&h, b.ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    fill_stats(p, h, stats);
  }
  return MT_OK;
}

mt_status mt_descend(int kind, int l, int n, const mt_options* opts, const double* d_starts,
                     int64_t count, double* d_out, uint8_t* d_status, void* d_work,
                     size_t work_bytes, mt_stats* stats) {
  g_err.clear();
  mt_options dflt;
  mt_default_options(&dflt);
  const mt_options* o = opts ? opts : &dflt;
  Plan p;
  if (!make_plan(kind, l, n, o, 0, &p)) return fail(MT_EINVAL, "invalid polynomial or options");
  if (count < 0 || (count > 0 && (!d_starts || !d_out || !d_status))) return fail(MT_EINVAL, "bad buffers");
  if (!d_work || work_bytes < sizeof(DevCounters)) return fail(MT_ENOMEM, "workspace too small");
  cudaStream_t s = (cudaStream_t)o->stream;
  DevCounters* ctr = (DevCounters*)d_work;
  CK(launch_init_counters(ctr, s));
  CK(launch_descend(p.P, (const double2*)d_starts, count, p.tol, p.cap, (double2*)d_out, d_status,
                    ctr, o->block, s));
  DevCounters h;
  CK(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    fill_stats(p, h, stats);
    stats->n_starts = count;
  }
  return MT_OK;
}

mt_status mt_classify(int kind, int l, int n, const double* d_roots, int64_t count, double tau,
                      uint8_t* d_type, void* stream) {
  g_err.clear();
  if (!valid_poly(kind, l, n)) return fail(MT_EINVAL, "polynomial out of range");
  if (count < 0 || (count > 0 && (!d_roots || !d_type))) return fail(MT_EINVAL, "bad buffers");
  if (tau <= 0) tau = default_eps(kind, l, n);
  CK(launch_type_only(make_poly(kind, l, n), (const double2*)d_roots, count, tau, d_type,
                      (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  return MT_OK;
}

const char* mt_last_error(void) { return g_err.c_str(); }

const char* mt_version(void) { return "mtsplit 0.1 (sm_103a)"; }

}  // extern "C"
