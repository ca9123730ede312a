// mt_internal.h -- types shared between the host orchestration (mt_api.cu)
// and the kernel translation units.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mt {

// Polynomial descriptor passed by value to the kernels.
//   kind 0: P = p_n        m = n,          lcap = -1
//   kind 1: P = s_{l,n}    m = l + n - 1,  lcap = l - 1
struct PolyDev {
  int kind;
  int l, n;
  int m;
  int lcap;
  int log2d;  // deg P = 2^log2d
};

// Device-side counters of one split (zeroed at the start of a call).
struct DevCounters {
  unsigned long long walk_newton;
  unsigned long long desc_newton;
  unsigned long long steps_fp32;
  unsigned long long steps_dd;
  unsigned long long n_conv;
  unsigned long long n_diverge;
  unsigned long long n_timeout;
  unsigned long long walk_fail;
  unsigned long long n_reps;        // distinct roots, upper half (set by cluster pass)
  unsigned long long n_reps_real;
  unsigned long long n_full;        // full conjugate-closed count
  unsigned long long cluster_overflow;
  unsigned long long n_cert_pass;   // full list
  unsigned long long min_radius_bits;
  unsigned long long max_radius_bits;
  unsigned long long queue_head;    // work queue of the persistent descent
  unsigned long long queue_head2;   // second queue (batched walk)
  unsigned long long seed_newton;   // Newton steps of the seed lifts (part of walk_newton)
  unsigned long long desc_fp32;     // binary32 Newton steps of the descents (part of desc_newton)
  unsigned long long n_finish;      // binary64 finishes of the mixed tier (run heads)
  unsigned long long n_mult_full;   // q_{l,n}: full list counted with multiplicity (Thm fact_mis)
  unsigned long long finish_newton; // binary64 Newton steps of the mixed tier's finish (part of desc_newton)
  unsigned long long desc_orbit;    // batched descents: orbit steps summed over their Newton steps
  unsigned long long n_heads_conv;  // mixed tier: finished group heads that converged
  unsigned long long n_tip64;       // mixed tier: descents redone in binary64 at the left tip
  unsigned long long n_c32_fin;     // mixed tier: descents left for the binary64 finish
  unsigned long long type_count[64];
};

// Several polynomials in one pass (the batched Misiurewicz split): the
// polynomial of each candidate / representative / output root, and
// per-polynomial counters.  All null for a single polynomial.
constexpr int PSTAT_W = 68;  // per polynomial: n_reps, n_real, n_full, n_cert, 64 type counts
struct SegView {
  const PolyDev* tab = nullptr;         // [np] polynomials
  const uint16_t* seg = nullptr;        // per candidate (original start index)
  uint16_t* rep_seg = nullptr;          // per representative
  uint16_t* out_seg = nullptr;          // per output root
  unsigned long long* pstat = nullptr;  // [np][PSTAT_W]
};

// One polynomial of a batch: its level-line layout and where its seeds,
// chunks and starts begin in the concatenated arrays.
struct BatchEntry {
  PolyDev P;
  int log2N0;
  int cap;          // Newton cap max{20, I_N log2 d}
  int64_t N0;       // chunks around the whole line
  int64_t L;        // sub-steps per chunk
  int64_t nchunks;  // chunks of the upper half (N0 / 2)
  int64_t seed_off, chunk_off, start_off;
};

// The polynomial domain (kind 0: p_n, 1: s_{l,n}, 2: q_{l,n}) and the
// kernel descriptor of a polynomial in it.
bool valid_poly(int kind, int l, int n);
PolyDev make_poly(int kind, int l, int n);

// Per-kernel timing: CUDA events recorded around single launches on the
// launch stream (as external event nodes inside a stream capture, so they
// time the graph replay).  A no-op unless the host orchestration armed a
// timer set for the current call on this thread.
enum KSlot { KS_WALK = 0, KS_DESC64 = 1, KS_DESC32 = 2, KS_FINISH = 3, KS_N = 4 };
cudaError_t ktimer_begin(int slot, cudaStream_t s);
cudaError_t ktimer_end(cudaStream_t s);

// ---- launchers (each returns the launch error) ----------------------------

// a1 + a2: seeds of the chunked level line: seeds[j] = point with external
// angle index t = j / N0 on |P| = lambda0, j = 0 .. N0/2.
cudaError_t launch_seed_lift(const PolyDev& P, double lambda0, int64_t N0, int shrink_steps,
                             double2* seeds, DevCounters* ctr, cudaStream_t s);

// a3: walk chunk j from seeds[j] to seeds[j+1] in L sub-steps (M per turn),
// writing every 'every'-th point to starts[g / every].
cudaError_t launch_walk(const PolyDev& P, double lambda0, int M, int every, int64_t L,
                        int64_t nchunks, const double2* seeds, double2* starts, DevCounters* ctr,
                        cudaStream_t s, int block = 64);

// a4: persistent Newton descent over 'count' starts.
cudaError_t launch_descend(const PolyDev& P, const double2* starts, int64_t count, double tol,
                           int cap, double2* cand, uint8_t* status, DevCounters* ctr, int block,
                           cudaStream_t s);
// The same descents (binary64, stop rules of launch_descend) from the
// starts list[0 .. *nlist) only; outcomes at the listed indices, not
// counted in ctr (the caller counts them).
cudaError_t launch_descend_list(const PolyDev& P, const double2* starts, const uint32_t* list,
                                const unsigned long long* nlist, int64_t count, double tol, int cap,
                                double2* cand, uint8_t* status, DevCounters* ctr, cudaStream_t s);

// a1-a4 in the mixed tier (binary32 perturbation around binary64 anchors).
// seed_bad [N0/2 + 1] and chunk_fail [nchunks] receive the per-item
// failures that the binary64 repairs then redo.
cudaError_t launch_seed_lift_mixed(const PolyDev& P, double lambda0, int64_t N0, int shrink_steps,
                                   double2* seeds, uint8_t* seed_bad, DevCounters* ctr, cudaStream_t s);
// j0 / nch: chunks [j0, j0 + nch) only, their starts written from index 0
// (a streamed split's piece); nch < 0: the whole line
cudaError_t launch_walk_mixed(const PolyDev& P, double lambda0, int M, int every, int64_t L,
                              int64_t nchunks, int K, const double2* seeds, double2* starts,
                              uint8_t* chunk_fail, DevCounters* ctr, cudaStream_t s, int block = 64,
                              int64_t j0 = 0, int64_t nch = -1);
cudaError_t launch_mixed_repair_seeds(const PolyDev& P, double lambda0, int64_t N0, int shrink,
                                      double2* seeds, uint8_t* seed_bad, DevCounters* ctr,
                                      cudaStream_t s);
cudaError_t launch_mixed_repair_walk(const PolyDev& P, double lambda0, int M, int every, int64_t L,
                                     int64_t nchunks, int shrink, const double2* seeds,
                                     double2* starts, uint8_t* chunk_fail, DevCounters* ctr,
                                     cudaStream_t s, int64_t j0 = 0, int64_t nch = -1);
// Scratch of the binary64 finish of the mixed tier (count entries each):
// the sort of the binary32 end points, the group heads (in sorted order)
// and their scan, the list of heads and the links of their followers.
struct FinishScratch {
  uint64_t *keys, *keys_alt;
  uint32_t *vals, *vals_alt;      // sorted permutation; vals_alt then holds the head list
  uint32_t *head, *pos, *list;
  uint8_t* link;
  void *scan_tmp, *radix_tmp;     // scan_temp_bytes(count), radix_temp_bytes(count)
  unsigned long long* nheads;     // device counter
};
// starts: in, the starts; out, the binary32 end points (binary64 values,
// folded into the upper half where a finish followed).  cand: the
// candidates (also the binary32 deltas and scales before the finish).
cudaError_t launch_descend_mixed(const PolyDev& P, double2* starts, int64_t count, double tol, int cap,
                                 double2* cand, uint8_t* status, void* anchors, const FinishScratch& fin,
                                 DevCounters* ctr, cudaStream_t s);
size_t mixed_anchor_bytes(const PolyDev& P, int64_t count);

// Batched (several polynomials) seeds, walk and descents.
cudaError_t launch_seed_lift_batch(const BatchEntry* E, const int64_t* seed_off, int np,
                                   int64_t total, double lambda0, int shrink, double2* seeds,
                                   DevCounters* ctr, cudaStream_t s);
cudaError_t launch_walk_batch(const BatchEntry* E, const int64_t* chunk_off, int np, int64_t total,
                              double lambda0, int M, int every, const double2* seeds,
                              double2* starts, DevCounters* ctr, cudaStream_t s);
cudaError_t launch_descend_batch(const BatchEntry* E, const int64_t* start_off, int np,
                                 int64_t count, double tol, const double2* starts, double2* cand,
                                 uint8_t* status, uint16_t* seg, DevCounters* ctr, cudaStream_t s);
cudaError_t launch_seg_keys(const uint32_t* vals, const uint16_t* seg, const uint8_t* status,
                            int64_t count, uint64_t* keys, cudaStream_t s);

// a0: plain evaluation of P and P' at points.
cudaError_t launch_eval(const PolyDev& P, const double2* c, int64_t count, double2* out,
                        cudaStream_t s);

// a5: fold candidates and build sort keys.
cudaError_t launch_fold_keys(const uint8_t* status, double2* cand, int64_t count, double eps,
                             uint64_t* keys, uint32_t* vals, cudaStream_t s);
// the fold over list[0 .. *n_list) (entry t = candidate list[t]), the
// converged entries counted in *n_ok (zeroed here)
cudaError_t launch_fold_keys_list(const uint32_t* list, const unsigned long long* n_list, int64_t cap,
                                  const uint8_t* status, double2* cand, double eps, uint64_t* keys, uint32_t* vals,
                                  unsigned long long* n_ok, cudaStream_t s);

// Exclusive scan of u32 (in place allowed), with total written to *total.
size_t scan_temp_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, void* temp,
                                  unsigned long long* total, cudaStream_t s);

// LSD radix sort of (key, val) pairs on bits [0, 64).  The result ends in
// (keys, vals); (keys_alt, vals_alt) are scratch of the same size.
size_t radix_temp_bytes(int64_t n);
// n_dev: NULL, or a device count (at most n) of the entries to sort; the
// launches are sized for n
cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                             uint32_t* vals_alt, int64_t n, void* temp, cudaStream_t s,
                             const unsigned long long* n_dev = nullptr);
// Stable passes on bits [begin_bit, end_bit) only (multiples of 8); the
// result is in (keys, vals) after an even number of passes, else in the alt
// buffers (*in_alt = true).
cudaError_t radix_sort_bits(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                            int64_t n, void* temp, int begin_bit, int end_bit, bool* in_alt,
                            cudaStream_t s);

// Cluster pass on Re-sorted candidates: flag[p] = 1 if sorted candidate p
// starts a new root (no earlier candidate within the Chebyshev pixel).
cudaError_t launch_cluster(const double2* cand, const uint32_t* vals, int64_t count,
                           const unsigned long long* n_valid, double eps, uint32_t* flag,
                           DevCounters* ctr, cudaStream_t s, SegView sv = SegView());

// Gather flagged candidates into reps (order of the sort) and set n_reps.
cudaError_t launch_compact(const double2* cand, const uint32_t* vals, const uint32_t* flag,
                           const uint32_t* pos, int64_t count, double2* reps, DevCounters* ctr,
                           cudaStream_t s, SegView sv = SegView());

// a6: polish + type of each rep (upper half), multiplicities for emission.
cudaError_t launch_classify(const PolyDev& P, double2* reps, const unsigned long long* n_reps,
                            int64_t cap, double tau, int polish, uint8_t* type, uint32_t* mult,
                            DevCounters* ctr, cudaStream_t s, SegView sv = SegView());

// a7: certify reps (sorted by Re): radius from nearest neighbours, disk test.
// a6 + a7 in one pass for p_n (kind 0): type, conjugate multiplicity,
// certificate and radius of each representative (k_classify + k_certify).
cudaError_t launch_certify_typed(const PolyDev& P, const double2* reps, const unsigned long long* n_reps,
                                 int64_t cap, double tol, double tau, uint8_t* type, uint32_t* mult,
                                 uint8_t* pass, double* radius, DevCounters* ctr, cudaStream_t s);
cudaError_t launch_certify(const PolyDev& P, const double2* reps, const unsigned long long* n_reps,
                           int64_t cap, double tol, const uint32_t* mult, uint8_t* pass,
                           double* radius, DevCounters* ctr, cudaStream_t s,
                           SegView sv = SegView(), const uint8_t* type = nullptr);

// Emit the full conjugate-closed list sorted by (Re, Im).
cudaError_t launch_emit(const double2* reps, const unsigned long long* n_reps, int64_t cap_reps,
                        const uint32_t* mult, const uint32_t* pos, const uint8_t* type,
                        int mis_code, double2* out, uint8_t* is_mis, int64_t cap_out,
                        cudaStream_t s, SegView sv = SegView());
cudaError_t launch_fix_ties(double2* out, const unsigned long long* n_full, int64_t cap_out,
                            uint8_t* is_mis, cudaStream_t s, SegView sv = SegView(),
                            double2* out_lo = nullptr);

// Standalone type (a6 without polish) for mt_classify.
cudaError_t launch_type_only(const PolyDev& P, const double2* roots, int64_t count, double tau,
                             uint8_t* type, cudaStream_t s);

// Newton-basin certificate (Thm proofContract) of a list sorted through
// 'order', with the proven radii of the localisation test.
cudaError_t launch_basin(const PolyDev& P, const double2* pts, const uint32_t* order, int64_t count,
                         const double* radius, double eps_max, double* basin, DevCounters* ctr,
                         cudaStream_t s);

// Separation statistics, tier 1, over a list sorted by Re through 'order'
// (lo may be null): nn_out[i] (optional) = distance to the nearest other
// root of the (masked) list; band_min[0..63] = per-band minima, [64] =
// overall minimum (bit patterns of doubles), [65] = roots left to the strip
// tiers, listed in iso_idx / iso_best (room for n each) with the best
// distance found so far; [66] = roots left by tier 2 to tier 3.
cudaError_t launch_separation(const double2* hi, const double2* lo, const uint32_t* order, int64_t n,
                              const uint8_t* mask, double* nn_out, unsigned long long* band_min,
                              uint32_t* iso_idx, double* iso_best, cudaStream_t s);
// log2 of the strip count for n roots (about 16 per strip, 2^10 .. 2^20)
int separation_strips_log2(int64_t n);
// (Re strip, Im) index: keys / vals sorted (keys_alt, vals_alt, rtmp are
// the sort's scratch), offs [2^log2s + 1] = each strip's first entry
cudaError_t launch_strip_index(const double2* hi, int64_t n, int log2s, uint64_t* keys, uint32_t* vals,
                               uint64_t* keys_alt, uint32_t* vals_alt, void* rtmp, uint32_t* offs,
                               cudaStream_t s);
// tiers 2 and 3 over the niso roots of iso_idx / iso_best (iso2_*: room for
// niso roots passed from tier 2 to tier 3)
cudaError_t launch_separation_strips(const double2* hi, const double2* lo, const uint8_t* mask,
                                     const uint64_t* skeys, const uint32_t* sidx, const uint32_t* offs,
                                     int log2s, const uint32_t* iso_idx, const double* iso_best, int64_t niso,
                                     uint32_t* iso2_idx, double* iso2_best, double* nn_out,
                                     unsigned long long* band_min, cudaStream_t s);

// Emission's per-root byte: mis_code >= 0 writes 1 where the type code is
// mis_code (Mis(l,n) of s_{l,n}); MIS_CODE_RAW writes the type code itself
// (period k of p_n; k for Mis(l,k) / 32 + k for Hyp(k) of s_{l,n}).
constexpr int MIS_CODE_RAW = 256;

// q_{l,n} through its factors (eq. polySimple telescoped, q_{l,n} = p_n^2
// prod_{j=2..l} s_{j,n}): append the roots of one factor, with their type
// codes, to the union list.  j == 0: the factor p_n, every root, Hyp(k) of
// multiplicity floor((l-1)/k) + 2; else s_{j,n}, its Mis(j,k) roots (codes
// below 32), multiplicity 1.  Counts appended roots, their multiplicities,
// roots without a valid code and real roots (cnt[0] .. cnt[3]).
cudaError_t launch_qf_append(const double2* roots, const uint8_t* type, int64_t count, int j, int l, int n,
                             double2* u_roots, uint8_t* u_pre, uint8_t* u_per, uint8_t* u_mult, int64_t cap,
                             unsigned long long* cnt, cudaStream_t s);
// keys[p] = order-preserving key of Re (use_im: Im) of z[perm ? perm[p] : p],
// vals[p] = perm ? perm[p] : p, for p < *n_dev.
cudaError_t launch_qf_keys(const double2* z, const uint32_t* perm, int64_t cap, const unsigned long long* n_dev,
                           int use_im, uint64_t* keys, uint32_t* vals, cudaStream_t s);
// out[p] = u[perm[p]] for roots and the three type bytes (null outputs skipped).
cudaError_t launch_qf_gather(const uint32_t* perm, int64_t cap, const unsigned long long* n_dev,
                             const double2* u_roots, const uint8_t* u_pre, const uint8_t* u_per,
                             const uint8_t* u_mult, double2* roots, uint8_t* pre, uint8_t* per, uint8_t* mult,
                             cudaStream_t s);

// Zero the counters (min radius set to +inf).
cudaError_t launch_init_counters(DevCounters* ctr, cudaStream_t s);
// keys[i] = order-preserving key of Re pts[i], vals[i] = i.
cudaError_t launch_keys_plain(const double2* pts, int64_t count, uint64_t* keys, uint32_t* vals,
                              cudaStream_t s);
// q_{l,n}: exact type (preperiod, period) and multiplicity of each root.
cudaError_t launch_type_q(const PolyDev& P, const double2* roots, int64_t count, double tau, uint8_t* pre,
                          uint8_t* per, uint8_t* mult, cudaStream_t s);
// Standalone certificate of an arbitrary list sorted through 'order'
// (type: q_{l,n} only, the type codes of the points, or null).
cudaError_t check_sqrt_up(unsigned long long* n_fail, double* max_rel, cudaStream_t s);
cudaError_t launch_certify_list(const PolyDev& P, const double2* pts, const uint32_t* order,
                                int64_t count, double tol, uint8_t* pass, double* radius,
                                DevCounters* ctr, cudaStream_t s, const uint8_t* type = nullptr);

// ---- the double-double tier (mt_ddtier.cu) ----------------------------------
// dd values are pairs of binary64 (hi, lo), 16 bytes like a double2.
struct dd;
cudaError_t dd_collect_bad(const double2* reps, const unsigned long long* n_reps, int64_t cap,
                           const uint8_t* pass, const double* radius, double thr, double2* bad,
                           unsigned long long* nbad, int max_bad, cudaStream_t s);
cudaError_t dd_mark_pieces(const double2* cand, const uint8_t* status, int64_t S, int every,
                           int64_t Ls, int64_t npieces, const double2* bad, const uint64_t* klo,
                           const uint64_t* khi, int nbad, double R, uint32_t* flag, cudaStream_t s);
cudaError_t dd_mark_pieces_fix(const int2* candq, int64_t S, int every, int64_t Ls, int64_t npieces,
                               const double2* bad, int nbad, double R, uint32_t* flag, cudaStream_t s);
// streamed splits: walk of chunks [j0, j0 + nch) (starts from index j0 L / every
// written at 0), and the append of a piece's representatives to the list G
cudaError_t launch_walk_range(const PolyDev& P, double lambda0, int M, int every, int64_t L, int64_t nchunks,
                              int64_t j0, int64_t nch, const double2* seeds, double2* starts, DevCounters* ctr,
                              cudaStream_t s, int block);
cudaError_t launch_stream_append(const double2* cand, const uint8_t* status, const uint32_t* vals,
                                 const uint32_t* flag, const uint32_t* pos, int64_t count, double2* G,
                                 unsigned long long* g_count, int64_t g_cap, int2* candq, cudaStream_t s);
cudaError_t launch_piece_valid(const DevCounters* ctr, unsigned long long* snap, unsigned long long* n_valid,
                               cudaStream_t s);
cudaError_t dd_piece_ids(const uint32_t* flag, const uint32_t* pos, int64_t npieces, int64_t* ids,
                         int64_t ids_cap, cudaStream_t s);
cudaError_t dd_near_reps(const double2* reps, const unsigned long long* n_reps, int64_t cap,
                         const double2* bad, const uint64_t* klo, const uint64_t* khi, int nbad, double R,
                         uint32_t* near, unsigned long long* nnear, int64_t near_cap, cudaStream_t s);
cudaError_t dd_seeds(const PolyDev& P, double lambda0, int64_t NQ, int shrink, const int64_t* ids,
                     int64_t nb, uint32_t* cnt, uint32_t* off, void* scan_tmp, dd* sx, dd* sy,
                     DevCounters* ctr, cudaStream_t s);
cudaError_t dd_walk(const PolyDev& P, double lambda0, int M, int every, int64_t Ls, int64_t npieces,
                    const int64_t* ids, const uint32_t* off, int64_t nb, const dd* sx, const dd* sy,
                    dd* stx, dd* sty, uint8_t* st_ok, DevCounters* ctr, cudaStream_t s);
cudaError_t dd_descend(const PolyDev& P, int64_t count, const dd* zx0, const dd* zy0,
                       const uint8_t* ok0, double tol, int cap, const double2* bad, int nbad,
                       double R, dd* ox, dd* oy, unsigned long long* nout, int64_t out_cap,
                       DevCounters* ctr, cudaStream_t s);
cudaError_t dd_polish(const PolyDev& P, const double2* reps, const uint32_t* near,
                      const unsigned long long* nnear, int64_t near_cap, int64_t launch_n, double tol,
                      const double2* bad, int nbad, double R, double margin, uint8_t* drop, dd* ox,
                      dd* oy, unsigned long long* nout, int64_t out_cap, DevCounters* ctr,
                      cudaStream_t s);
cudaError_t dd_keys(const dd* zx, dd* zy, const unsigned long long* nz, int64_t zcap, double eps,
                    uint64_t* keys, uint32_t* vals, cudaStream_t s);
cudaError_t dd_cluster(const dd* zx, const dd* zy, const uint32_t* vals, const unsigned long long* nz,
                       int64_t zcap, double eps, uint32_t* flag, cudaStream_t s);
cudaError_t dd_compact(const dd* zx, const dd* zy, const uint32_t* vals, const uint32_t* flag,
                       const uint32_t* pos, int64_t zcap, dd* rx, dd* ry, cudaStream_t s);
cudaError_t dd_type_cert(const PolyDev& P, const dd* rx, const dd* ry, const unsigned long long* nz,
                         double tau, double tol, const double2* reps, const unsigned long long* n_main,
                         const uint8_t* drop, const double* radius, double wmax, uint8_t* type,
                         uint8_t* pass, uint32_t* mult, int64_t zcap, DevCounters* ctr,
                         cudaStream_t s);
cudaError_t dd_keep(const unsigned long long* n_reps, int64_t cap, const uint32_t* mult,
                    const uint8_t* drop, const uint8_t* type, const uint8_t* pass, uint32_t* kmult,
                    DevCounters* ctr, cudaStream_t s);
cudaError_t dd_emit(const double2* reps, const unsigned long long* n_reps, int64_t cap,
                    const uint32_t* kmult, const uint32_t* mpos, const unsigned long long* mt,
                    const uint8_t* type, int mis_code, const dd* zrx, const dd* zry,
                    const unsigned long long* nz, int64_t zcap, const uint32_t* zmult,
                    const uint32_t* zmpos, const unsigned long long* zt, const uint8_t* ztype,
                    double2* out, double2* out_lo, uint8_t* is_mis, int64_t cap_out,
                    DevCounters* ctr, cudaStream_t s);
cudaError_t dd_basin(const PolyDev& P, const double2* hi, const double2* lo, const uint32_t* order,
                     int64_t n, const double* radius, double eps_max, double* basin, DevCounters* ctr,
                     cudaStream_t s);
cudaError_t dd_certify_list(const PolyDev& P, const double2* hi, const double2* lo,
                            const uint32_t* order, int64_t n, double tol, uint8_t* pass,
                            double* radius, DevCounters* ctr, cudaStream_t s);

int device_sm_count();

// Set the thread-local message returned by mt_last_error().
void set_error_message(const char* msg);

// Kernel launches issued by this library on the calling thread (reported in
// mt_stats.n_launches).
extern thread_local unsigned long long g_launches;
#define MT_COUNT_LAUNCH(k) (::mt::g_launches += (k))

}  // namespace mt
