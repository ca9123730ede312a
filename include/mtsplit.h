/*
 * mtsplit.h -- C ABI of the GB300 level-line Newton splitter.
 *
 * Finds every root of the hyperbolic polynomials
 *     p_0 = 0,  p_{k+1}(c) = p_k(c)^2 + c,   deg p_n = 2^(n-1)
 * (Mihalache & Vigneron, "How to split a tera-polynomial", Sec. 1,
 * eq. def:hyp_poly) and of the simplified Misiurewicz polynomials
 *     s_{l,n} = q_{l,n} / q_{l-1,n} = p_{l+n-1} + p_{l-1},  deg = 2^(l+n-2)
 * (eq. polySimple, eq. polyMisSimple), with the method of Sec. 4:
 * a discrete level line |P| = lambda0 (eq. defDiscreteLev) walked with the
 * Newton-with-target map (Prop. computeLevelLine), Newton descents from
 * c_L points per root (Algorithm S_par), a separated sorted set of roots
 * (Sec. 6.1, eq. nsetAsumption), and a disk-arithmetic certificate per root
 * (Thm proofRoots, Thm diskArithmetic).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are DEVICE pointers (any CUDA allocation; the
 *    Python binding uses torch tensors).  The caller owns every buffer; the
 *    library never allocates or frees device memory.  Host pointers are
 *    named h_* or are plain scalars / structs.
 *  - Work runs asynchronously on opts->stream (a cudaStream_t; NULL = the
 *    legacy default stream).  Entry points that return counts (n_out,
 *    stats) synchronise that stream before returning.
 *  - Roots are complex128 in torch layout: d_roots[2*i] = Re, d_roots[2*i+1]
 *    = Im.  A split returns ALL roots of P (conjugates included, divisor
 *    periods included), sorted by (Re, Im) (eq. defLexi); real roots have
 *    Im = +0.0.  d_roots_lo (optional, same layout) receives the low parts
 *    of double-double roots (zeros in plain FP64 mode); the order is then
 *    that of the double-double values (roots whose Re hi parts are equal
 *    are ordered by their Re low parts first).
 *  - Workspace: d_work / work_bytes is caller-provided scratch of at least
 *    mt_workspace_bytes(...) bytes, 256-byte aligned.  Its contents are
 *    undefined on entry and on exit; calls sharing a workspace must be
 *    ordered on one stream.
 *  - Errors: no exception crosses the ABI.  Every function returns an
 *    mt_status; mt_last_error() gives a thread-local message for the last
 *    failure on the calling thread.
 */
#ifndef MTSPLIT_H
#define MTSPLIT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MT_API __attribute__((visibility("default")))
#else
#define MT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MT_OK = 0,
  MT_EINVAL = 1,       /* argument outside the domain (n, l, sizes, options)      */
  MT_ENOMEM = 2,       /* workspace smaller than mt_workspace_bytes()              */
  MT_ECAPACITY = 3,    /* cap < number of roots; *n_out holds the required size    */
  MT_ECUDA = 4,        /* a CUDA call failed (message in mt_last_error())          */
  MT_EINCOMPLETE = 5,  /* root count != degree after all retries                   */
  MT_ETIMEOUT = 6,     /* a bounded device scan (root-set clustering, certificate
                          neighbours) hit its cap and the result is incomplete or
                          uncertified                                           */
  MT_ECERT = 7         /* at least one root failed the disk certificate            */
} mt_status;

typedef enum {
  MT_FP64 = 0,   /* every step in binary64                                      */
  MT_MIXED = 1,  /* binary32 level-line tracking and early Newton, binary64 finish */
  MT_DD = 2      /* binary64 with double-double for the clustered roots          */
} mt_precision;

/* Options.  Fill with mt_default_options() and override fields. */
typedef struct {
  int prec;            /* mt_precision                                              */
  double tol;          /* Newton stop: |step| < tol (0 -> 1e-13 FP64, 1e-26 DD)     */
  double lambda0;      /* outer level (0 -> 5 for p_n, 100 for s_{l,n}; Sec. 4.2)   */
  int M;               /* level-line points per turn (0 -> 8; Sec. 6.3.1)          */
  int c_L;             /* descents per root (0 -> 4; Sec. 4.2)                      */
  int chunk_log2;      /* log2 of level-line points walked per lane (0 -> auto)     */
  int block;           /* CUDA block size for the Newton kernels (0 -> auto)        */
  int max_retries;     /* doublings of (M, c_L) when roots are missing (default 1;
                          they stop once M would exceed 64, and the last attempt's
                          result and status stand).  MT_MIXED and MT_DD first
                          repeat a failed attempt in binary64; a negative value
                          keeps the first attempt only (no repeat of any kind) */
  double eps_dup;      /* separation of the root set (0 -> rule of the library)     */
  double cert_tol;     /* certificate radius cap (0 -> 1e-12 FP64, 1e-20 DD)       */
  int use_graph;       /* 1: capture the launch sequence in a CUDA graph and replay */
  void* stream;        /* cudaStream_t                                              */
  /* MT_DD only.  A binary64 pass runs first; around each root whose
     certificate failed or needed a shrunken radius, the disk of radius
     dd_radius is redone in double-double (level-line chunks, descents,
     root set, types, certificates).  dd_all = 1 redoes every root. */
  double dd_radius;    /* zone radius (0 -> 1e-11 for p_n, n <= 29; else 1e-9)      */
  int dd_all;          /* 1: the whole split in double-double                       */
  /* Streamed split: the level line is walked and descended in this many
     pieces (a power of two), each piece's root set appended to one list
     whose own root set is the result; the starts never all reside in
     memory.  0 -> automatic: 1, or the fewest pieces of at most 2^28 starts
     once the upper half holds more than 2^31 starts (p_32 and up).
     Given explicitly, the pieces run in the requested tier; the automatic
     streaming runs its first attempt in binary64. */
  int stream_pieces;
} mt_options;

#define MT_MAX_TYPES 64

/* Counters of one call (host struct, filled before return). */
typedef struct {
  int64_t degree;          /* deg P                                               */
  int64_t n_roots;         /* distinct roots found (full list)                    */
  int64_t n_real;          /* real roots among them                               */
  int64_t n_starts;        /* descents started (upper half of the level line)     */
  int64_t n_conv;          /* descents that converged                             */
  int64_t n_repeat;        /* converged descents that hit an already found root   */
  int64_t n_diverge;       /* descents stopped by a long jump / non-finite value  */
  int64_t n_timeout;       /* descents stopped by the iteration cap               */
  int64_t walk_newton;     /* Newton steps on the level line (seeds + walk)       */
  int64_t desc_newton;     /* Newton steps in descents (all tiers)                */
  int64_t steps_fp32;      /* of which in binary32                                */
  int64_t steps_dd;        /* of which in double-double                           */
  int64_t walk_fail;       /* level-line chunks whose end missed the next seed    */
  int64_t n_cert_pass;     /* roots (full list) that passed the disk certificate  */
  int64_t count_by_type[MT_MAX_TYPES]; /* p_n: [k] = roots of exact period k;
                                          s_{l,n}: [k] = Mis(l,k), [32+k] = Hyp(k);
                                          q_{l,n}: the same, and [0] = Mis(j,k),
                                          j < l (distinct roots, full list)      */
  int32_t M, c_L;          /* values finally used                                  */
  int32_t retries;         /* (M, c_L) doublings performed                         */
  int32_t n_chunks;        /* level-line chunks (lanes of the walk)                */
  int64_t n_launches;      /* CUDA kernels launched by the call                    */
  double max_cert_radius;  /* largest certified radius                             */
  double min_cert_radius;  /* smallest certified radius                            */
  double eps_dup;          /* separation used                                      */
  float ms_total;          /* device time of the call (CUDA events)                */
  float ms_walk;           /* device time of seeds + level-line walk               */
  float ms_descend;        /* device time of the Newton descents                   */
  float ms_dedup;          /* device time of fold + sort + cluster + emit          */
  float ms_certify;        /* device time of classify + certify                    */
  int32_t prec_used;       /* tier of the attempt that produced the result
                              (MT_DD when a double-double pass ran)              */
  float ms_dd;             /* device time of the double-double pass                */
  int64_t n_zones;         /* double-double zone centres (0 in dd_all mode)        */
  int64_t n_zone_roots;    /* roots (upper half) produced by the dd pass           */
  int64_t n_dd_pieces;     /* 32-sub-step pieces of the level line redone in dd    */
  int64_t seed_newton;     /* Newton steps of the seed lifts (part of walk_newton) */
  int64_t desc_fp32;       /* binary32 Newton steps of the descents                */
  float ms_seeds;          /* device time of the seed lifts (part of ms_walk)      */
  int32_t reserved;
  int64_t n_finish;        /* binary64 finishes in the mixed tier (one per run of
                              descents that reached the same root in binary32)   */
  int64_t n_mult;          /* roots counted with multiplicity (q_{l,n}; n_roots
                              for the polynomials with simple roots)            */
  /* Device time of single kernels (CUDA events around their launches on the
     call's stream, also inside a captured graph), summed over their
     launches; 0 where the kernel did not run or was not timed.  For the
     roofline of each kernel against the FMA rate of its own pipe. */
  float ms_k_walk;         /* the level-line walk (k_walk / k_walk_mixed)         */
  float ms_k_desc64;       /* binary64 descents (k_descend; mixed tier: the tip redo) */
  float ms_k_desc32;       /* binary32 descents of the mixed tier (k_descend_mixed) */
  float ms_k_finish;       /* binary64 finish of the mixed tier (k_finish_f64)    */
  int64_t finish_newton;   /* binary64 Newton steps of k_finish_f64               */
  int32_t n_k_timed;       /* kernel launches timed in the four fields above      */
  int32_t n_tip64;         /* mixed tier: descents that ended within 1e-3 of the
                              left tip c = -2 and were redone in binary64 from
                              their start (Sec. 6.3.2: the tip roots close in
                              faster than binary32 resolves them)               */
  int64_t desc_orbit_steps; /* batched split: orbit steps summed over the descents'
                               Newton steps (the orbit length varies by polynomial;
                               0 for a single polynomial, whose is fixed)          */
  /* The first attempt of the call (before any (M, c_L) doubling or binary64
     repeat): its roots found, roots certified, level-line chunks that
     skipped a turn, and its tier (MT_DD when its double-double pass ran). */
  int64_t first_n_roots;
  int64_t first_n_cert_pass;
  int32_t first_walk_fail;
  int32_t first_prec;
} mt_stats;

/* Defaults documented field by field above. */
MT_API void mt_default_options(mt_options* opts);

/* deg p_n = 2^(n-1) (n in [1, 40]); -1 if out of range. */
MT_API int64_t mt_degree_hyperbolic(int n);
/* deg s_{l,n} = 2^(l+n-2) (l >= 2, n >= 1, l + n <= 41); -1 if out of range. */
MT_API int64_t mt_degree_misiurewicz(int l, int n);

/* Scratch bytes a split of P needs (kind 0: p_n, kind 1: s_{l,n}, kind 2:
   q_{l,n}) with these options; 0 if the arguments are invalid. */
MT_API size_t mt_workspace_bytes(int kind, int l, int n, const mt_options* opts);

/* Split p_n (Sec. 4.2, Algorithm S_par; hypQuick of Sec. 6.3.1).
   d_roots: [cap][2] doubles, receives all 2^(n-1) roots sorted by (Re, Im).
   d_roots_lo: NULL or [cap][2]: low parts in MT_DD mode.
   *n_out: number of roots written (or required size on MT_ECAPACITY).
   stats: optional.  Returns MT_EINCOMPLETE if roots are still missing after
   opts->max_retries doublings, MT_ECERT if a root failed its certificate. */
MT_API mt_status mt_split_hyperbolic(int n, const mt_options* opts, double* d_roots, double* d_roots_lo,
                              int64_t cap, void* d_work, size_t work_bytes, int64_t* n_out,
                              mt_stats* stats);

/* Split s_{l,n} = p_{l+n-1} + p_{l-1} (eq. polySimple; misSimpleQuick of
   Sec. 6.3.1).  d_is_mis: NULL or [cap] bytes, 1 where the root lies in
   Mis(l,n) (eq. def:mis), 0 for the other roots of s_{l,n} (Hyp(k),
   k | gcd(n, l-1), and Mis(l,k), k | n, k < n). */
MT_API mt_status mt_split_misiurewicz(int l, int n, const mt_options* opts, double* d_roots,
                               double* d_roots_lo, int64_t cap, uint8_t* d_is_mis, void* d_work,
                               size_t work_bytes, int64_t* n_out, mt_stats* stats);

/* Split q_{l,n} = p_{l+n} - p_l (eq. def:mis; misQuick of Sec. 6.3.1), whose
   roots are multiple (Thm fact_mis): Hyp(k), k | n, of multiplicity
   eta_l(k) = floor((l-1)/k) + 2, and Mis(j,k), 2 <= j <= l, k | n, simple.
   l >= 1, n >= 1, l + n <= 40.  opts->prec = MT_FP64: Newton descents on
   q itself (below); MT_DD: through its factors, q_{l,n} = p_n^2
   prod_{j=2..l} s_{j,n} (eq. polySimple telescoped from q_{0,n} = p_n, with
   s_{1,n} = p_n), each factor split by the certified double-double split of
   its own kind (mt_split_hyperbolic / mt_split_misiurewicz); Hyp(k) roots
   come from p_n, Mis(j,k) roots from s_{j,n}, the union sorted by (Re, Im)
   and every root certified as a simple root of its factor (the tip Mis
   points from order 20 on lie closer than binary64 descents on q resolve);
   MT_MIXED: MT_EINVAL.  d_roots: [cap][2] doubles, receives the distinct roots sorted
   by (Re, Im); *n_out their number.  d_mult, d_pre, d_per: NULL or [cap]
   bytes: multiplicity, preperiod j (0 for Hyp) and period k of each root
   (255 / 0 where no type matched).  Complete when the multiplicities add up
   to 2^(l+n-1) (stats->n_mult); else MT_EINCOMPLETE after the retries.
   Every root is certified (Thm proofRoots): in MT_FP64 a Mis root as a
   simple root of q, a Hyp root as a simple root of p_n (MT_ECERT if one
   fails); in MT_DD each root as a simple root of its factor.
   Descents on q that contract linearly take the multiplicity step of eq.
   newtonAcc; q is evaluated in the product form p_n prod_{j<=l} s_{j,n} of
   eq. polySimple, which keeps its relative accuracy up to a multiple root.
   Workspace: mt_workspace_bytes(2, l, n, opts) (for MT_DD: the largest
   factor's split plus the union list and its sort). */
MT_API mt_status mt_split_misiurewicz_q(int l, int n, const mt_options* opts, double* d_roots, int64_t cap,
                                        uint8_t* d_mult, uint8_t* d_pre, uint8_t* d_per, void* d_work,
                                        size_t work_bytes, int64_t* n_out, mt_stats* stats);

/* Split every s_{l,n} with l >= 2, n >= 1, l + n <= max_order in ONE pass:
   one persistent launch drains the level-line chunks of all polynomials,
   one persistent launch drains all descents.  Roots of pair number p (pairs
   ordered by l, then n) are d_roots[h_offsets[p] .. h_offsets[p+1]).
   h_offsets: host array of npairs + 1 entries (npairs = number of pairs).
   stats: optional array of npairs entries.
   mt_misiurewicz_pairs returns npairs for max_order and, when h_l and h_n
   are given, writes the first min(npairs, capacity) pairs (l, n) in that
   order (host arrays, no device work). */
MT_API int mt_misiurewicz_pairs(int max_order, int* h_l, int* h_n, int capacity);
MT_API size_t mt_workspace_bytes_misiurewicz_batch(int max_order, const mt_options* opts);
MT_API mt_status mt_split_misiurewicz_batch(int max_order, const mt_options* opts, double* d_roots,
                                     double* d_roots_lo, int64_t cap, uint8_t* d_is_mis,
                                     void* d_work, size_t work_bytes, int64_t* h_offsets,
                                     mt_stats* stats);

/* Certify given roots of P (kind 0: p_n, kind 1: s_{l,n}, kind 2: q_{l,n},
   binary64 only, a root typed Hyp(k) proven as a root of p_n) with the disk
   test of Thm proofRoots evaluated in disk arithmetic (Thm diskArithmetic):
   root j gets the radius r_j = min(tol, 0.45 * distance to the nearest other
   root or conjugate) and passes iff r_j * dist(0, B') > sup |P(c_j)| where
   B' encloses P'(D(c_j, r_j)).  Passing disks are pairwise disjoint, so
   count == degree with every root passing proves the list complete
   (Thm certif).  d_roots: [count][2] (any order); d_roots_lo: NULL or
   [count][2], the low parts of double-double roots (then the orbit runs in
   double-double and tol = 0 means 1e-20); d_pass: [count] bytes; d_radius:
   [count] doubles (NULL allowed).  *n_pass receives the number of passing
   roots. */
MT_API size_t mt_certify_workspace_bytes(int64_t count);
MT_API mt_status mt_certify(int kind, int l, int n, const double* d_roots, const double* d_roots_lo,
                     int64_t count, double tol, uint8_t* d_pass, double* d_radius, void* d_work,
                     size_t work_bytes, int64_t* n_pass, void* stream);

/* Newton-basin certificate (Thm proofContract; Thm certif, the radius
   eps_N of Fig. rootCertif): root j, proven by mt_certify to lie in
   D(c_j, r_j) (d_radius), gets the largest eps_j = min(eps_max, 0.25 nn_j)
   / 4^k with eps_j > 3 eta_j (eta_j <= r_j the localisation radius the
   disk test itself yields) such that P'(D(c_j, eps_j)) lies in a disk B'
   with dist(0, B') > 2 diam(B').  Then D(c_j, eps_j) lies in the basin of
   attraction of the root for the Newton map: Newton from any point of it
   converges to that root.  d_basin[j] = eps_j, or 0 where no radius passes
   (r_j = 0, or no eps above 3 eta_j).  d_roots_lo: NULL or the low parts
   (double-double centres).  eps_max: 0 -> 1e-6.  *n_pass: roots with a
   basin radius.  q_{l,n} (kind 2): MT_EINVAL, the theorem is for simple
   roots.  Workspace: mt_certify_workspace_bytes(count). */
MT_API mt_status mt_certify_basin(int kind, int l, int n, const double* d_roots, const double* d_roots_lo,
                                  int64_t count, const double* d_radius, double eps_max, double* d_basin,
                                  void* d_work, size_t work_bytes, int64_t* n_pass, void* stream);

/* Separation statistics of a root list (Sec. 6.3.2: the minimal distance
   within Hyp(n) is ~118.4 / 4^n, attained by the two left-most real roots;
   Fig. separationHistogram bins it over I_k = (-2 + 4^-(k+1), -2 + 4^-k]).
   d_roots: [count][2]; d_roots_lo: NULL or the low parts (distances then in
   double-double); d_mask: NULL or [count] bytes, the set = roots with
   mask != 0 (e.g. the exact period n from mt_classify).  Outputs, all
   optional: d_nn [count] doubles, the distance from each root of the set
   to its nearest other root of the set (0 outside the set, +inf if it is
   alone); h_band_min [64] host doubles, per band k the smallest d_nn over
   the set's roots with Re c + 2 in (4^-(k+1), 4^-k] (band 0 also takes
   Re c + 2 > 1, band 63 everything below 4^-63; +inf if empty); *h_min the
   smallest over the set.  Entries must be finite.  Three tiers, each
   settling some roots and handing the rest on with their best distance so
   far as a bound: a scan of up to 64 neighbours in the list sorted by Re,
   then a walk in Im over a (Re strip, Im) index (one thread per root), then
   the same walk with one block per root for isolated roots.  The index only
   chooses which pairs are compared, so every distance is exact.  Errors: MT_EINVAL (negative count, count above
   2^32 - 1, null roots), MT_ENOMEM (workspace smaller than
   mt_separation_workspace_bytes(count)), MT_ECUDA.  Synchronises the
   stream before returning. */
MT_API size_t mt_separation_workspace_bytes(int64_t count);
MT_API mt_status mt_separation(int64_t count, const double* d_roots, const double* d_roots_lo,
                               const uint8_t* d_mask, double* d_nn, double* h_band_min,
                               double* h_min, void* d_work, size_t work_bytes, void* stream);

/* Autotuner (the paper tunes nothing; a GPU-layout choice).  Runs complete
   splits of P for each candidate level-line chunk length 2^c (c = 3 .. 10
   sub-steps per lane) and walk block size (32, 64, 128), three runs each,
   and keeps the fastest in a process-wide table keyed by (kind, l, n,
   tier).  Later calls whose options leave chunk_log2 / block at 0 use the
   tuned values.  d_roots, cap, d_work, work_bytes are those of a split;
   candidates whose workspace exceeds work_bytes are skipped.  Outputs:
   best chunk_log2, block size and device milliseconds (any may be NULL). */
MT_API mt_status mt_autotune(int kind, int l, int n, const mt_options* opts, double* d_roots,
                             int64_t cap, void* d_work, size_t work_bytes, int* best_chunk_log2,
                             int* best_block, float* best_ms);

/* ---- single steps of the path, exposed for parity checks ---------------- */

/* Orbit evaluation (Sec. 1, eq. def:hyp_poly, and its c-derivative): for
   each point d_c[2i], d_c[2i+1], writes d_out[4i..4i+3] = Re P, Im P,
   Re P', Im P' in binary64 (q_{l,n}: the product form of eq. polySimple).
   No workspace. */
MT_API mt_status mt_eval(int kind, int l, int n, const double* d_c, int64_t count, double* d_out,
                  void* stream);

/* Steps a1-a3 only: real end point, lifted seeds and the level-line walk.
   d_starts: [cap][2], receives the (c_L/2) d + 1 starts of the upper half of
   the discrete level line L_{lambda0, c_L d}(P) (eq. defDiscreteLev) in
   external-angle order, start s satisfying P = lambda0 e^{2 i pi s / c_L}. */
MT_API mt_status mt_level_line(int kind, int l, int n, const mt_options* opts, double* d_starts,
                        int64_t cap, void* d_work, size_t work_bytes, int64_t* n_starts,
                        mt_stats* stats);

/* Step a4 only: Newton descent (eq. Newton) from each start, capped at
   max{20, I_N log2 d}.  d_out: [count][2] final iterate; d_status: [count]
   bytes (0 converged, 1 divergent, 2 timeout). */
MT_API mt_status mt_descend(int kind, int l, int n, const mt_options* opts, const double* d_starts,
                     int64_t count, double* d_out, uint8_t* d_status, void* d_work,
                     size_t work_bytes, mt_stats* stats);

/* Step a6 only: type of each root (eq. def:hyp / def:mis), d_type[i] =
   period k for p_n, or k (Mis(l,k)) / 32 + k (Hyp(k)) for s_{l,n} and
   q_{l,n}, and 0 for Mis(j,k), j < l, of q_{l,n}; 255 if no type was
   recognised.  tau: Newton-size threshold (0 -> default). */
MT_API mt_status mt_classify(int kind, int l, int n, const double* d_roots, int64_t count, double tau,
                      uint8_t* d_type, void* stream);

/* ---- certificate without any device allocation --------------------------- */

/* Largest list mt_certify_static accepts, and the size of the device array
   that holds its scratch. */
#define MT_CERTIFY_STATIC_MAX_ROOTS 131072
#define MT_CERTIFY_STATIC_BYTES (4u << 20)

/* The certificate of mt_certify for callers that cannot allocate device
   memory -- code running in a host callback or an allocator hook, or a
   plug-in inside a process whose device memory belongs to another
   runtime's pool.  They pass only the roots and the output arrays; there
   is no workspace argument and no allocation of any kind.  (The paper has
   no counterpart: this is a deployment variant of mt_certify.)
   Arguments and results are those of mt_certify (without d_roots_lo and
   the workspace) for kinds 0 (p_n) and 1 (s_{l,n}); kind 2 (q_{l,n}) returns
   MT_EINVAL.  d_roots [count][2] device, d_pass [count] device bytes,
   d_radius [count] device doubles or NULL, *n_pass host.
   The scratch is one static device array of MT_CERTIFY_STATIC_BYTES that
   every GPU loading the library keeps until the process exits; count above
   MT_CERTIFY_STATIC_MAX_ROOTS returns MT_ECAPACITY.  The first call on a
   device looks up that array's device address (with the device current);
   make that first call before any stream capture.  All calls share the
   array, so calls that overlap on the GPU race: order them (one stream, or
   synchronise between them).  Synchronises 'stream' before returning. */
MT_API mt_status mt_certify_static(int kind, int l, int n, const double* d_roots, int64_t count,
                                   double tol, uint8_t* d_pass, double* d_radius, int64_t* n_pass,
                                   void* stream);

/* ---- measurement ------------------------------------------------------- */

/* FMA issue rate of the current GPU in TFLOP/s (2 flops per FMA): every SM
   runs independent FMA chains (x <- x a + b) in binary64 (prec = MT_FP64)
   or binary32 (prec = MT_MIXED) for a fixed number of rounds, timed with
   CUDA events on 'stream'.  The denominator of the ALU roofline of the
   Newton kernels, whose bound is the FMA pipe of their precision (the paper
   has no counterpart; it times a CPU).  d_work: at least
   mt_fma_peak_workspace_bytes() bytes (the chains' final values).
   Synchronises 'stream'. */
MT_API size_t mt_fma_peak_workspace_bytes(void);
MT_API mt_status mt_fma_peak(int prec, void* d_work, size_t work_bytes, double* tflops, void* stream);

/* Self-check of the certificate's binary32 square-root upper bound (Thm
   proofRoots needs upper bounds of |z| and |p'|; the disk orbit takes them
   as sqrt.approx.f32 times 1 + 2^-19, rounded upward): over every normal
   binary32 x, *n_fail = how many x have bound^2 < x (exact in binary64;
   0 means the bound holds on this GPU) and *max_rel = the largest relative
   error of the approximation itself.  Runs on 'stream' (about 2^31
   evaluations, a few milliseconds) and synchronises it. */
MT_API mt_status mt_check_sqrt_up(unsigned long long* n_fail, double* max_rel, void* stream);

/* Thread-local message of the last failure ("" if none). */
MT_API const char* mt_last_error(void);

/* Library version string. */
MT_API const char* mt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MTSPLIT_H */
